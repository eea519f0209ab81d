// Fused D2Q5 IREBM step: Algorithm 3 on the D2Q5 lattice (Sec. 3.2), the
// lattice the paper writes its 2D closures for (Sec. 4.2).
//
// Velocities 0 rest, 1 (+1,0), 2 (0,+1), 3 (-1,0), 4 (0,-1); weights 1/3 and
// 1/6 (c_s^2 = 1/3).  The state is the post-collision population Omega_i
// (Eq. 12) in five SoA planes.  For every node y a step does
//   pull       q_0 = Omega_0(y), q_1 = Omega_1(y - e_x), q_3 = Omega_3(y + e_x),
//              q_2 = Omega_2(y - e_y), q_4 = Omega_4(y + e_y)
//   closures   the one unknown q_i of a wall node (two at a corner):
//              Dirichlet, Eq. (16) (Eq. 15 shared by weight at a corner);
//              adiabatic, bounce-back (Sec. 4.2.2) or the Neumann closure of
//              Eq. (17), M0(q) = M0(q) of the node one step inwards
//   moments    m0 = sum_i q_i, theta = sum_i Omega_i(y) (= M0(f))
//   Newton     theta' = root of Eq. (14), deferred to the job kernel as for D2Q9
//   update     Omega~_i = (1 - omega) q_i + w_i (theta' - (1 - omega) m0)
//
// Work unit: a warp tile of one segment of 32 N consecutive columns (N = 4
// floats or 2 doubles per lane, one 128-bit load per plane and row) by tile_h
// rows.  The warp walks up its rows: plane 2 is pulled from the row below
// (kept in registers from the previous row), plane 4 from the row above
// (loaded with the previous row and kept for this row's moments), planes 0, 1
// and 3 from the row itself, 1 and 3 shifted along x through warp shuffles
// with one element fetched beyond each end of the segment.  The next row's
// loads are issued before this row's arithmetic.  Every population is read
// once per step, plus one halo row of planes 2 and 4 per tile: 20 + 20 bytes
// per node in FP32, 40 + 40 in FP64.
#include "step_common.cuh"

namespace lbm {

#ifndef LBM_D2Q5_NF
#define LBM_D2Q5_NF 4   // floats per lane (FP32 form)
#endif
#ifndef LBM_D2Q5_ND
#define LBM_D2Q5_ND 2   // doubles per lane (FP64 form)
#endif
template <typename P> struct V5;
template <> struct V5<float> { static constexpr int N = LBM_D2Q5_NF; };
template <> struct V5<double> { static constexpr int N = LBM_D2Q5_ND; };

__device__ __forceinline__ void d5_ld(const float* p, float (&v)[4])
{
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void d5_ld(const float* p, float (&v)[2])
{
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void d5_ld(const double* p, double (&v)[2])
{
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void d5_ld(const double* p, double (&v)[1]) { v[0] = __ldg(p); }

// ---------------------------------------------------------------- closures
// A D2Q5 wall node (nx, ny >= 3): q_1 is unknown at x = 0, q_3 at x = nx - 1,
// q_2 at y = 0, q_4 at y = ny - 1.
struct Wall5 {
    unsigned unk;   // bit i: q_i not defined by streaming
    int wall;       // Dirichlet wall (first of W, E, S, N), -1 if none
    int sx, sy;     // Eq. (17): the node one step inwards (the diagonal one at a corner)
};

__device__ __forceinline__ Wall5 wall5_info(int x, int y, const Problem& pb)
{
    Wall5 w;
    const bool W = x == 0, E = x == pb.nx - 1, S = y == 0, N = y == pb.ny - 1;
    w.unk = (W ? 2u : 0u) | (S ? 4u : 0u) | (E ? 8u : 0u) | (N ? 16u : 0u);
    const int walls = (W ? 1 : 0) | (E ? 2 : 0) | (S ? 4 : 0) | (N ? 8 : 0);
    w.wall = -1;
    for (int k = 0; k < 4; ++k)
        if (((walls >> k) & 1) && pb.wall_kind[k] == 1) {
            w.wall = k;
            break;
        }
    w.sx = x + (W ? 1 : (E ? -1 : 0));
    w.sy = y + (S ? 1 : (N ? -1 : 0));
    return w;
}

// The streamed populations of an interior node (x, y), read from the source state.
template <typename P>
__device__ __forceinline__ void pulled5(const P* __restrict__ src, const Problem& pb, int x, int y, P (&q)[5])
{
    const long long pl = pb.plane, pitch = pb.pitch;
    const P* r = src + (long long)(y + 1) * pitch + x;
    q[0] = r[0];
    q[1] = r[pl - 1];
    q[2] = r[2 * pl - pitch];
    q[3] = r[3 * pl + 1];
    q[4] = r[4 * pl + pitch];
}

// FP64 form.  q holds the pulled values (unknown entries are overwritten), u
// the node's own Omega.  Returns the boundary flux (filled q minus Omega that
// leaves the lattice); wall reports the node's Dirichlet wall or -1.
__device__ __noinline__ double wall5_closure_d(double* q, const double* u, int x, int y, const Problem& pb,
                                               const double* __restrict__ src, int& wall)
{
    const Wall5 wi = wall5_info(x, y, pb);
    wall = wi.wall;
    double out = 0.0, in = 0.0;
#pragma unroll
    for (int j = 1; j < 5; ++j)
        if ((wi.unk >> d2_opp(j)) & 1) out += u[j];
    if (wi.wall >= 0 || pb.bb_mode == 2) {
        double m0t;
        if (wi.wall >= 0) {
            double th = 0.0;
#pragma unroll
            for (int i = 4; i >= 0; --i) th += u[i];
            m0t = dir_m0_target_d(th, wi.wall, pb);
        } else {
            double nq[5];
            pulled5<double>(src, pb, wi.sx, wi.sy, nq);
            m0t = 0.0;
#pragma unroll
            for (int i = 4; i >= 0; --i) m0t += nq[i];
        }
        // the unknown q share what the known ones leave, in proportion to w_i (equal)
        double known = 0.0;
        int nu = 0;
#pragma unroll
        for (int i = 4; i >= 0; --i) {
            if ((wi.unk >> i) & 1) ++nu;
            else known += q[i];
        }
        const double r = (m0t - known) / (double)nu;
#pragma unroll
        for (int i = 1; i < 5; ++i)
            if ((wi.unk >> i) & 1) {
                q[i] = r;
                in += r;
            }
    } else {
        // bounce-back: the opposite direction is always known on D2Q5 with nx, ny >= 3
#pragma unroll
        for (int i = 1; i < 5; ++i)
            if ((wi.unk >> i) & 1) {
                const int o = d2_opp(i);
                q[i] = pb.bb_mode == 0 ? q[o] : u[o];
                in += q[i];
            }
    }
    return in - out;
}

// FP32 form with float-float sums.
__device__ __noinline__ ff wall5_closure_f(float* q, const float* u, int x, int y, const Problem& pb,
                                           const float* __restrict__ src, int& wall)
{
    const Wall5 wi = wall5_info(x, y, pb);
    wall = wi.wall;
    ff out{0.f, 0.f}, in{0.f, 0.f};
#pragma unroll
    for (int j = 1; j < 5; ++j)
        if ((wi.unk >> d2_opp(j)) & 1) ff_add(out, u[j]);
    if (wi.wall >= 0 || pb.bb_mode == 2) {
        ff m0t{0.f, 0.f};   // target of M0(q), less the state's shift sh (q, u are Omega - w_i sh)
        if (wi.wall >= 0) {
            const float sh = __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(src) + pb.tail_off));
            ff th{0.f, 0.f};
#pragma unroll
            for (int i = 4; i >= 0; --i) ff_add(th, u[i]);
            ff_add(th, sh);
            m0t = dir_m0_target_f(th, wi.wall, pb);
            ff_add(m0t, -sh);
        } else {
            float nq[5];
            pulled5<float>(src, pb, wi.sx, wi.sy, nq);
#pragma unroll
            for (int i = 4; i >= 0; --i) ff_add(m0t, nq[i]);
        }
        ff known{0.f, 0.f};
        int nu = 0;
#pragma unroll
        for (int i = 4; i >= 0; --i) {
            if ((wi.unk >> i) & 1) ++nu;
            else ff_add(known, q[i]);
        }
        const float r = ((m0t.hi - known.hi) + (m0t.lo - known.lo)) / (float)nu;
#pragma unroll
        for (int i = 1; i < 5; ++i)
            if ((wi.unk >> i) & 1) {
                q[i] = r;
                ff_add(in, r);
            }
    } else {
#pragma unroll
        for (int i = 1; i < 5; ++i)
            if ((wi.unk >> i) & 1) {
                const int o = d2_opp(i);
                q[i] = pb.bb_mode == 0 ? q[o] : u[o];
                ff_add(in, q[i]);
            }
    }
    ff f{in.hi, in.lo};
    ff_add(f, -out.hi);
    f.lo -= out.lo;
    return f;
}

// ---------------------------------------------------------------- one row
// The update of one row of the warp's segment.  qf: pulled q (closed here at
// wall nodes), u: the nodes' own Omega.  EDGE = false: the caller knows that
// the row has no wall node and no column beyond nx in this segment.
template <typename P, int N, bool REC, bool EDGE>
__device__ __forceinline__ void row5_update(const Problem& pb, const P* __restrict__ src, P* __restrict__ drow,
                                            int y, int x0, int lane, P (&qf)[5][N], const P (&u)[5][N],
                                            double* __restrict__ rec, Acc<P>& acc, TileSums& ts, int pi,
                                            NewtonJob* jobs, unsigned int* job_count, const P omc, const float om_f,
                                            const double omc_d, const P w0, const P w1, const float thr_f)
{
    const int nx = pb.nx, ny = pb.ny;
    const long long pl = pb.plane;
    // the state's shift (FP32 form: the stored values are Omega_i - w_i sh; 0 in FP64)
    const float sh = sizeof(P) == 4 ? __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(src) + pb.tail_off))
                                    : 0.f;
    P c[N];
    double thn[REC ? N : 1];
    bool newton_k[N], dir_k[N];
    int wall_k[N];
    typename M0T<P>::T m0[N];
#pragma unroll
    for (int k = 0; k < N; ++k) { dir_k[k] = false; wall_k[k] = -1; }
    if constexpr (EDGE) {
        bool any_wall = false;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int x = x0 + k;
            any_wall |= (x < nx) && (x == 0 || x == nx - 1 || y == 0 || y == ny - 1);
        }
        if (any_wall) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const int x = x0 + k;
                if (x < nx && (x == 0 || x == nx - 1 || y == 0 || y == ny - 1)) {
                    P qq[5], uu[5];
#pragma unroll
                    for (int i = 0; i < 5; ++i) { qq[i] = qf[i][k]; uu[i] = u[i][k]; }
                    if constexpr (sizeof(P) == 4) {
                        const ff fl = wall5_closure_f(qq, uu, x, y, pb, src, wall_k[k]);
                        ff_add(ts.flux_f, fl.hi);
                        ts.flux_f.lo += fl.lo;
                    } else {
                        ts.flux += wall5_closure_d(qq, uu, x, y, pb, src, wall_k[k]);
                    }
                    dir_k[k] = wall_k[k] >= 0;
#pragma unroll
                    for (int i = 0; i < 5; ++i) qf[i][k] = qq[i];
                }
            }
        }
    }

    bool any_newton = false;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int x = x0 + k;
        const bool valid = !EDGE || x < nx;
        float tf = 0.f, mf = 0.f;
        if constexpr (sizeof(P) == 4) {
            // a plain FP32 sum decides saturation and gives theta' = m0 there, to the
            // rounding of the stored populations; float-float sums only where needed
#pragma unroll
            for (int i = 4; i >= 0; --i) { tf += u[i][k]; mf += qf[i][k]; }
            tf += sh;   // theta; mf stays M0(q) - sh
        } else {
            m0_init(m0[k]);
#pragma unroll
            for (int i = 4; i >= 0; --i) { tf += approx_float(u[i][k]); m0_add(m0[k], qf[i][k]); }
            mf = m0_f(m0[k]);
        }
        const float mt = mf + sh;   // M0(q)
        const float marg = 1e-5f * (1.0f + fabsf(tf));
        const bool sat_liq = tf >= thr_f + marg && mt >= thr_f + marg;
        const bool sat_sol = tf <= -thr_f - marg && mt <= -thr_f - marg;
        newton_k[k] = valid && !dir_k[k] && !(sat_liq || sat_sol);
        any_newton |= newton_k[k];
        if (!valid) {
            c[k] = (P)0;
            if constexpr (REC) thn[k] = 0.0;
#pragma unroll
            for (int i = 0; i < 5; ++i) qf[i][k] = (P)0;
        } else if (dir_k[k]) {
            // theta' = theta_D; c = theta_D - (1 - omega) m0
            const int wk = wall_k[k];
            ts.dir_count[wk] += 1;
            if constexpr (sizeof(P) == 4) {
                ff mm{0.f, 0.f};
#pragma unroll
                for (int i = 4; i >= 0; --i) ff_add(mm, qf[i][k]);
                const float oc = (float)omc;
                c[k] = (P)(((pb.wall_th_hi[wk] - sh) - oc * mm.hi) + (pb.wall_th_lo[wk] - oc * mm.lo));
                acc.add_ff(ff{pb.wall_th_hi[wk], pb.wall_th_lo[wk]});
            } else {
                c[k] = (P)(pb.wall_theta[wk] - omc_d * m0_d(m0[k]));
                acc.add_d(pb.wall_theta[wk]);
            }
            if constexpr (REC) thn[k] = pb.wall_theta[wk];
        } else if (!newton_k[k]) {
            // saturated: theta' = m0, no source; c = omega m0
            if constexpr (sizeof(P) == 4) {
                c[k] = (P)(om_f * mf);   // less omega sh
                acc.add_f(mf);           // less sh
                ts.shifted += 1;
                if constexpr (REC) thn[k] = (double)mf + (double)sh;
            } else {
                const double md = m0_d(m0[k]);
                c[k] = (P)(pb.omega * md);
                acc.add_d(md);
                if constexpr (REC) thn[k] = md;
            }
            ts.liquid += sat_liq ? 1 : 0;
        }
    }
    if (__any_sync(kFull, any_newton)) {
        // deferred Newton solves: append (m0, theta) to the job list, store q_i unrelaxed
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) cnt += newton_k[k] ? 1 : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(job_count, (unsigned)total);
        base = __shfl_sync(kFull, base, 0);
        unsigned slot = base + (unsigned)(incl - cnt);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (!newton_k[k]) continue;
            NewtonJob jb;
            jb.prob = pi;
            jb.node = y * nx + x0 + k;
            if constexpr (sizeof(P) == 4) {
                // FP32 form: the job kernel forms m0 and theta from memory
                jb.m0 = jb.theta = 0.0;
            } else {
                double th = 0.0;
#pragma unroll
                for (int i = 4; i >= 0; --i) th += u[i][k];
                jb.m0 = m0_d(m0[k]);
                jb.theta = th;
            }
            jobs[slot] = jb;
            ++slot;
            c[k] = (P)0;
            if constexpr (REC) thn[k] = 0.0;
        }
    }

    // Omega~_i = (1 - omega) q_i + w_i c
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const P wi = i == 0 ? w0 : w1;
        P o[N];
#pragma unroll
        for (int k = 0; k < N; ++k) o[k] = newton_k[k] ? qf[i][k] : fma(omc, qf[i][k], wi * c[k]);
        stv_n(drow + i * pl, o);
    }
    if constexpr (REC) st_rec<N>(rec + (long long)y * pb.pitch + x0, thn);
}

// EEBM row update (Algorithm 2 in the stored-Omega form, as for D2Q9): after
// the pulls and the closures (Dirichlet target M0(q) = H(theta_D); Eq. 17 and
// bounce-back unchanged), H = M0(q), theta = Theta(H), and
// Omega~_i = (1-omega) q_i + omega w_i theta (i != 0),
// Omega~_0 = (1-omega) q_0 + omega (H - (1-w_0) theta).  No Newton node; the
// energy is the sum of H.
template <typename P, int N, bool REC, bool EDGE>
__device__ __forceinline__ void row5_update_eebm(const Problem& pb, const P* __restrict__ src, P* __restrict__ drow,
                                                 int y, int x0, P (&qf)[5][N], const P (&u)[5][N],
                                                 double* __restrict__ rec, Acc<P>& acc, TileSums& ts, const P omc,
                                                 const P w0, const P w1)
{
    const int nx = pb.nx, ny = pb.ny;
    const long long pl = pb.plane;
    if constexpr (EDGE) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int x = x0 + k;
            if (x < nx && (x == 0 || x == nx - 1 || y == 0 || y == ny - 1)) {
                P qq[5], uu[5];
                int wall;
#pragma unroll
                for (int i = 0; i < 5; ++i) { qq[i] = qf[i][k]; uu[i] = u[i][k]; }
                if constexpr (sizeof(P) == 4) {
                    const ff fl = wall5_closure_f(qq, uu, x, y, pb, src, wall);
                    ff_add(ts.flux_f, fl.hi);
                    ts.flux_f.lo += fl.lo;
                } else {
                    ts.flux += wall5_closure_d(qq, uu, x, y, pb, src, wall);
                }
#pragma unroll
                for (int i = 0; i < 5; ++i) qf[i][k] = qq[i];
            }
        }
    }
    const P om = (P)1 - omc;
    const P inv_ste = (P)pb.inv_ste;
    // the state's shift in enthalpy units (FP32 form; 0 in FP64)
    const P sh = sizeof(P) == 4 ? (P)__ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(src) + pb.tail_off))
                                : (P)0;
    P hs = 0;
    double thn[REC ? N : 1];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const bool valid = !EDGE || x0 + k < nx;
        P Hs = 0;   // H less the shift
#pragma unroll
        for (int i = 4; i >= 0; --i) Hs += qf[i][k];
        if (!valid) {
            Hs = 0;
#pragma unroll
            for (int i = 0; i < 5; ++i) qf[i][k] = (P)0;
        }
        hs += Hs;
        if constexpr (sizeof(P) == 4) ts.shifted += valid ? 1 : 0;
        const P H = Hs + sh;
        const P th = eebm_theta(H, inv_ste);
        if constexpr (REC) thn[k] = (double)th;
        // stored values less w_i sh
        qf[0][k] = fma(omc, qf[0][k], om * (H - ((P)1 - w0) * th - w0 * sh));
#pragma unroll
        for (int i = 1; i < 5; ++i) qf[i][k] = fma(omc, qf[i][k], om * w1 * (th - sh));
    }
    if constexpr (sizeof(P) == 4) acc.add_ff(ff{hs, 0.f});
    else acc.add_d(hs);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        P o[N];
#pragma unroll
        for (int k = 0; k < N; ++k) o[k] = qf[i][k];
        stv_n(drow + i * pl, o);
    }
    if constexpr (REC) st_rec<N>(rec + (long long)y * pb.pitch + x0, thn);
}

// ---------------------------------------------------------------- warp tile
template <typename P, bool REC>
__device__ __forceinline__ void d2q5_tile(const Problem& pb, const P* __restrict__ src, P* __restrict__ dst,
                                          double* __restrict__ rec, int seg, int ya, int yb, Acc<P>& acc,
                                          TileSums& ts, int pi, NewtonJob* jobs, unsigned int* job_count)
{
    constexpr int N = V5<P>::N;
    const int lane = threadIdx.x & 31;
    const int segx = seg * 32 * N;
    const int x0 = segx + lane * N;
    const long long pl = pb.plane;
    const long long pitch = pb.pitch;
    const bool has_left = segx > 0;
    const bool has_right = segx + 32 * N < pb.nx;
    const bool seg_interior = has_left && has_right;   // no wall column, every node inside
    // problem constants, converted once per tile
    const P omc = (P)(1.0 - pb.omega);
    const float om_f = pb.omega_f;
    const double omc_d = 1.0 - pb.omega;
    const P w0 = lat_wp<P>(5, 0), w1 = lat_wp<P>(5, 1);
    const float thr_f = pb.sat_f;
    const int ny = pb.ny;

    auto rp = [&](int i, int r) -> const P* { return src + i * pl + (long long)(r + 1) * pitch + x0; };
    auto hl = [&](int i, int r) -> P {
        return (lane == 0 && has_left) ? __ldg(src + i * pl + (long long)(r + 1) * pitch + segx - 1) : (P)0;
    };
    auto hr = [&](int i, int r) -> P {
        return (lane == 31 && has_right) ? __ldg(src + i * pl + (long long)(r + 1) * pitch + segx + 32 * N) : (P)0;
    };

    // plane 2 of the row below the tile (pulled into its first row) and plane 4
    // of the first row (its own Omega_4)
    P up2[N], cu4[N];
    d5_ld(rp(2, ya - 1), up2);
    d5_ld(rp(4, ya), cu4);
    // loads of one row: planes 0..3 at row y, plane 4 at row y + 1, and the
    // elements beyond the segment for the planes shifted along x
    struct RowLoads {
        P r0[N], r1[N], r2[N], r3[N], n4[N];
        P h1, h3;
    };
    auto issue = [&](RowLoads& L, int y) {
        d5_ld(rp(0, y), L.r0);
        d5_ld(rp(1, y), L.r1);
        d5_ld(rp(2, y), L.r2);
        d5_ld(rp(3, y), L.r3);
        d5_ld(rp(4, y + 1), L.n4);
        L.h1 = hl(1, y);
        L.h3 = hr(3, y);
    };
    RowLoads cur;
    issue(cur, ya);
    for (int y = ya; y < yb; ++y) {
        RowLoads nxt;
        if (y + 1 < yb) issue(nxt, y + 1);
        P qf[5][N], u[5][N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            qf[0][k] = cur.r0[k]; qf[2][k] = up2[k]; qf[4][k] = cur.n4[k];
            u[0][k] = cur.r0[k]; u[1][k] = cur.r1[k]; u[2][k] = cur.r2[k]; u[3][k] = cur.r3[k]; u[4][k] = cu4[k];
        }
        from_left<P, N>(cur.r1, cur.h1, lane, qf[1]);
        from_right<P, N>(cur.r3, cur.h3, lane, qf[3]);
        P* drow = dst + (long long)(y + 1) * pitch + x0;
        if (pb.method == 1)
            row5_update_eebm<P, N, REC, true>(pb, src, drow, y, x0, qf, u, rec, acc, ts, omc, w0, w1);
        else if (seg_interior && y > 0 && y < ny - 1)
            row5_update<P, N, REC, false>(pb, src, drow, y, x0, lane, qf, u, rec, acc, ts, pi, jobs, job_count, omc,
                                          om_f, omc_d, w0, w1, thr_f);
        else
            row5_update<P, N, REC, true>(pb, src, drow, y, x0, lane, qf, u, rec, acc, ts, pi, jobs, job_count, omc,
                                         om_f, omc_d, w0, w1, thr_f);
        // roll the register window
#pragma unroll
        for (int k = 0; k < N; ++k) { up2[k] = cur.r2[k]; cu4[k] = cur.n4[k]; }
        cur = nxt;
    }
}

// Four resident 128-thread blocks per SM (at most 128 registers, a few values
// spilled to L1): measured on the 4096^2 cavity, 0.159 ms per FP32 launch
// against 0.198 ms uncapped (168 registers, three blocks) and 0.177 ms with two
// floats per lane
#ifndef LBM_D2Q5_MIN_BLOCKS
#define LBM_D2Q5_MIN_BLOCKS 4
#endif

template <typename P, bool REC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, LBM_D2Q5_MIN_BLOCKS) d2q5_step_kernel(StepArgs a)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int slot = warp; slot < a.nslots; slot += nwarps) {
        int pi, t;
        if (a.schedule) {
            const int2 s = a.schedule[slot];
            pi = s.x;
            t = s.y;
        } else {
            pi = 0;
            t = slot;
        }
        const Problem& pb = a.probs[pi];
        DevStats* st = &a.stats[pb.stats];
        const int seg = t % pb.nseg;
        const int strip = t / pb.nseg;
        const int ya = strip * pb.tile_h;
        const int yb = min(pb.ny, ya + pb.tile_h);
        Acc<P> acc;
        TileSums ts;
        d2q5_tile<P, REC>(pb, static_cast<const P*>(pb.state[a.parity]), static_cast<P*>(pb.state[a.parity ^ 1]),
                          a.rec, seg, ya, yb, acc, ts, pi, a.jobs, a.job_count);
        flush_tile_sums<P>(acc, ts, st, lane);
    }
    // statistics are published by the job kernel that follows every step
}

int d2q5_segment_width(int precision) { return precision == 1 ? 32 * V5<float>::N : 32 * V5<double>::N; }

cudaError_t launch_d2q5_step(int precision, const StepArgs& a, cudaStream_t s)
{
    const int grid = (a.nslots + kWarpsPerBlock - 1) / kWarpsPerBlock;   // one tile per warp
    if (grid <= 0) return cudaErrorInvalidValue;
    if (precision == 1) {
        if (a.rec) d2q5_step_kernel<float, true><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
        else d2q5_step_kernel<float, false><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
    } else {
        if (a.rec) d2q5_step_kernel<double, true><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
        else d2q5_step_kernel<double, false><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace lbm
