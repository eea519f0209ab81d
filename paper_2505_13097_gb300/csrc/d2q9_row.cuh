// Row update of the D2Q9 step kernels, shared by the warp-tile kernel
// (FP64 form, the no-allocation step), the TMA row-pipeline kernel (FP32
// batches) and the wall rows of the flat FP32 step:
// the boundary closures of Sec. 4.2 at wall nodes, the moments, the exact
// saturated branch, the hand-off of nodes that need the local Newton solve of
// Eq. (14), and the relaxation toward the next step's Omega (Eq. 12).
#pragma once

#include "step_common.cuh"

namespace lbm {

// Boundary closures of Sec. 4.2 at one wall node (x, y).  q holds the pulled
// values (entries of unknown directions are overwritten), u the node's own
// Omega.  Returns the boundary flux contribution (filled q minus Omega that
// leaves the lattice) as a float-float pair; wall reports the node's Dirichlet
// wall (first in W, E, S, N) or -1.
struct WallInfo {
    unsigned unk;   // bit i: q_i not defined by streaming
    int wall;       // Dirichlet wall index, -1 for bounce-back
};

__device__ __forceinline__ WallInfo wall_info(int x, int y, const Problem& pb)
{
    WallInfo w;
    w.unk = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int sx = x - d2_ex(i), sy = y - d2_ey(i);
        if (sx < 0 || sx >= pb.nx || sy < 0 || sy >= pb.ny) w.unk |= 1u << i;
    }
    const int walls = (x == 0 ? 1 : 0) | (x == pb.nx - 1 ? 2 : 0) | (y == 0 ? 4 : 0) | (y == pb.ny - 1 ? 8 : 0);
    w.wall = -1;
    for (int k = 0; k < 4; ++k)
        if (((walls >> k) & 1) && pb.wall_kind[k] == 1) {
            w.wall = k;
            break;
        }
    return w;
}

// FP64 form: the closure in FP64.
static __device__ __noinline__ double wall_closure_d(double* q, const double* u, int x, int y, const Problem& pb, int& wall)
{
    const WallInfo wi = wall_info(x, y, pb);
    wall = wi.wall;
    double out = 0.0, in = 0.0;
#pragma unroll
    for (int j = 1; j < 9; ++j)
        if ((wi.unk >> d2_opp(j)) & 1) out += u[j];
    if (wi.wall >= 0) {
        // Eq. (14) with theta' = theta_D fixes M0(q) = theta_D + (phi(theta_D) - phi(theta))/Ste;
        // the unknown q share what the known ones leave, in proportion to w_i
        double th = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) th += u[i];
        const double m0t = dir_m0_target_d(th, wi.wall, pb);
        double known = 0.0, wu = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if ((wi.unk >> i) & 1) wu += d2_w(i);
            else known += q[i];
        }
        const double r = (m0t - known) / wu;
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if ((wi.unk >> i) & 1) {
                q[i] = d2_w(i) * r;
                in += q[i];
            }
    } else {
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if ((wi.unk >> i) & 1) {
                const int o = d2_opp(i);
                q[i] = (pb.bb_mode == 0 && !((wi.unk >> o) & 1)) ? q[o] : u[o];
                in += q[i];
            }
    }
    return in - out;
}

// FP32 form: the same closure with float-float sums and no FP64 instruction on
// the common path (dir_m0_target_f).  q and u hold Omega less w_i sh (the
// state's shift): theta = sum u + sh, and the unknown q share the target less sh.
static __device__ __noinline__ ff wall_closure_f(float* q, const float* u, int x, int y, const Problem& pb, int& wall,
                                                 float sh)
{
    const WallInfo wi = wall_info(x, y, pb);
    wall = wi.wall;
    ff out{0.f, 0.f}, in{0.f, 0.f};
#pragma unroll
    for (int j = 1; j < 9; ++j)
        if ((wi.unk >> d2_opp(j)) & 1) ff_add(out, u[j]);
    if (wi.wall >= 0) {
        const int k = wi.wall;
        ff th{0.f, 0.f}, known{0.f, 0.f};
        float wu = 0.f;
#pragma unroll
        for (int i = 8; i >= 0; --i) {
            ff_add(th, u[i]);
            if ((wi.unk >> i) & 1) wu += d2_wf(i);
            else ff_add(known, q[i]);
        }
        ff_add(th, sh);
        ff m0t = dir_m0_target_f(th, k, pb);
        ff_add(m0t, -sh);
        // R = m0t - sum(known), shared by the unknown q in proportion to w_i
        const float r = ((m0t.hi - known.hi) + (m0t.lo - known.lo)) / wu;
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if ((wi.unk >> i) & 1) {
                q[i] = d2_wf(i) * r;
                ff_add(in, q[i]);
            }
    } else {
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if ((wi.unk >> i) & 1) {
                const int o = d2_opp(i);
                q[i] = (pb.bb_mode == 0 && !((wi.unk >> o) & 1)) ? q[o] : u[o];
                ff_add(in, q[i]);
            }
    }
    ff f{in.hi, in.lo};
    ff_add(f, -out.hi);
    f.lo -= out.lo;
    return f;
}


template <typename P>
__device__ __forceinline__ float approx_sum(const P* u);
template <>
__device__ __forceinline__ float approx_sum<float>(const float* u)
{
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) s += u[i];
    return s;
}
template <>
__device__ __forceinline__ float approx_sum<double>(const double* u)
{
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) s += approx_float(u[i]);
    return s;
}

// Nodes whose local Newton solve is deferred go to a sink: reserve(total,
// lane) returns (to every lane) the first of `total` consecutive slots, and
// put(slot, job) stores one job.  The global job list below is solved by
// newton_jobs_kernel after the step.
struct GlobalJobSink {
    NewtonJob* jobs;
    unsigned int* count;
    __device__ __forceinline__ unsigned reserve(unsigned total, int lane)
    {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(count, total);
        return __shfl_sync(kFull, base, 0);
    }
    __device__ __forceinline__ void put(unsigned slot, const NewtonJob& j) const { jobs[slot] = j; }
};

// Everything of one row after the pulls: wall closures, moments, the exact
// saturated branch, hand-off of Newton nodes to the sink, relaxation and
// stores (Omega~_i = (1-omega) q_i + w_i c with c = theta' - (1-omega) m0).
// A Newton node's q_i are stored unrelaxed; whoever solves it relaxes them in
// place.
template <typename P, int N>
struct GlobalRowOut {
    P* row;          // dst + (y + 1) * pitch + x0
    long long pl;
    __device__ __forceinline__ void store(int i, const P (&o)[N]) const { stv_n(row + i * pl, o); }
};

template <typename P, int N, bool REC, bool EDGE, typename Out, typename Sink>
__device__ __forceinline__ void row_update(const Problem& pb, int y, int x0, int lane, P (&qf)[9][N], const P (&u0)[N],
                                           const P (&u1)[N], const P (&u2)[N], const P (&u3)[N], const P (&u4)[N],
                                           const P (&u5)[N], const P (&u6)[N], const P (&u7)[N], const P (&u8)[N],
                                           const Out& out, double* __restrict__ rec, Acc<P>& acc, TileSums& ts,
                                           int pi, Sink& sink, const P omc,
                                           const float om_f, const double omc_d, const P (&wP)[3], const float thr_f,
                                           const int nx, const int ny, const float sh)
{
    // sh: the state's shift (FP32 form; the stored values are Omega_i - w_i sh)
    const long long pitch = pb.pitch;
    P c[N];          // per node: theta' - (1-omega) m0, rounded to P
    double thn[REC ? N : 1];
    bool newton_k[N];
    typename M0T<P>::T m0[N];
    bool any_wall = false;
    bool dir_k[N];
    int wall_k[N];
#pragma unroll
    for (int k = 0; k < N; ++k) { dir_k[k] = false; wall_k[k] = -1; }
    if constexpr (EDGE) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int x = x0 + k;
            any_wall |= (x < nx) && (x == 0 || x == nx - 1 || y == 0 || y == ny - 1);
        }
    }
    // EDGE = false: the caller knows the warp's row has no wall node and no node beyond nx
    if (EDGE && __any_sync(kFull, any_wall)) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int x = x0 + k;
            if (x < nx && (x == 0 || x == nx - 1 || y == 0 || y == ny - 1)) {
                P qq[9], uu[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) qq[i] = qf[i][k];
                uu[0] = u0[k]; uu[1] = u1[k]; uu[2] = u2[k]; uu[3] = u3[k]; uu[4] = u4[k];
                uu[5] = u5[k]; uu[6] = u6[k]; uu[7] = u7[k]; uu[8] = u8[k];
                if constexpr (sizeof(P) == 4) {
                    const ff fl = wall_closure_f(qq, uu, x, y, pb, wall_k[k], sh);
                    ff_add(ts.flux_f, fl.hi);
                    ts.flux_f.lo += fl.lo;
                } else {
                    ts.flux += wall_closure_d(qq, uu, x, y, pb, wall_k[k]);
                }
                dir_k[k] = wall_k[k] >= 0;
#pragma unroll
                for (int i = 0; i < 9; ++i) qf[i][k] = qq[i];
            }
        }
    }

    bool any_newton = false;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int x = x0 + k;
        const bool valid = !EDGE || x < nx;
        const P u[9] = {u0[k], u1[k], u2[k], u3[k], u4[k], u5[k], u6[k], u7[k], u8[k]};
        const float tf = sizeof(P) == 4 ? approx_sum<P>(u) + sh : approx_sum<P>(u);
        float mf;   // FP32 form: M0(q) less sh
        if constexpr (sizeof(P) == 4) {
            // FP32 form: a plain FP32 sum (small weights first) decides saturation and
            // gives theta' = m0 there, to the rounding of the stored populations; the
            // float-float sum is formed only where it is needed (Newton and
            // Dirichlet nodes)
            mf = 0.f;
#pragma unroll
            for (int i = 8; i >= 0; --i) mf += qf[i][k];
        } else {
            m0_init(m0[k]);
#pragma unroll
            for (int i = 8; i >= 0; --i) m0_add(m0[k], qf[i][k]);
            mf = m0_f(m0[k]);
        }
        const float mt = sizeof(P) == 4 ? mf + sh : mf;   // M0(q)
        const float marg = 1e-5f * (1.0f + fabsf(tf));
        const bool sat_liq = tf >= thr_f + marg && mt >= thr_f + marg;
        const bool sat_sol = tf <= -thr_f - marg && mt <= -thr_f - marg;
        newton_k[k] = valid && !dir_k[k] && !(sat_liq || sat_sol);
        any_newton |= newton_k[k];
        if (!valid) {
            c[k] = (P)0;
            if constexpr (REC) thn[k] = 0.0;
#pragma unroll
            for (int i = 0; i < 9; ++i) qf[i][k] = (P)0;
        } else if (dir_k[k]) {
            // theta' = theta_D; c = theta_D - (1-omega) m0
            const int wk = wall_k[k];
            ts.dir_count[wk] += 1;
            if constexpr (sizeof(P) == 4) {
                ff mm;
                m0_init(mm);
#pragma unroll
                for (int i = 8; i >= 0; --i) ff_add(mm, qf[i][k]);
                const float oc = (float)omc;
                // c less omega sh: (theta_D - sh) - (1-omega) M0(q less sh)
                c[k] = (P)(((pb.wall_th_hi[wk] - sh) - oc * mm.hi) + (pb.wall_th_lo[wk] - oc * mm.lo));
                acc.add_ff(ff{pb.wall_th_hi[wk], pb.wall_th_lo[wk]});
            } else {
                c[k] = (P)(pb.wall_theta[wk] - omc_d * m0_d(m0[k]));
                acc.add_d(pb.wall_theta[wk]);
            }
            if constexpr (REC) thn[k] = pb.wall_theta[wk];
        } else if (!newton_k[k]) {
            // saturated: theta' = m0, no source; c = omega * m0
            if constexpr (sizeof(P) == 4) {
                // less the shift: c - omega sh = omega (m0 - sh); the energy term m0 - sh
                c[k] = (P)(om_f * mf);
                acc.add_f(mf);
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
    const bool row_newton = __any_sync(kFull, any_newton);
    if (row_newton) {
        // The local Newton solve of these nodes is deferred to the job kernel,
        // which spreads the FP64 work of the front band over the whole GPU:
        // append (m0, theta) to the job list and store q_i unrelaxed.
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
        const unsigned base = sink.reserve((unsigned)total, lane);
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
                const P u[9] = {u0[k], u1[k], u2[k], u3[k], u4[k], u5[k], u6[k], u7[k], u8[k]};
                double th = 0.0;
#pragma unroll
                for (int i = 8; i >= 0; --i) th += u[i];
                jb.m0 = m0_d(m0[k]);
                jb.theta = th;
            }
            sink.put(slot, jb);
            ++slot;
            c[k] = (P)0;
            if constexpr (REC) thn[k] = 0.0;
        }
    }

    // Omega~_i = (1-omega) q_i + w_i c, with w_i c formed once per weight class;
    // Newton nodes are stored unrelaxed (only rows that have some test for them)
    P wc[3][N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        wc[0][k] = wP[0] * c[k];
        wc[1][k] = wP[1] * c[k];
        wc[2][k] = wP[2] * c[k];
    }
    if (row_newton) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int cl = i == 0 ? 0 : (i <= 4 ? 1 : 2);
            P o[N];
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = newton_k[k] ? qf[i][k] : fma(omc, qf[i][k], wc[cl][k]);
            out.store(i, o);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int cl = i == 0 ? 0 : (i <= 4 ? 1 : 2);
            P o[N];
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = fma(omc, qf[i][k], wc[cl][k]);
            out.store(i, o);
        }
    }
    if constexpr (REC) {
        st_rec<N>(rec + (long long)y * pitch + x0, thn);
    }

}

// EEBM row update (Algorithm 2 in the stored-Omega form): after the pulls and
// the closures (Dirichlet target M0(q) = H(theta_D)), H = M0(q) is the
// enthalpy, theta = Theta(H), and the collision relaxes toward the modified
// equilibrium, Omega~_i = (1-omega) q_i + omega w_i theta for i != 0 and
// Omega~_0 = (1-omega) q_0 + omega (H - (1-w_0) theta).  No Newton node; the
// energy is the sum of H.
template <typename P, int N, bool REC, bool EDGE, typename Out>
__device__ __forceinline__ void row_update_eebm(const Problem& pb, int y, int x0, P (&qf)[9][N], const P (&u0)[N],
                                                const P (&u1)[N], const P (&u2)[N], const P (&u3)[N],
                                                const P (&u4)[N], const P (&u5)[N], const P (&u6)[N],
                                                const P (&u7)[N], const P (&u8)[N], const Out& out,
                                                double* __restrict__ rec, Acc<P>& acc, TileSums& ts, const P omc,
                                                const P (&wP)[3], const int nx, const int ny, const float sh)
{
    // sh: the state's shift in enthalpy units (FP32 form; stored Omega_i - w_i sh)
    const long long pitch = pb.pitch;
    if constexpr (EDGE) {
        bool any_wall = false;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int x = x0 + k;
            any_wall |= (x < nx) && (x == 0 || x == nx - 1 || y == 0 || y == ny - 1);
        }
        if (__any_sync(kFull, any_wall)) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const int x = x0 + k;
                if (x < nx && (x == 0 || x == nx - 1 || y == 0 || y == ny - 1)) {
                    P qq[9], uu[9];
                    int wall;
#pragma unroll
                    for (int i = 0; i < 9; ++i) qq[i] = qf[i][k];
                    uu[0] = u0[k]; uu[1] = u1[k]; uu[2] = u2[k]; uu[3] = u3[k]; uu[4] = u4[k];
                    uu[5] = u5[k]; uu[6] = u6[k]; uu[7] = u7[k]; uu[8] = u8[k];
                    if constexpr (sizeof(P) == 4) {
                        const ff fl = wall_closure_f(qq, uu, x, y, pb, wall, sh);
                        ff_add(ts.flux_f, fl.hi);
                        ts.flux_f.lo += fl.lo;
                    } else {
                        ts.flux += wall_closure_d(qq, uu, x, y, pb, wall);
                    }
#pragma unroll
                    for (int i = 0; i < 9; ++i) qf[i][k] = qq[i];
                }
            }
        }
    }
    const P om = (P)1 - omc;
    const P inv_ste = (P)pb.inv_ste;
    P hs = 0;
    double thn[REC ? N : 1];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const bool valid = !EDGE || x0 + k < nx;
        P Hs = 0;   // H less the shift (FP32 form)
#pragma unroll
        for (int i = 8; i >= 0; --i) Hs += qf[i][k];
        if (!valid) {
            Hs = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) qf[i][k] = (P)0;
        }
        hs += Hs;
        if constexpr (sizeof(P) == 4) {
            const float H = Hs + sh;
            const float th = eebm_theta(H, inv_ste);
            if constexpr (REC) thn[k] = (double)th;
            ts.shifted += valid ? 1 : 0;
            // stored values less w_i sh: omega (H - (1-w_0) theta - w_0 sh) and omega w_i (theta - sh)
            qf[0][k] = fma(omc, qf[0][k], om * (H - ((P)1 - wP[0]) * th - wP[0] * sh));
            const float tr = th - sh;
#pragma unroll
            for (int i = 1; i < 9; ++i) qf[i][k] = fma(omc, qf[i][k], om * (i <= 4 ? wP[1] : wP[2]) * tr);
        } else {
            const P H = Hs;
            const P th = eebm_theta(H, inv_ste);
            if constexpr (REC) thn[k] = (double)th;
            qf[0][k] = fma(omc, qf[0][k], om * (H - ((P)1 - wP[0]) * th));
#pragma unroll
            for (int i = 1; i < 9; ++i) qf[i][k] = fma(omc, qf[i][k], om * (i <= 4 ? wP[1] : wP[2]) * th);
        }
    }
    if constexpr (sizeof(P) == 4) acc.add_ff(ff{hs, 0.f});
    else acc.add_d(hs);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        P o[N];
#pragma unroll
        for (int k = 0; k < N; ++k) o[k] = qf[i][k];
        out.store(i, o);
    }
    if constexpr (REC) st_rec<N>(rec + (long long)y * pitch + x0, thn);
}

}  // namespace lbm
