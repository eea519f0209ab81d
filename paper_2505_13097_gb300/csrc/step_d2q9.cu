// Fused D2Q9 IREBM step: one kernel launch per time step of Algorithm 3.
//
// The state is the post-collision population Omega_i (Eq. 12), SoA planes.
// For every node y a step does
//   pull       q_i(y) = Omega_i(y - e_i)                       (Algorithm 3, streaming)
//   closures   missing q_i at wall nodes (Sec. 4.2, Eq. 15 and bounce-back)
//   moments    m0 = sum_i q_i, theta(y) = sum_i Omega_i(y)       (sum Omega = M0(f))
//   Newton     theta' = root of Eq. (14) from theta (Algorithm 3)
//   update     f~_i = q_i + w_i (phi(theta) - phi(theta'))/Ste  (Eq. 13)
//   collision  Omega~_i = (1-omega) f~_i + omega w_i theta'     (Eq. 12 of the next step)
// which folds into Omega~_i = (1-omega) q_i + w_i c with c = theta' - (1-omega) m0.
//
// Work unit: a warp tile = one segment of 32*N consecutive x nodes (N = 4
// floats or 2 doubles per thread, one 128-bit load per plane and row) times
// tile_h rows.  The warp marches up its rows keeping the rows it still needs
// in registers: planes with e_y = +1 are pulled from row y-1 (kept from the
// previous row), planes with e_y = -1 from row y+1 (loaded one row ahead and
// kept for the moments of the next row).  Shifts by e_x = +-1 go through warp
// shuffles; lanes 0 and 31 fetch the one element beyond the segment.  Every
// population is read once and written once per step (plus one halo row per
// tile for the six planes with e_y != 0).
//
// FP32 form: populations stored and relaxed in FP32; m0 and theta summed as
// float-float (exact to ~2^-48); the Newton solve in FP64.  Nodes where theta
// and m0 both lie beyond kSat*delta on the same side of the melting point
// take the exact saturated branch (phi = 0 or 1 on both sides of Eq. 14, so
// theta' = m0 and the source vanishes) without any FP64 work.
// FP64 form: everything in FP64 (the saturation test uses the integer pipe).
#include "step_common.cuh"

namespace lbm {

template <typename P> struct Vw;
template <> struct Vw<float> { static constexpr int N = 4; };
template <> struct Vw<double> { static constexpr int N = 2; };

template <typename P>
__device__ __forceinline__ void ldv(const P* p, P (&v)[Vw<P>::N]);
template <>
__device__ __forceinline__ void ldv<float>(const float* p, float (&v)[4])
{
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ldv<double>(const double* p, double (&v)[2])
{
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
}
template <typename P>
__device__ __forceinline__ void stv(P* p, const P (&v)[Vw<P>::N]);
template <>
__device__ __forceinline__ void stv<float>(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void stv<double>(double* p, const double (&v)[2])
{
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}


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
__device__ __noinline__ double wall_closure_d(double* q, const double* u, int x, int y, const Problem& pb, int& wall)
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
// the common path (dir_m0_target_f).
__device__ __noinline__ ff wall_closure_f(float* q, const float* u, int x, int y, const Problem& pb, int& wall)
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
            if ((wi.unk >> i) & 1) wu += (float)d2_w(i);
            else ff_add(known, q[i]);
        }
        const ff m0t = dir_m0_target_f(th, k, pb);
        // R = m0t - sum(known), shared by the unknown q in proportion to w_i
        const float r = ((m0t.hi - known.hi) + (m0t.lo - known.lo)) / wu;
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if ((wi.unk >> i) & 1) {
                q[i] = (float)d2_w(i) * r;
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


// ---------------------------------------------------------------- row ring
// Each warp streams its rows through a ring of kStages row slots in shared
// memory with cp.async (16-byte copies that bypass L1), so several rows are in
// flight per warp without holding registers.  A slot holds one row of all nine
// planes (32*N values each) plus the one element left and right of the
// segment for the planes that are shifted along x.  Row y is computed from the
// slots of rows y-1, y and y+1; the load of row y+kStages-1 is then issued into
// the slot of row y-1.  Waits are cp.async.wait_group (no spinning).
#ifndef LBM_RING_STAGES
#define LBM_RING_STAGES 5
#endif
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 4
#endif
constexpr int kStages = LBM_RING_STAGES;

template <typename P>
struct Ring {
    static constexpr int N = Vw<P>::N;
    static constexpr int ROW = 32 * N;                  // values per plane row
    static constexpr int HALO = 9 * ROW;                // offset of the halo values
    static constexpr int SLOT = (9 * ROW + 18 + 3) / 4 * 4;   // values per slot, 16-byte multiple
    static constexpr int WARP_BYTES = kStages * SLOT * (int)sizeof(P);
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

// Issue the copies of row r (-1 .. ny) of all planes into `slot`.
template <typename P>
__device__ __forceinline__ void ring_load(P* slot, const P* src, long long pl, long long pitch, int r, int segx,
                                          int lane, bool has_left, bool has_right)
{
    using R = Ring<P>;
    const P* row = src + (long long)(r + 1) * pitch + segx;
#pragma unroll
    for (int i = 0; i < 9; ++i) cp_async16(slot + i * R::ROW + lane * R::N, row + i * pl + lane * R::N);
    if (lane == 0 && has_left) {
        // planes shifted along +x (1, 5, 8) pull the element left of the segment
        cp_async_small<sizeof(P)>(slot + R::HALO + 2 * 1, row + 1 * pl - 1);
        cp_async_small<sizeof(P)>(slot + R::HALO + 2 * 5, row + 5 * pl - 1);
        cp_async_small<sizeof(P)>(slot + R::HALO + 2 * 8, row + 8 * pl - 1);
    }
    if (lane == 31 && has_right) {
        // planes shifted along -x (3, 6, 7) pull the element right of the segment
        cp_async_small<sizeof(P)>(slot + R::HALO + 2 * 3 + 1, row + 3 * pl + R::ROW);
        cp_async_small<sizeof(P)>(slot + R::HALO + 2 * 6 + 1, row + 6 * pl + R::ROW);
        cp_async_small<sizeof(P)>(slot + R::HALO + 2 * 7 + 1, row + 7 * pl + R::ROW);
    }
}

template <typename P>
__device__ __forceinline__ void lds(const P* p, P (&v)[Vw<P>::N]);
template <>
__device__ __forceinline__ void lds<float>(const float* p, float (&v)[4])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void lds<double>(const double* p, double (&v)[2])
{
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x; v[1] = t.y;
}

// Everything of one row after the pulls: wall closures, moments, the exact
// saturated branch, deferral of Newton nodes to the job list, relaxation and
// stores (Omega~_i = (1-omega) q_i + w_i c with c = theta' - (1-omega) m0).
// Row outputs: straight to the plane rows in global memory, or to a row buffer
// in shared memory that a TMA bulk store writes out.
template <typename P, int N>
struct GlobalRowOut {
    P* row;          // dst + (y + 1) * pitch + x0
    long long pl;
    __device__ __forceinline__ void store(int i, const P (&o)[N]) const { stv_n(row + i * pl, o); }
};

template <typename P, int N, bool REC, bool EDGE, typename Out>
__device__ __forceinline__ void row_update(const Problem& pb, int y, int x0, int lane, P (&qf)[9][N], const P (&u0)[N],
                                           const P (&u1)[N], const P (&u2)[N], const P (&u3)[N], const P (&u4)[N],
                                           const P (&u5)[N], const P (&u6)[N], const P (&u7)[N], const P (&u8)[N],
                                           const Out& out, double* __restrict__ rec, Acc<P>& acc, TileSums& ts,
                                           DevStats* st, int pi, NewtonJob* jobs, unsigned int* job_count, const P omc,
                                           const float om_f, const double omc_d, const P (&wP)[3], const float thr_f,
                                           const int nx, const int ny)
{
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
                    const ff fl = wall_closure_f(qq, uu, x, y, pb, wall_k[k]);
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
    float row_m0 = 0.f;   // FP32 form: sum of theta' = m0 over this lane's saturated nodes
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int x = x0 + k;
        const bool valid = !EDGE || x < nx;
        const P u[9] = {u0[k], u1[k], u2[k], u3[k], u4[k], u5[k], u6[k], u7[k], u8[k]};
        const float tf = approx_sum<P>(u);
        float mf;
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
        const float marg = 1e-5f * (1.0f + fabsf(tf));
        const bool sat_liq = tf >= thr_f + marg && mf >= thr_f + marg;
        const bool sat_sol = tf <= -thr_f - marg && mf <= -thr_f - marg;
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
                c[k] = (P)((pb.wall_th_hi[wk] - oc * mm.hi) + (pb.wall_th_lo[wk] - oc * mm.lo));
                acc.add_ff(ff{pb.wall_th_hi[wk], pb.wall_th_lo[wk]});
            } else {
                c[k] = (P)(pb.wall_theta[wk] - omc_d * m0_d(m0[k]));
                acc.add_d(pb.wall_theta[wk]);
            }
            if constexpr (REC) thn[k] = pb.wall_theta[wk];
        } else if (!newton_k[k]) {
            // saturated: theta' = m0, no source; c = omega * m0
            if constexpr (sizeof(P) == 4) {
                c[k] = (P)(om_f * mf);
                row_m0 += mf;
                if constexpr (REC) thn[k] = (double)mf;
            } else {
                const double md = m0_d(m0[k]);
                c[k] = (P)(pb.omega * md);
                acc.add_d(md);
                if constexpr (REC) thn[k] = md;
            }
            ts.liquid += sat_liq ? 1 : 0;
        }
    }
    if constexpr (sizeof(P) == 4) acc.add_ff(ff{row_m0, 0.f});
    if (__any_sync(kFull, any_newton)) {
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
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(job_count, (unsigned)total);
        base = __shfl_sync(kFull, base, 0);
        unsigned slot = base + (unsigned)(incl - cnt);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (!newton_k[k]) continue;
            const P u[9] = {u0[k], u1[k], u2[k], u3[k], u4[k], u5[k], u6[k], u7[k], u8[k]};
            NewtonJob jb;
            jb.prob = pi;
            jb.node = y * nx + x0 + k;
            if constexpr (sizeof(P) == 4) {
                ff t, mm;
                m0_init(t);
                m0_init(mm);
#pragma unroll
                for (int i = 8; i >= 0; --i) {
                    ff_add(t, u[i]);
                    ff_add(mm, qf[i][k]);
                }
                float* pm = reinterpret_cast<float*>(&jb.m0);
                float* pt = reinterpret_cast<float*>(&jb.theta);
                pm[0] = mm.hi; pm[1] = mm.lo;
                pt[0] = t.hi; pt[1] = t.lo;
            } else {
                double th = 0.0;
#pragma unroll
                for (int i = 8; i >= 0; --i) th += u[i];
                jb.m0 = m0_d(m0[k]);
                jb.theta = th;
            }
            jobs[slot] = jb;
            ++slot;
            c[k] = (P)0;
            if constexpr (REC) thn[k] = 0.0;
        }
    }

    // Omega~_i = (1-omega) q_i + w_i c
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const P wi = i == 0 ? wP[0] : (i <= 4 ? wP[1] : wP[2]);
        P o[N];
#pragma unroll
        for (int k = 0; k < N; ++k) o[k] = newton_k[k] ? qf[i][k] : fma(omc, qf[i][k], wi * c[k]);
        out.store(i, o);
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
                                                const P (&wP)[3], const int nx, const int ny)
{
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
                        const ff fl = wall_closure_f(qq, uu, x, y, pb, wall);
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
        P H = 0;
#pragma unroll
        for (int i = 8; i >= 0; --i) H += qf[i][k];
        if (!valid) {
            H = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) qf[i][k] = (P)0;
        }
        const P th = eebm_theta(H, inv_ste);
        hs += H;
        if constexpr (REC) thn[k] = (double)th;
        qf[0][k] = fma(omc, qf[0][k], om * (H - ((P)1 - wP[0]) * th));
#pragma unroll
        for (int i = 1; i < 9; ++i) qf[i][k] = fma(omc, qf[i][k], om * (i <= 4 ? wP[1] : wP[2]) * th);
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

// One warp tile: segment `seg` of problem pb, rows [ya, yb).
template <typename P, bool REC>
__device__ __forceinline__ void d2q9_tile(const Problem& pb, const P* __restrict__ src, P* __restrict__ dst,
                                          double* __restrict__ rec, int seg, int ya, int yb, Acc<P>& acc,
                                          TileSums& ts, DevStats* st, P* ring, int pi, NewtonJob* jobs,
                                          unsigned int* job_count)
{
    using R = Ring<P>;
    constexpr int N = R::N;
    const int lane = threadIdx.x & 31;
    const int segx = seg * 32 * N;
    const int x0 = segx + lane * N;
    const long long pl = pb.plane;
    const long long pitch = pb.pitch;
    const bool has_left = segx > 0;
    const bool has_right = segx + 32 * N < pb.nx;
    // problem constants, converted once per tile (the compiler cannot hoist loads
    // of *pb above the stores of the loop, and a conversion from FP64 costs an
    // FP64-pipe instruction on this GPU)
    const P omc = (P)(1.0 - pb.omega);
    const float om_f = (float)pb.omega;
    const double omc_d = 1.0 - pb.omega;
    const double inv_delta = pb.inv_delta;
    const int nx = pb.nx, ny = pb.ny;
    const P wP[3] = {(P)d2_w(0), (P)d2_w(1), (P)d2_w(5)};
    const float thr_f = (float)pb.sat;

    // prologue: rows ya-1 .. ya+kStages-2 (one per slot), one commit group per row.
    // Iteration y then needs rows <= y+1 and leaves rows y+2 .. y+kStages-2 in
    // flight (wait_group kStages-3); it refills the slot of row y-1 with row y+kStages-1.
#pragma unroll
    for (int s = 0; s < kStages; ++s) {
        const int r = ya - 1 + s;
        if (r <= yb) ring_load<P>(ring + ((r + 1) % kStages) * R::SLOT, src, pl, pitch, r, segx, lane, has_left, has_right);
        cp_async_commit();
    }

    for (int y = ya; y < yb; ++y) {
        cp_async_wait<kStages - 3>();   // rows <= y+1 have landed (for this lane)
        __syncwarp();                   // ... and for every lane of the warp
        const P* sm1 = ring + ((y) % kStages) * R::SLOT;        // row y-1  (slot index (r+1) % S)
        const P* s0 = ring + ((y + 1) % kStages) * R::SLOT;     // row y
        const P* sp1 = ring + ((y + 2) % kStages) * R::SLOT;    // row y+1

        P u0[N], u1[N], u2[N], u3[N], u4[N], u5[N], u6[N], u7[N], u8[N];
        lds<P>(s0 + 0 * R::ROW + lane * N, u0);
        lds<P>(s0 + 1 * R::ROW + lane * N, u1);
        lds<P>(s0 + 2 * R::ROW + lane * N, u2);
        lds<P>(s0 + 3 * R::ROW + lane * N, u3);
        lds<P>(s0 + 4 * R::ROW + lane * N, u4);
        lds<P>(s0 + 5 * R::ROW + lane * N, u5);
        lds<P>(s0 + 6 * R::ROW + lane * N, u6);
        lds<P>(s0 + 7 * R::ROW + lane * N, u7);
        lds<P>(s0 + 8 * R::ROW + lane * N, u8);

        P qf[9][N];
        {
            P t[N], s[N];
#pragma unroll
            for (int k = 0; k < N; ++k) qf[0][k] = u0[k];
            from_left<P, N>(u1, s0[R::HALO + 2 * 1], lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[1][k] = s[k];
            from_right<P, N>(u3, s0[R::HALO + 2 * 3 + 1], lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[3][k] = s[k];
            lds<P>(sm1 + 2 * R::ROW + lane * N, t);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[2][k] = t[k];
            lds<P>(sm1 + 5 * R::ROW + lane * N, t);
            from_left<P, N>(t, sm1[R::HALO + 2 * 5], lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[5][k] = s[k];
            lds<P>(sm1 + 6 * R::ROW + lane * N, t);
            from_right<P, N>(t, sm1[R::HALO + 2 * 6 + 1], lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[6][k] = s[k];
            lds<P>(sp1 + 4 * R::ROW + lane * N, t);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[4][k] = t[k];
            lds<P>(sp1 + 7 * R::ROW + lane * N, t);
            from_right<P, N>(t, sp1[R::HALO + 2 * 7 + 1], lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[7][k] = s[k];
            lds<P>(sp1 + 8 * R::ROW + lane * N, t);
            from_left<P, N>(t, sp1[R::HALO + 2 * 8], lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[8][k] = s[k];
        }

        // every lane has its values of row y-1 in registers: refill that slot with
        // row y+kStages-1 now, so the load overlaps this row's arithmetic
        __syncwarp();
        {
            const int rn = y + kStages - 1;
            if (rn <= yb) ring_load<P>(ring + ((rn + 1) % kStages) * R::SLOT, src, pl, pitch, rn, segx, lane, has_left, has_right);
            cp_async_commit();
        }
        if (pb.method == 1)
            row_update_eebm<P, N, REC, true>(pb, y, x0, qf, u0, u1, u2, u3, u4, u5, u6, u7, u8,
                                             GlobalRowOut<P, N>{dst + (long long)(y + 1) * pitch + x0, pl}, rec, acc,
                                             ts, omc, wP, nx, ny);
        else
            row_update<P, N, REC, true>(pb, y, x0, lane, qf, u0, u1, u2, u3, u4, u5, u6, u7, u8,
                                        GlobalRowOut<P, N>{dst + (long long)(y + 1) * pitch + x0, pl}, rec, acc, ts, st,
                                        pi, jobs, job_count, omc, om_f, omc_d, wP, thr_f, nx, ny);

    }
    cp_async_wait<0>();
    __syncwarp();
}

// ---------------------------------------------------------------- direct tile
// Same update with rows loaded straight from global memory into registers:
// 2 floats (FP32 form) or 1 double per thread, so a warp covers 256 bytes of
// each plane row and the kernel needs few registers and no shared memory; many
// resident warps keep enough rows in flight.  Planes pulled along +y come from
// the previous row (kept shifted in registers), planes pulled along -y from the
// next row (loaded one row ahead and kept for the moments of the next row).
#ifndef LBM_DIRECT_PREFETCH
#define LBM_DIRECT_PREFETCH 1
#endif

template <typename P> struct Vd;
template <> struct Vd<float> { static constexpr int N = 2; };
template <> struct Vd<double> { static constexpr int N = 1; };

__device__ __forceinline__ void ldg_n(const float* p, float (&v)[2])
{
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ldg_n(const double* p, double (&v)[1]) { v[0] = __ldg(p); }

template <typename P, bool REC>
__device__ __forceinline__ void d2q9_tile_direct(const Problem& pb, const P* __restrict__ src, P* __restrict__ dst,
                                                 double* __restrict__ rec, int seg, int ya, int yb, Acc<P>& acc,
                                                 TileSums& ts, DevStats* st, int pi, NewtonJob* jobs,
                                                 unsigned int* job_count)
{
    constexpr int N = Vd<P>::N;
    const int lane = threadIdx.x & 31;
    const int segx = seg * 32 * N;
    const int x0 = segx + lane * N;
    const long long pl = pb.plane;
    const long long pitch = pb.pitch;
    const bool has_left = segx > 0;
    const bool has_right = segx + 32 * N < pb.nx;
    const bool seg_interior = has_left && has_right;   // no wall column, every node inside
    const P omc = (P)(1.0 - pb.omega);
    const float om_f = (float)pb.omega;
    const double omc_d = 1.0 - pb.omega;
    const int nx = pb.nx, ny = pb.ny;
    const P wP[3] = {(P)d2_w(0), (P)d2_w(1), (P)d2_w(5)};
    const float thr_f = (float)pb.sat;

    auto rp = [&](int i, int r) -> const P* { return src + i * pl + (long long)(r + 1) * pitch + x0; };
    auto hl = [&](int i, int r) -> P {
        return (lane == 0 && has_left) ? __ldg(src + i * pl + (long long)(r + 1) * pitch + segx - 1) : (P)0;
    };
    auto hr = [&](int i, int r) -> P {
        return (lane == 31 && has_right) ? __ldg(src + i * pl + (long long)(r + 1) * pitch + segx + 32 * N) : (P)0;
    };

    P up2[N], up5[N], up6[N], cu4[N], cu7[N], cu8[N];
    {
        P t[N];
        ldg_n(rp(2, ya - 1), up2);
        ldg_n(rp(5, ya - 1), t);
        from_left<P, N>(t, hl(5, ya - 1), lane, up5);
        ldg_n(rp(6, ya - 1), t);
        from_right<P, N>(t, hr(6, ya - 1), lane, up6);
        ldg_n(rp(4, ya), cu4);
        ldg_n(rp(7, ya), cu7);
        ldg_n(rp(8, ya), cu8);
    }
    // loads of one row: planes 0,1,3,2,5,6 at row y, planes 4,7,8 at row y+1, and
    // the elements beyond the segment for the planes shifted along x
    struct RowLoads {
        P r0[N], r1[N], r3[N], c2[N], c5[N], c6[N], n4[N], n7[N], n8[N];
        P h1, h3, h5, h6, h7, h8;
    };
    auto issue = [&](RowLoads& L, int y) {
        ldg_n(rp(0, y), L.r0);
        ldg_n(rp(1, y), L.r1);
        ldg_n(rp(3, y), L.r3);
        ldg_n(rp(2, y), L.c2);
        ldg_n(rp(5, y), L.c5);
        ldg_n(rp(6, y), L.c6);
        ldg_n(rp(4, y + 1), L.n4);
        ldg_n(rp(7, y + 1), L.n7);
        ldg_n(rp(8, y + 1), L.n8);
        L.h1 = hl(1, y);
        L.h3 = hr(3, y);
        L.h5 = hl(5, y);
        L.h6 = hr(6, y);
        L.h7 = hr(7, y + 1);
        L.h8 = hl(8, y + 1);
    };
    RowLoads cur;
    issue(cur, ya);
    for (int y = ya; y < yb; ++y) {
        // next row's loads first, so they are in flight during this row's arithmetic
        RowLoads nxt;
        if (LBM_DIRECT_PREFETCH && y + 1 < yb) issue(nxt, y + 1);
        P qf[9][N];
        {
            P s[N];
#pragma unroll
            for (int k = 0; k < N; ++k) {
                qf[0][k] = cur.r0[k]; qf[2][k] = up2[k]; qf[4][k] = cur.n4[k]; qf[5][k] = up5[k]; qf[6][k] = up6[k];
            }
            from_left<P, N>(cur.r1, cur.h1, lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[1][k] = s[k];
            from_right<P, N>(cur.r3, cur.h3, lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[3][k] = s[k];
            from_right<P, N>(cur.n7, cur.h7, lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[7][k] = s[k];
            from_left<P, N>(cur.n8, cur.h8, lane, s);
#pragma unroll
            for (int k = 0; k < N; ++k) qf[8][k] = s[k];
        }
        if (pb.method == 1)
            row_update_eebm<P, N, REC, true>(pb, y, x0, qf, cur.r0, cur.r1, cur.c2, cur.r3, cu4, cur.c5, cur.c6, cu7,
                                             cu8, GlobalRowOut<P, N>{dst + (long long)(y + 1) * pitch + x0, pl}, rec,
                                             acc, ts, omc, wP, nx, ny);
        else if (seg_interior && y > 0 && y < ny - 1)
            row_update<P, N, REC, false>(pb, y, x0, lane, qf, cur.r0, cur.r1, cur.c2, cur.r3, cu4, cur.c5, cur.c6, cu7,
                                         cu8, GlobalRowOut<P, N>{dst + (long long)(y + 1) * pitch + x0, pl}, rec, acc,
                                         ts, st, pi, jobs, job_count, omc, om_f, omc_d, wP, thr_f, nx, ny);
        else
            row_update<P, N, REC, true>(pb, y, x0, lane, qf, cur.r0, cur.r1, cur.c2, cur.r3, cu4, cur.c5, cur.c6, cu7,
                                        cu8, GlobalRowOut<P, N>{dst + (long long)(y + 1) * pitch + x0, pl}, rec, acc,
                                        ts, st, pi, jobs, job_count, omc, om_f, omc_d, wP, thr_f, nx, ny);
        // roll the register window
#pragma unroll
        for (int k = 0; k < N; ++k) { up2[k] = cur.c2[k]; cu4[k] = cur.n4[k]; cu7[k] = cur.n7[k]; cu8[k] = cur.n8[k]; }
        from_left<P, N>(cur.c5, cur.h5, lane, up5);
        from_right<P, N>(cur.c6, cur.h6, lane, up6);
        if (LBM_DIRECT_PREFETCH) {
            cur = nxt;
        } else if (y + 1 < yb) {
            issue(cur, y + 1);
        }
    }
}

#ifndef LBM_STEP_DIRECT
#define LBM_STEP_DIRECT 1
#endif




template <typename P, bool REC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, LBM_STEP_MIN_BLOCKS) d2q9_step_kernel(StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    using R = Ring<P>;
    const int wib = threadIdx.x >> 5;
    P* ring = reinterpret_cast<P*>(smem + wib * R::WARP_BYTES);
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
        const P* src = static_cast<const P*>(pb.state[a.parity]);
        P* dst = static_cast<P*>(pb.state[a.parity ^ 1]);
        Acc<P> acc;
        TileSums ts;
#if LBM_STEP_DIRECT
        d2q9_tile_direct<P, REC>(pb, src, dst, a.rec, seg, ya, yb, acc, ts, st, pi, a.jobs, a.job_count);
#else
        d2q9_tile<P, REC>(pb, src, dst, a.rec, seg, ya, yb, acc, ts, st, ring, pi, a.jobs, a.job_count);
#endif
        flush_tile_sums<P>(acc, ts, st, lane);
    }
    // statistics are published by the job kernel that follows every step
}

// ---------------------------------------------------------------- TMA row pipeline
// Single-problem FP32 step, warp-specialized.  A block owns a strip of
// kTmaW = 128 columns and a contiguous range of rows [ya, yb).  A producer
// warp streams rows of all nine planes into a ring of shared-memory slots
// with TMA tensor loads (136 columns: four more on each side for the pulls
// along x; outside the tensor the hardware fills zeros); a load completes on
// the slot's `full` mbarrier.  Four consumer warps (32 columns each, one node
// per lane) take the pulled values of row y from the slots of rows y-1, y and
// y+1 (shared-memory loads at +-1 column, no shuffles), run the row update
// above, store their outputs straight to global memory, and release the slot
// of row y-1 on its `empty` mbarrier, which the producer waits on before it
// reuses the slot.  The consumers are not synchronized with one another, and
// the ring keeps up to kTmaStages rows in flight per block without holding
// registers.  Every mbarrier wait is bounded: on a timeout the kernel records
// LBM_ERR_TIMEOUT, stops, and the producer waits (bounded) for its own copies
// in flight before it exits.
#ifndef LBM_TMA_STAGES
#define LBM_TMA_STAGES 8
#endif
constexpr int kTmaStages = LBM_TMA_STAGES;
constexpr int kTmaBox = kTmaW + 2 * kTmaHalo;                  // 136 loaded columns
constexpr int kTmaSlot = (9 * kTmaBox * 4 + 127) / 128 * 32;   // floats per slot (128-byte multiple)
constexpr int kTmaConsumers = kTmaW / 32;                       // consumer warps
constexpr int kTmaThreads = kTmaW + 32;                         // + the producer warp
constexpr unsigned kTmaRowBytes = 9u * kTmaBox * 4u;             // bytes one row load delivers

#ifndef LBM_TMA_MIN_BLOCKS
#define LBM_TMA_MIN_BLOCKS 5   // resident blocks per SM the register budget is fitted to
#endif

template <bool REC>
__global__ void __launch_bounds__(kTmaThreads, LBM_TMA_MIN_BLOCKS) d2q9_tma_kernel(const StepArgs a, const __grid_constant__ TmaMaps m)
{
    __shared__ __align__(128) float ring[kTmaStages * kTmaSlot];
    __shared__ __align__(8) unsigned long long full[kTmaStages];
    __shared__ __align__(8) unsigned long long empty[kTmaStages];

    int pi, seg, ya, yb;
    const CUtensorMap* lmap;
    if (m.tiles) {
        const int4 t = m.tiles[blockIdx.x];
        pi = t.x;
        seg = t.y;
        ya = t.z;
        yb = t.w;
        lmap = &m.gmaps[2 * pi + a.parity];
    } else {
        pi = 0;
        seg = blockIdx.x % m.nsegs;
        const int part = blockIdx.x / m.nsegs;
        const int nyp = a.probs[0].ny;
        ya = (int)((long long)nyp * part / m.nparts);
        yb = (int)((long long)nyp * (part + 1) / m.nparts);
        lmap = &m.load[a.parity];
    }
    const Problem& pb = a.probs[pi];
    DevStats* st = &a.stats[pb.stats];
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int nx = pb.nx, ny = pb.ny;
    const int segx = seg * kTmaW;

    if (tid == 0) {
        for (int k = 0; k < kTmaStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kTmaConsumers);
        }
        fence_mbar_init();
    }
    __syncthreads();
    // row r (ya-1 <= r <= yb) is the k-th load, k = r - ya + 1: slot k % S, use k / S

    if (warp == kTmaConsumers) {
        // ---- producer
        if (lane == 0) {
            int last = -1;   // last k issued
            bool ok = true;
            for (int r = ya - 1; r <= yb; ++r) {
                const int k = r - (ya - 1);
                const int sl = k % kTmaStages;
                if (k >= kTmaStages && !mbar_wait_bounded(&empty[sl], (unsigned)((k / kTmaStages - 1) & 1))) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&full[sl], kTmaRowBytes);
                tma_load_rows(lmap, ring + sl * kTmaSlot, &full[sl], segx - kTmaHalo, r + 1);
                last = k;
            }
            if (!ok) {
                atomicExch(&st->error, 4);   // LBM_ERR_TIMEOUT
                // the copies still in flight land before the block may exit
                for (int k = max(0, last - kTmaStages + 1); k <= last; ++k)
                    (void)mbar_wait_bounded(&full[k % kTmaStages], (unsigned)((k / kTmaStages) & 1));
            }
        }
        return;
    }

    // ---- consumers
    const int x = segx + tid;
    const float omc = (float)(1.0 - pb.omega);
    const float om_f = (float)pb.omega;
    const double omc_d = 1.0 - pb.omega;
    const float wP[3] = {(float)d2_w(0), (float)d2_w(1), (float)d2_w(5)};
    const float thr_f = (float)pb.sat;
    const int wx0 = segx + warp * 32;   // first column of this warp
    const bool warp_interior_x = wx0 > 0 && wx0 + 31 < nx - 1;
    float* dst = static_cast<float*>(pb.state[a.parity ^ 1]);
    const long long pl = pb.plane;
    const long long pitch = pb.pitch;
    Acc<float> acc;
    TileSums ts;
    auto wait_row = [&](int r) -> bool {
        const int k = r - (ya - 1);
        return mbar_wait_bounded(&full[k % kTmaStages], (unsigned)((k / kTmaStages) & 1));
    };
    bool ok = wait_row(ya - 1) && wait_row(ya);
    for (int y = ya; ok && y < yb; ++y) {
        ok = wait_row(y + 1);
        if (!ok) break;
        const int km = y - 1 - (ya - 1);
        const float* sm1 = ring + (km % kTmaStages) * kTmaSlot + kTmaHalo + tid;
        const float* s0 = ring + ((km + 1) % kTmaStages) * kTmaSlot + kTmaHalo + tid;
        const float* sp1 = ring + ((km + 2) % kTmaStages) * kTmaSlot + kTmaHalo + tid;
        float u0[1], u1[1], u2[1], u3[1], u4[1], u5[1], u6[1], u7[1], u8[1];
        u0[0] = s0[0 * kTmaBox]; u1[0] = s0[1 * kTmaBox]; u2[0] = s0[2 * kTmaBox];
        u3[0] = s0[3 * kTmaBox]; u4[0] = s0[4 * kTmaBox]; u5[0] = s0[5 * kTmaBox];
        u6[0] = s0[6 * kTmaBox]; u7[0] = s0[7 * kTmaBox]; u8[0] = s0[8 * kTmaBox];
        float qf[9][1];
        qf[0][0] = u0[0];
        qf[1][0] = s0[1 * kTmaBox - 1];    // Omega_1(x - 1, y)
        qf[3][0] = s0[3 * kTmaBox + 1];    // Omega_3(x + 1, y)
        qf[2][0] = sm1[2 * kTmaBox];       // Omega_2(x, y - 1)
        qf[5][0] = sm1[5 * kTmaBox - 1];   // Omega_5(x - 1, y - 1)
        qf[6][0] = sm1[6 * kTmaBox + 1];   // Omega_6(x + 1, y - 1)
        qf[4][0] = sp1[4 * kTmaBox];       // Omega_4(x, y + 1)
        qf[7][0] = sp1[7 * kTmaBox + 1];   // Omega_7(x + 1, y + 1)
        qf[8][0] = sp1[8 * kTmaBox - 1];   // Omega_8(x - 1, y + 1)
        // every lane has read the slot of row y - 1: release it to the producer
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[km % kTmaStages]);
        const GlobalRowOut<float, 1> out{dst + (long long)(y + 1) * pitch + x, pl};
        if (pb.method == 1)
            row_update_eebm<float, 1, REC, true>(pb, y, x, qf, u0, u1, u2, u3, u4, u5, u6, u7, u8, out, a.rec, acc, ts,
                                                 omc, wP, nx, ny);
        else if (warp_interior_x && y > 0 && y < ny - 1)
            row_update<float, 1, REC, false>(pb, y, x, lane, qf, u0, u1, u2, u3, u4, u5, u6, u7, u8, out, a.rec, acc,
                                             ts, st, pi, a.jobs, a.job_count, omc, om_f, omc_d, wP, thr_f, nx, ny);
        else
            row_update<float, 1, REC, true>(pb, y, x, lane, qf, u0, u1, u2, u3, u4, u5, u6, u7, u8, out, a.rec, acc,
                                            ts, st, pi, a.jobs, a.job_count, omc, om_f, omc_d, wP, thr_f, nx, ny);
    }
    if (!ok && lane == 0) atomicExch(&st->error, 4);   // LBM_ERR_TIMEOUT
    flush_tile_sums<float>(acc, ts, st, lane);
}

// ---------------------------------------------------------------- Newton jobs
// Local Newton solves deferred by the step kernel (Eq. 14, mixed-precision
// form), one job per lane, consecutive jobs per warp; Q = 9 (D2Q9) or 5 (D2Q5)
// planes.  For each job:
//   theta' = m0 + (phi(theta) - phi(root))/Ste,  c = theta' - (1-omega) m0,
//   Omega~_i = (1-omega) q_i + w_i c   (q_i was stored by the step kernel).
// Energy contributions theta' + phi(theta')/Ste are summed per problem as
// exact 128-bit fixed-point integers (independent of the job order).  The last
// warp to finish publishes the step statistics and clears the job list.
template <typename P, bool REC, int Q>
__global__ void __launch_bounds__(128) newton_jobs_kernel(JobArgs a)
{
    const unsigned count = *reinterpret_cast<volatile unsigned*>(a.job_count);
    const int lane = threadIdx.x & 31;
    const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nw = (gridDim.x * blockDim.x) >> 5;
    for (unsigned base = gw * 32; base < count; base += nw * 32) {
        const unsigned j = base + lane;
        int sidx = -1, it = 0;
        Fx e{0, 0ull};
        if (j < count) {
            const NewtonJob jb = a.jobs[j];
            const Problem& pb = a.probs[jb.prob];
            sidx = pb.stats;
            double m0, th;
            if constexpr (sizeof(P) == 4) {
                const float* pm = reinterpret_cast<const float*>(&jb.m0);
                const float* pt = reinterpret_cast<const float*>(&jb.theta);
                m0 = (double)pm[0] + (double)pm[1];
                th = (double)pt[0] + (double)pt[1];
            } else {
                m0 = jb.m0;
                th = jb.theta;
            }
            const double pth = phi_of(th, pb.inv_delta);
            const NewtonOut nr = newton_mixed(m0, th, pth, pb);
            if (!nr.ok || !isfinite(nr.root)) atomicOr(&a.stats[sidx].error, 3);
            const double tn = m0 + (pth - nr.phi_root) * pb.inv_ste;
            const P c = (P)(tn - (1.0 - pb.omega) * m0);
            const P omc = (P)(1.0 - pb.omega);
            const int x = jb.node % pb.nx, y = jb.node / pb.nx;
            P* d = static_cast<P*>(pb.state[a.parity ^ 1]) + (long long)(y + 1) * pb.pitch + x;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const P wi = (P)lat_w(Q, i);
                d[i * pb.plane] = fma(omc, d[i * pb.plane], wi * c);
            }
            if (REC) a.rec[(long long)y * pb.pitch + x] = tn;
            e = to_fixed(tn + nr.phi_root * pb.inv_ste);
            it = nr.iters;
        }
        // lanes of the same problem: the lowest lane sums them exactly and adds once
        const unsigned grp = __match_any_sync(kFull, sidx);
        const int leader = __ffs(grp) - 1;
        Fx sum{0, 0ull};
        int n = 0, mx = 0;
        for (int l = 0; l < 32; ++l) {
            Fx v;
            v.hi = __shfl_sync(kFull, e.hi, l);
            v.lo = __shfl_sync(kFull, e.lo, l);
            const int vi = __shfl_sync(kFull, it, l);
            if ((grp >> l) & 1) {
                fx_add(sum, v);
                ++n;
                mx = max(mx, vi);
            }
        }
        if (lane == leader && sidx >= 0) {
            DevStats* st = &a.stats[sidx];
            acc_add_fx(&st->cur_energy, sum);
            atomicAdd(&st->cur_newton, (unsigned long long)n);
            atomicMax(&st->cur_maxit, mx);
        }
    }
    // last block: publish every problem's step statistics, clear the job list
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        for (int p = threadIdx.x; p < a.nprob; p += blockDim.x) publish_stats(&a.stats[a.probs[p].stats], &a.probs[p]);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            *a.job_count = 0u;
            *a.ticket = 0u;
        }
    }
}

template <typename P>
constexpr int step_smem_bytes()
{
    return LBM_STEP_DIRECT ? 0 : kWarpsPerBlock * Ring<P>::WARP_BYTES;
}

template <typename P, bool REC>
static cudaError_t launch_t(const StepArgs& a, int grid, cudaStream_t s)
{
    constexpr int sm = step_smem_bytes<P>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(d2q9_step_kernel<P, REC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    d2q9_step_kernel<P, REC><<<grid, kWarpsPerBlock * 32, sm, s>>>(a);
    return cudaGetLastError();
}

int d2q9_segment_width(int precision)
{
    if (LBM_STEP_DIRECT) return precision == 1 ? 32 * Vd<float>::N : 32 * Vd<double>::N;
    return precision == 1 ? 32 * 4 : 32 * 2;
}

cudaError_t launch_d2q9_step(int precision, const StepArgs& a, int grid, cudaStream_t s)
{
    if (grid <= 0) return cudaErrorInvalidValue;
    if (precision == 1) return a.rec ? launch_t<float, true>(a, grid, s) : launch_t<float, false>(a, grid, s);
    return a.rec ? launch_t<double, true>(a, grid, s) : launch_t<double, false>(a, grid, s);
}

cudaError_t launch_d2q9_tma(const StepArgs& a, const TmaMaps& m, cudaStream_t s)
{
    const int grid = m.tiles ? m.ntiles : m.nsegs * m.nparts;
    if (grid <= 0) return cudaErrorInvalidValue;
    if (a.rec) d2q9_tma_kernel<true><<<grid, kTmaThreads, 0, s>>>(a, m);
    else d2q9_tma_kernel<false><<<grid, kTmaThreads, 0, s>>>(a, m);
    return cudaGetLastError();
}

int d2q9_tma_blocks_per_sm()
{
    // all of the unified L1 / shared memory as shared memory: five blocks per SM
    cudaFuncSetAttribute(d2q9_tma_kernel<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(d2q9_tma_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, d2q9_tma_kernel<false>, kTmaThreads, 0);
    return n > 0 ? n : 1;
}

template <int Q>
static void launch_jobs_q(int precision, const JobArgs& a, int grid, cudaStream_t s)
{
    if (precision == 1) {
        if (a.rec) newton_jobs_kernel<float, true, Q><<<grid, 128, 0, s>>>(a);
        else newton_jobs_kernel<float, false, Q><<<grid, 128, 0, s>>>(a);
    } else {
        if (a.rec) newton_jobs_kernel<double, true, Q><<<grid, 128, 0, s>>>(a);
        else newton_jobs_kernel<double, false, Q><<<grid, 128, 0, s>>>(a);
    }
}

cudaError_t launch_newton_jobs(int precision, int q, const JobArgs& a, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * 8;   // 8 x 128 threads per SM: about one pass over ~150k nodes
    if (q == 9) launch_jobs_q<9>(precision, a, grid, s);
    else if (q == 5) launch_jobs_q<5>(precision, a, grid, s);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

int d2q9_blocks_per_sm(int precision)
{
    int n = 0;
    if (precision == 1) {
        cudaFuncSetAttribute(d2q9_step_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             step_smem_bytes<float>());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, d2q9_step_kernel<float, false>, kWarpsPerBlock * 32,
                                                      step_smem_bytes<float>());
    } else {
        cudaFuncSetAttribute(d2q9_step_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             step_smem_bytes<double>());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, d2q9_step_kernel<double, false>, kWarpsPerBlock * 32,
                                                      step_smem_bytes<double>());
    }
    return n > 0 ? n : 1;
}

}  // namespace lbm
