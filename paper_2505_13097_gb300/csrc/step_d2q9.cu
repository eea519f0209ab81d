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
#include "lbm_device.cuh"

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

// value at x-1 (pull along e_x = +1); h = element left of the segment
template <typename P, int N>
__device__ __forceinline__ void from_left(const P (&v)[N], P h, int lane, P (&s)[N])
{
    P up = __shfl_up_sync(kFull, v[N - 1], 1);
    s[0] = lane == 0 ? h : up;
#pragma unroll
    for (int k = 1; k < N; ++k) s[k] = v[k - 1];
}
// value at x+1 (pull along e_x = -1); h = element right of the segment
template <typename P, int N>
__device__ __forceinline__ void from_right(const P (&v)[N], P h, int lane, P (&s)[N])
{
    P dn = __shfl_down_sync(kFull, v[0], 1);
    s[N - 1] = lane == 31 ? h : dn;
#pragma unroll
    for (int k = 0; k < N - 1; ++k) s[k] = v[k + 1];
}

// Boundary closures of Sec. 4.2 at one wall node (x, y).  q holds the pulled
// values (entries of unknown directions are overwritten), u the node's own
// Omega.  Returns the boundary flux contribution (filled q minus Omega that
// leaves the lattice); dir/theta_d report a Dirichlet node.
template <typename P>
__device__ __noinline__ double wall_closure(P* q, const P* u, int x, int y, const Problem& pb, bool& dir, double& theta_d)
{
    unsigned unk = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        int sx = x - d2_ex(i), sy = y - d2_ey(i);
        if (sx < 0 || sx >= pb.nx || sy < 0 || sy >= pb.ny) unk |= 1u << i;
    }
    int walls = (x == 0 ? 1 : 0) | (x == pb.nx - 1 ? 2 : 0) | (y == 0 ? 4 : 0) | (y == pb.ny - 1 ? 8 : 0);
    dir = false;
    theta_d = 0.0;
    for (int k = 0; k < 4; ++k)
        if (((walls >> k) & 1) && pb.wall_kind[k] == 1) {
            dir = true;
            theta_d = pb.wall_theta[k];
            break;
        }
    double out = 0.0, in = 0.0;
#pragma unroll
    for (int j = 1; j < 9; ++j)
        if ((unk >> d2_opp(j)) & 1) out += (double)u[j];
    if (dir) {
        // Eq. (14) with theta' = theta_D fixes M0(q) = theta_D + (phi(theta_D) - phi(theta))/Ste;
        // the unknown q share what the known ones leave, in proportion to w_i.
        double th = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) th += (double)u[i];
        double m0t = theta_d + (phi_of(theta_d, pb.inv_delta) - phi_of(th, pb.inv_delta)) * pb.inv_ste;
        double known = 0.0, wu = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if ((unk >> i) & 1) wu += d2_w(i);
            else known += (double)q[i];
        }
        double r = (m0t - known) / wu;
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if ((unk >> i) & 1) {
                q[i] = (P)(d2_w(i) * r);
                in += (double)q[i];
            }
    } else {
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if ((unk >> i) & 1) {
                int o = d2_opp(i);
                q[i] = (pb.bb_mode == 0 && !((unk >> o) & 1)) ? q[o] : u[o];
                in += (double)q[i];
            }
    }
    return in - out;
}

template <typename P>
struct Acc;   // per-lane accumulator of sum theta' (float-float or double)
template <>
struct Acc<float> {
    ff s{0.f, 0.f};
    __device__ void add_ff(const ff& v) { ff_add(s, v.hi); s.lo = __fadd_rn(s.lo, v.lo); }
    __device__ void add_d(double v) { float h = (float)v; ff_add(s, h); s.lo = __fadd_rn(s.lo, (float)(v - (double)h)); }
    __device__ double get() const { return ff_to_double(s); }
};
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ void add_d(double v) { s += v; }
    __device__ double get() const { return s; }
};

// m0 accumulator type per precision
template <typename P> struct M0T;
template <> struct M0T<float> { using T = ff; };
template <> struct M0T<double> { using T = double; };

__device__ __forceinline__ void m0_init(ff& a) { a.hi = 0.f; a.lo = 0.f; }
__device__ __forceinline__ void m0_init(double& a) { a = 0.0; }
__device__ __forceinline__ void m0_add(ff& a, float v) { ff_add(a, v); }
__device__ __forceinline__ void m0_add(double& a, double v) { a += v; }
__device__ __forceinline__ double m0_d(const ff& a) { return ff_to_double(a); }
__device__ __forceinline__ double m0_d(const double& a) { return a; }
__device__ __forceinline__ float m0_f(const ff& a) { return a.hi; }
__device__ __forceinline__ float m0_f(const double& a) { return approx_float(a); }

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

struct TileSums {
    double flux = 0.0, phi_sum = 0.0;
    int liquid = 0, newton = 0, maxit = 0;
};

// One warp tile: segment `seg` of problem pb, rows [ya, yb).
template <typename P>
__device__ __forceinline__ void d2q9_tile(const Problem& pb, const P* __restrict__ src, P* __restrict__ dst,
                                          double* __restrict__ rec, int seg, int ya, int yb, Acc<P>& acc,
                                          TileSums& ts, DevStats* st)
{
    constexpr int N = Vw<P>::N;
    const int lane = threadIdx.x & 31;
    const int segx = seg * 32 * N;
    const int x0 = segx + lane * N;
    const long long pl = pb.plane;
    const long long pitch = pb.pitch;
    const bool has_left = segx > 0;
    const bool has_right = segx + 32 * N < pb.nx;
    const P omc = (P)(1.0 - pb.omega);
    const P wP[3] = {(P)d2_w(0), (P)d2_w(1), (P)d2_w(5)};
    const double thr = kSat * pb.delta;
    const float thr_f = (float)thr;

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
        ldv<P>(rp(2, ya - 1), up2);
        ldv<P>(rp(5, ya - 1), t);
        from_left<P, N>(t, hl(5, ya - 1), lane, up5);
        ldv<P>(rp(6, ya - 1), t);
        from_right<P, N>(t, hr(6, ya - 1), lane, up6);
        ldv<P>(rp(4, ya), cu4);
        ldv<P>(rp(7, ya), cu7);
        ldv<P>(rp(8, ya), cu8);
    }

    for (int y = ya; y < yb; ++y) {
        P r0[N], r1[N], r3[N], c2[N], c5[N], c6[N], n4[N], n7[N], n8[N];
        ldv<P>(rp(0, y), r0);
        ldv<P>(rp(1, y), r1);
        ldv<P>(rp(3, y), r3);
        ldv<P>(rp(2, y), c2);
        ldv<P>(rp(5, y), c5);
        ldv<P>(rp(6, y), c6);
        ldv<P>(rp(4, y + 1), n4);
        ldv<P>(rp(7, y + 1), n7);
        ldv<P>(rp(8, y + 1), n8);
        const P h1 = hl(1, y), h3 = hr(3, y), h5 = hl(5, y), h6 = hr(6, y), h7 = hr(7, y + 1), h8 = hl(8, y + 1);

        P q1[N], q3[N], q7[N], q8[N];
        from_left<P, N>(r1, h1, lane, q1);
        from_right<P, N>(r3, h3, lane, q3);
        from_right<P, N>(n7, h7, lane, q7);
        from_left<P, N>(n8, h8, lane, q8);

        P c[N];          // per node: theta' - (1-omega) m0, rounded to P
        P qf[9][N];      // pulled (and wall-filled) populations
        double thn[N];   // theta' for the record plane
        bool newton_k[N];
        typename M0T<P>::T m0[N];
        bool any_wall = false;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            qf[0][k] = r0[k]; qf[1][k] = q1[k]; qf[2][k] = up2[k]; qf[3][k] = q3[k]; qf[4][k] = n4[k];
            qf[5][k] = up5[k]; qf[6][k] = up6[k]; qf[7][k] = q7[k]; qf[8][k] = q8[k];
            const int x = x0 + k;
            any_wall |= (x < pb.nx) && (x == 0 || x == pb.nx - 1 || y == 0 || y == pb.ny - 1);
        }
        bool dir_k[N];
        double thd_k[N];
#pragma unroll
        for (int k = 0; k < N; ++k) { dir_k[k] = false; thd_k[k] = 0.0; }
        if (__any_sync(kFull, any_wall)) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const int x = x0 + k;
                if (x < pb.nx && (x == 0 || x == pb.nx - 1 || y == 0 || y == pb.ny - 1)) {
                    P qq[9], uu[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) qq[i] = qf[i][k];
                    uu[0] = r0[k]; uu[1] = r1[k]; uu[2] = c2[k]; uu[3] = r3[k]; uu[4] = cu4[k];
                    uu[5] = c5[k]; uu[6] = c6[k]; uu[7] = cu7[k]; uu[8] = cu8[k];
                    ts.flux += wall_closure<P>(qq, uu, x, y, pb, dir_k[k], thd_k[k]);
#pragma unroll
                    for (int i = 0; i < 9; ++i) qf[i][k] = qq[i];
                }
            }
        }

        bool any_newton = false;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int x = x0 + k;
            const bool valid = x < pb.nx;
            m0_init(m0[k]);
            // small weights first
#pragma unroll
            for (int i = 8; i >= 0; --i) m0_add(m0[k], qf[i][k]);
            P u[9] = {r0[k], r1[k], c2[k], r3[k], cu4[k], c5[k], c6[k], cu7[k], cu8[k]};
            const float tf = approx_sum<P>(u);
            const float mf = m0_f(m0[k]);
            const float marg = 1e-5f * (1.0f + fabsf(tf));
            const bool sat_liq = tf >= thr_f + marg && mf >= thr_f + marg;
            const bool sat_sol = tf <= -thr_f - marg && mf <= -thr_f - marg;
            newton_k[k] = valid && !dir_k[k] && !(sat_liq || sat_sol);
            any_newton |= newton_k[k];
            if (!valid) {
                c[k] = (P)0;
                thn[k] = 0.0;
#pragma unroll
                for (int i = 0; i < 9; ++i) qf[i][k] = (P)0;
            } else if (dir_k[k]) {
                const double md = m0_d(m0[k]);
                const double td = thd_k[k];
                c[k] = (P)(td - (1.0 - pb.omega) * md);
                thn[k] = td;
                acc.add_d(td);
                ts.phi_sum += phi_of(td, pb.inv_delta);
            } else if (!newton_k[k]) {
                // saturated: theta' = m0, no source; c = omega * m0
                if constexpr (sizeof(P) == 4) {
                    const ff& mm = m0[k];
                    c[k] = (P)__fmaf_rn((float)pb.omega, mm.hi, (float)pb.omega * mm.lo);
                    acc.add_ff(mm);
                    thn[k] = rec ? ff_to_double(mm) : 0.0;
                } else {
                    const double md = m0_d(m0[k]);
                    c[k] = (P)(pb.omega * md);
                    acc.add_d(md);
                    thn[k] = md;
                }
                ts.liquid += sat_liq ? 1 : 0;
            }
        }
        if (__any_sync(kFull, any_newton)) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                if (!newton_k[k]) continue;
                double th = 0.0;
                if constexpr (sizeof(P) == 4) {
                    ff t;
                    m0_init(t);
                    const P u[9] = {r0[k], r1[k], c2[k], r3[k], cu4[k], c5[k], c6[k], cu7[k], cu8[k]};
#pragma unroll
                    for (int i = 8; i >= 0; --i) ff_add(t, u[i]);
                    th = ff_to_double(t);
                } else {
                    const P u[9] = {r0[k], r1[k], c2[k], r3[k], cu4[k], c5[k], c6[k], cu7[k], cu8[k]};
#pragma unroll
                    for (int i = 8; i >= 0; --i) th += u[i];
                }
                const double md = m0_d(m0[k]);
                const double pth = phi_of(th, pb.inv_delta);
                NewtonOut nr = newton_solve(md, th, pth, pb.inv_ste, pb.inv_delta, pb.tol, pb.maxit);
                if (!nr.ok || !isfinite(nr.root)) atomicOr(&st->error, 3);
                // theta' = M0(f~) = m0 + (phi(theta) - phi(theta'))/Ste  (Eq. 13 summed over i)
                const double tn = md + (pth - nr.phi_root) * pb.inv_ste;
                c[k] = (P)(tn - (1.0 - pb.omega) * md);
                thn[k] = tn;
                acc.add_d(tn);
                ts.phi_sum += nr.phi_root;
                ts.newton += 1;
                ts.maxit = max(ts.maxit, nr.iters);
            }
        }

        // Omega~_i = (1-omega) q_i + w_i c
        P* drow = dst + (long long)(y + 1) * pitch + x0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const P wi = i == 0 ? wP[0] : (i <= 4 ? wP[1] : wP[2]);
            P o[N];
#pragma unroll
            for (int k = 0; k < N; ++k) o[k] = fma(omc, qf[i][k], wi * c[k]);
            stv<P>(drow + i * pl, o);
        }
        if (rec) {
            double* rr = rec + (long long)y * pitch + x0;
#pragma unroll
            for (int k = 0; k < N; k += 2) *reinterpret_cast<double2*>(rr + k) = make_double2(thn[k], thn[k + 1]);
        }

        // roll the register window
#pragma unroll
        for (int k = 0; k < N; ++k) { up2[k] = c2[k]; cu4[k] = n4[k]; cu7[k] = n7[k]; cu8[k] = n8[k]; }
        from_left<P, N>(c5, h5, lane, up5);
        from_right<P, N>(c6, h6, lane, up6);
    }
}

template <typename P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) d2q9_step_kernel(StepArgs a)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int slot = warp; slot < a.nslots; slot += nwarps) {
        int pi, t;
        if (a.schedule) {
            int2 s = a.schedule[slot];
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
        d2q9_tile<P>(pb, src, dst, a.rec, seg, ya, yb, acc, ts, st);
        // tile partial sums: fixed lane order, then one fixed-point atomic per quantity
        double e = warp_sum(acc.get() + ((double)ts.liquid + ts.phi_sum) * pb.inv_ste);
        double f = warp_sum(ts.flux);
        int nn = warp_sum_i(ts.newton);
        int mi = warp_max_i(ts.maxit);
        if (lane == 0) {
            acc_add(&st->cur_energy, e);
            acc_add(&st->cur_flux, f);
            if (nn) atomicAdd(&st->cur_newton, (unsigned long long)nn);
            if (mi) atomicMax(&st->cur_maxit, mi);
        }
    }
    finish_launch(a.stats, a.nprob, a.ticket);
}

int d2q9_segment_width(int precision) { return precision == 1 ? 32 * 4 : 32 * 2; }

cudaError_t launch_d2q9_step(int precision, const StepArgs& a, int grid, cudaStream_t s)
{
    if (grid <= 0) return cudaErrorInvalidValue;
    if (precision == 1) d2q9_step_kernel<float><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
    else d2q9_step_kernel<double><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbm
