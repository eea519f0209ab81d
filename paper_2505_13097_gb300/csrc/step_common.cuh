// Pieces shared by the D2Q9 and D2Q5 step kernels: vector stores, the
// per-lane accumulators of theta' and the boundary flux, and the warp flush
// of those sums into the exact fixed-point statistics.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// stores of one thread's N consecutive values (128-, 64- or 32/64-bit)
__device__ __forceinline__ void stv_n(float* p, const float (&v)[4]) { *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]); }
__device__ __forceinline__ void stv_n(float* p, const float (&v)[2]) { *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]); }
__device__ __forceinline__ void stv_n(double* p, const double (&v)[2]) { *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]); }
__device__ __forceinline__ void stv_n(double* p, const double (&v)[1]) { *p = v[0]; }
__device__ __forceinline__ void stv_n(float* p, const float (&v)[1]) { *p = v[0]; }

// theta' record of one thread's N nodes (FP64 plane)
template <int N>
__device__ __forceinline__ void st_rec(double* p, const double (&v)[N])
{
    if constexpr (N == 1) {
        *p = v[0];
    } else {
#pragma unroll
        for (int k = 0; k < N; k += 2) *reinterpret_cast<double2*>(p + k) = make_double2(v[k], v[k + 1]);
    }
}

template <typename P>
struct Acc;   // per-lane accumulator of sum theta' (float-float or double)
template <>
struct Acc<float> {
    ff s{0.f, 0.f};
    __device__ void add_ff(const ff& v) { ff_add(s, v.hi); s.lo = __fadd_rn(s.lo, v.lo); }
    __device__ void add_f(float v) { ff_add(s, v); }
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

struct TileSums {
    double flux = 0.0, phi_sum = 0.0;   // FP64 form
    ff flux_f{0.f, 0.f};                // FP32 form
    int dir_count[4] = {0, 0, 0, 0};   // Dirichlet nodes per wall (adds phi(theta_D)/Ste each)
    int liquid = 0, newton = 0, maxit = 0;
    int shifted = 0;                    // energy terms added less the state's shift
};

// A warp's partial sums, totalled in a fixed lane order (every lane gets the
// totals): energy and flux as exact fixed-point values, node counts as integers.
struct WarpSums {
    Fx e{0, 0ull}, f{0, 0ull};
    int nl = 0;        // saturated liquid nodes
    int nd[4] = {0, 0, 0, 0};   // Dirichlet nodes per wall
    int ns = 0;        // energy terms added less the state's shift
};

template <typename P>
__device__ __forceinline__ WarpSums warp_tile_sums(const Acc<P>& acc, const TileSums& ts)
{
    WarpSums w;
    if constexpr (sizeof(P) == 4) {
        ff se = acc.s, sf = ts.flux_f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float eh = __shfl_xor_sync(kFull, se.hi, o), el = __shfl_xor_sync(kFull, se.lo, o);
            const float fh = __shfl_xor_sync(kFull, sf.hi, o), fl = __shfl_xor_sync(kFull, sf.lo, o);
            ff_add(se, eh);
            se.lo += el;
            ff_add(sf, fh);
            sf.lo += fl;
        }
        w.e = float_to_fixed(se.hi);
        fx_add(w.e, float_to_fixed(se.lo));
        w.f = float_to_fixed(sf.hi);
        fx_add(w.f, float_to_fixed(sf.lo));
    } else {
        w.e = to_fixed(warp_sum(acc.get()));
        w.f = to_fixed(warp_sum(ts.flux));
    }
    w.nl = warp_sum_i(ts.liquid);
    w.ns = warp_sum_i(ts.shifted);
#pragma unroll
    for (int k = 0; k < 4; ++k) w.nd[k] = warp_sum_i(ts.dir_count[k]);
    return w;
}

__device__ __forceinline__ void add_sums(WarpSums& a, const WarpSums& b)
{
    fx_add(a.e, b.e);
    fx_add(a.f, b.f);
    a.nl += b.nl;
    a.ns += b.ns;
#pragma unroll
    for (int k = 0; k < 4; ++k) a.nd[k] += b.nd[k];
}

// Add sums to a problem's step accumulators (one thread); the fixed-point
// additions make the result independent of the order of the calls.
__device__ __forceinline__ void emit_sums(const WarpSums& w, DevStats* st)
{
    StepStripe* c = my_stripe(st);
    acc_add_fx(&c->energy, w.e);
    acc_add_fx(&c->flux, w.f);
    if (w.nl) atomicAdd(&c->liquid, (unsigned long long)w.nl);
    if (w.ns) atomicAdd(&c->shifted, (unsigned long long)w.ns);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (w.nd[k]) atomicAdd(&c->dir[k], (unsigned long long)w.nd[k]);
}

// A warp's partial sums in a fixed lane order, then exact fixed-point atomics.
template <typename P>
__device__ __forceinline__ void flush_tile_sums(const Acc<P>& acc, const TileSums& ts, DevStats* st, int lane)
{
    const WarpSums w = warp_tile_sums<P>(acc, ts);
    if (lane == 0) emit_sums(w, st);
}

// Target of M0(q) at a Dirichlet node on wall k (Eq. 14 with theta' = theta_D,
// Eq. 15): m0t = theta_D - (phi(theta) - phi(theta_D))/Ste, theta = M0(f) of
// the node; EEBM (Algorithm 2 keeps H = M0): the wall value's enthalpy.
// FP64 form: the wall node stays within rounding of theta_D, so the phi
// difference uses the tanh addition theorem with tanh(z) = z - z^3/3 + 2z^5/15
// for |z| <= 1e-4 (remainder < 1e-29), else tanh.
__device__ __forceinline__ double dir_m0_target_d(double th, int k, const Problem& pb)
{
    if (pb.method == 1) return pb.wall_H[k];
    const double z = (th - pb.wall_theta[k]) * pb.inv_delta;
    double dphi;
    if (fabs(z) <= 1e-4) {
        const double z2 = z * z;
        const double tz = z * (1.0 - z2 * (1.0 / 3.0 - z2 * (2.0 / 15.0)));
        const double td = pb.wall_tanh[k];
        dphi = 0.5 * tz * (1.0 - td) * (1.0 + td) / (1.0 + td * tz);   // phi(theta) - phi(theta_D)
    } else {
        dphi = phi_of(th, pb.inv_delta) - pb.wall_phi[k];
    }
    return pb.wall_theta[k] - dphi * pb.inv_ste;
}

// FP32 form as a float-float pair, with no FP64 instruction on the common
// path: phi(theta) - phi(theta_D) = phi'(theta_D)(theta - theta_D) +
// O((theta - theta_D)^2/delta^2), and the second-order term is below 1e-8 of
// FP32 resolution whenever |theta - theta_D| <= 1e-4 delta; otherwise the FP64
// expression is used.
__device__ __forceinline__ ff dir_m0_target_f(const ff& th, int k, const Problem& pb)
{
    if (pb.method == 1) return ff{pb.wall_H_hi[k], pb.wall_H_lo[k]};
    const float dth = (th.hi - pb.wall_th_hi[k]) + (th.lo - pb.wall_th_lo[k]);
    ff m0t{pb.wall_th_hi[k], pb.wall_th_lo[k]};
    if (fabsf(dth) <= pb.wall_dth_max) {
        ff_add(m0t, -pb.wall_slope[k] * dth);
    } else {
        const double dphi = phi_of(ff_to_double(th), pb.inv_delta) - pb.wall_phi[k];
        ff_add(m0t, (float)(-dphi * pb.inv_ste));
    }
    return m0t;
}

// ---------------------------------------------------------------- deferred Newton nodes
// One node whose local Newton solve was deferred (Eq. 14, mixed-precision
// form): theta' = m0 + (phi(theta) - phi(root))/Ste, c = theta' - (1-omega) m0,
// and the node's stored q_i are relaxed in place, Omega~_i = (1-omega) q_i +
// w_i c (Q = 9 or 5 planes of the step's output state[parity ^ 1]).  The
// result carries the node's energy term theta' + phi(theta')/Ste as an exact
// fixed-point value, its iteration count and its problem's statistics index.
struct NewtonResult {
    Fx e{0, 0ull};
    int it = 0;
    int sidx = -1;   // -1: no node (an idle lane)
};

template <typename P, bool REC, int Q>
__device__ __forceinline__ NewtonResult newton_job_apply(const NewtonJob& jb, const Problem& pb, int parity,
                                                         double* rec, DevStats* stats)
{
    NewtonResult r;
    r.sidx = pb.stats;
    // the stored q_i were written earlier in this launch, possibly by another
    // SM: load them from L2 (ld.global.cg), never from this SM's L1; the loads
    // are issued first so that their latency overlaps the solve
    const int x = jb.node % pb.nx, y = jb.node / pb.nx;
    const long long at = (long long)(y + 1) * pb.pitch + x;
    P* d = static_cast<P*>(pb.state[parity ^ 1]) + at;
    P qv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) qv[i] = __ldcg(d + i * pb.plane);
    double m0, th, sh = 0.0;
    if constexpr (sizeof(P) == 4) {
        // FP32 form: the job carries only the node; m0 = M0(q) from the stored
        // unrelaxed q_i and theta = M0(f) = sum of the node's Omega_i(t) (the
        // step's source state), both as float-float sums in the order the
        // step kernel uses (last plane first), plus the state's shift s
        const P* sv = static_cast<const P*>(pb.state[parity]) + at;
        ff mm{0.f, 0.f}, t{0.f, 0.f};
#pragma unroll
        for (int i = Q - 1; i >= 0; --i) {
            ff_add(t, __ldg(sv + i * pb.plane));
            ff_add(mm, qv[i]);
        }
        sh = (double)state_shift(pb, parity);
        m0 = ff_to_double(mm) + sh;
        th = ff_to_double(t) + sh;
    } else {
        m0 = jb.m0;
        th = jb.theta;
    }
    const double pth = phi_of(th, pb.inv_delta);
    const NewtonOut nr = newton_mixed(m0, th, pth, pb);
    if (!nr.ok || !isfinite(nr.root)) atomicCAS(&stats[r.sidx].error, 0, 3);
    const double tn = m0 + (pth - nr.phi_root) * pb.inv_ste;
    // c = theta' - (1-omega) m0; stored values less w_i s: c - omega s
    const P c = (P)((tn - sh) - (1.0 - pb.omega) * (m0 - sh));
    const P omc = (P)(1.0 - pb.omega);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const P wi = lat_wp<P>(Q, i);
        d[i * pb.plane] = fma(omc, qv[i], wi * c);
    }
    (void)x;
    if (REC) rec[(long long)y * pb.pitch + x] = tn;
    r.e = to_fixed(tn + nr.phi_root * pb.inv_ste);
    r.it = nr.iters;
    return r;
}

// The warp's results, grouped by problem: the lowest lane of each group sums
// its group's energy terms exactly and adds them, the node count, the
// iteration sum and the largest iteration count once.
__device__ __forceinline__ void newton_group_add(const NewtonResult& r, DevStats* stats)
{
    const int lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(kFull, r.sidx);
    const int leader = __ffs(grp) - 1;
    Fx sum{0, 0ull};
    int n = 0, mx = 0, its = 0;
    for (int l = 0; l < 32; ++l) {
        Fx v;
        v.hi = __shfl_sync(kFull, r.e.hi, l);
        v.lo = __shfl_sync(kFull, r.e.lo, l);
        const int vi = __shfl_sync(kFull, r.it, l);
        if ((grp >> l) & 1) {
            fx_add(sum, v);
            ++n;
            mx = max(mx, vi);
            its += vi;
        }
    }
    if (lane == leader && r.sidx >= 0) {
        DevStats* st = &stats[r.sidx];
        StepStripe* c = my_stripe(st);
        acc_add_fx(&c->energy, sum);
        atomicAdd(&c->newton, (unsigned long long)n);
        atomicAdd(&c->iters, (unsigned long long)its);
        atomicMax(&st->cur_maxit, mx);
    }
}

// ---------------------------------------------------------------- mbarriers and TMA
// Used by the warp-specialized TMA step kernel: a producer
// lane issues tiled tensor loads of whole rows into a ring of shared-memory
// slots, each completing on the slot's `full` mbarrier; consumers release a
// slot on its `empty` mbarrier.  Every wait is bounded.
constexpr int kTmaWaitLimit = 1 << 24;   // most try_wait calls of one wait (the time limit comes first)

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(b)) : "memory");
}
// try_wait: the thread sleeps in hardware until the phase completes or a short
// time limit passes, instead of spinning on issue slots the other warps need
// (measured 3 % faster than a test_wait spin)
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_addr(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of an mbarrier for at most limit_ns nanoseconds
// (and at most kTmaWaitLimit polls); false when the wait gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* b, unsigned parity, long long limit_ns)
{
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < kTmaWaitLimit; ++i) {
        if (mbar_try_wait(b, parity)) return true;
        if ((long long)(global_ns() - t0) > limit_ns) return false;
    }
    return false;
}
// one row of every plane of the tensor map, box origin (x, row, plane 0)
__device__ __forceinline__ void tma_load_rows(const CUtensorMap* m, float* dst, unsigned long long* bar, int x, int row)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        ::"r"(smem_addr(dst)), "l"(m), "r"(x), "r"(row), "r"(0), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

}  // namespace lbm
