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
};

// A warp's partial sums in a fixed lane order, then exact fixed-point atomics;
// node counts go to integer counters (the publisher adds their phi/Ste terms).
template <typename P>
__device__ __forceinline__ void flush_tile_sums(const Acc<P>& acc, const TileSums& ts, DevStats* st, int lane)
{
    Fx e, f;
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
        e = float_to_fixed(se.hi);
        fx_add(e, float_to_fixed(se.lo));
        f = float_to_fixed(sf.hi);
        fx_add(f, float_to_fixed(sf.lo));
    } else {
        e = to_fixed(warp_sum(acc.get()));
        f = to_fixed(warp_sum(ts.flux));
    }
    const int nl = warp_sum_i(ts.liquid);
    int nd[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) nd[w] = warp_sum_i(ts.dir_count[w]);
    if (lane == 0) {
        acc_add_fx(&st->cur_energy, e);
        acc_add_fx(&st->cur_flux, f);
        if (nl) atomicAdd(&st->cur_liquid, (unsigned long long)nl);
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (nd[w]) atomicAdd(&st->cur_dir[w], (unsigned long long)nd[w]);
    }
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

// ---------------------------------------------------------------- mbarriers and TMA
// Used by the warp-specialized TMA step kernel: a producer
// lane issues tiled tensor loads of whole rows into a ring of shared-memory
// slots, each completing on the slot's `full` mbarrier; consumers release a
// slot on its `empty` mbarrier.  Every wait is bounded.
constexpr int kTmaWaitLimit = 1 << 20;   // try_wait calls before a wait gives up

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
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* b, unsigned parity)
{
    for (int i = 0; i < kTmaWaitLimit; ++i)
        if (mbar_try_wait(b, parity)) return true;
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
