// Device helpers of the IREBM kernels: lattice constants, float-float sums,
// the regularized liquid fraction, the local Newton solve of Eq. (14),
// deterministic fixed-point reductions and the end-of-launch statistics.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lbm_internal.h"

namespace lbm {

constexpr unsigned kFull = 0xffffffffu;

// |x| >= kSat * delta  =>  tanh(x/delta) is +-1 in FP64 (1 - tanh(19.5) ~ 2e-17,
// below half an ulp of 1), so phi is exactly 0 or 1 there and phi' is 0.
constexpr double kSat = 19.5;

// ---------------------------------------------------------------- D2Q9 / D1Q3 / D2Q5
// D2Q9 velocities (Sec. 3.2): 0 rest; 1..4 = (+1,0),(0,+1),(-1,0),(0,-1);
// 5..8 = (+1,+1),(-1,+1),(-1,-1),(+1,-1).  Weights 4/9, 1/9, 1/36 (c_s^2 = 1/3).
__host__ __device__ constexpr int d2_ex(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int d2_ey(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int d2_opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }
__host__ __device__ constexpr double d2_w(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
// D1Q3: 0 rest, 1 = +1, 2 = -1; weights 2/3, 1/6, 1/6.
__host__ __device__ constexpr int d1_ex(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }
__host__ __device__ constexpr double d1_w(int i) { return i == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
// D2Q5: 0 rest, 1..4 = (+1,0),(0,+1),(-1,0),(0,-1) as in D2Q9; weights 1/3, 1/6 (c_s^2 = 1/3).
__host__ __device__ constexpr double d5_w(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
// weight i of the lattice with q velocities (3, 5 or 9)
__host__ __device__ constexpr double lat_w(int q, int i) { return q == 9 ? d2_w(i) : (q == 5 ? d5_w(i) : d1_w(i)); }

// FP32 weights.  The nearest floats to 4/9, 1/9, 1/36 sum to 1 + 2^-27, and
// those to 1/3, 1/6 (D2Q5) to 1 + 2^-25.  A relaxation toward w_i c in FP32
// multiplies the zeroth moment by that sum every step: on the 4096^2 melting
// workload (tau = 1) theta drifted by 7.5e-9 of itself per step, 2.5e-5 after
// 10,000 steps.  Here one weight of each set is one ulp below the nearest
// float (1/36, resp. 1/3), so that each set sums to exactly 1; the products
// w_i c still round, but without a bias.
__host__ __device__ constexpr float d2_wf(int i) { return i == 0 ? 0x1.c71c72p-2f : (i <= 4 ? 0x1.c71c72p-4f : 0x1.c71c70p-6f); }
__host__ __device__ constexpr float d5_wf(int i) { return i == 0 ? 0x1.555554p-2f : 0x1.555556p-3f; }
// the weights of the population precision P (float: the exact-sum sets above)
template <typename P> __host__ __device__ constexpr P lat_wp(int q, int i);
template <> __host__ __device__ constexpr float lat_wp<float>(int q, int i)
{
    return q == 9 ? d2_wf(i) : (q == 5 ? d5_wf(i) : (float)d1_w(i));
}
template <> __host__ __device__ constexpr double lat_wp<double>(int q, int i) { return lat_w(q, i); }

// ---------------------------------------------------------------- float-float
// Unevaluated sum hi + lo of two floats; two_sum is Knuth's error-free
// transformation (no fast-math: the compiler keeps the order of operations).
struct ff {
    float hi, lo;
};
__device__ __forceinline__ void ff_add(ff& a, float b)
{
    float s = __fadd_rn(a.hi, b);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}
__device__ __forceinline__ double ff_to_double(const ff& a) { return (double)a.hi + (double)a.lo; }

// Approximate float of a double from its high word only (sign, exponent and
// 20 mantissa bits; relative error < 2^-20), using the integer pipe.  Values
// below 2^-126 in magnitude give 0; non-finite or huge values give NaN.
__device__ __forceinline__ float approx_float(double d)
{
    int hi = __double2hiint(d);
    int e = (hi >> 20) & 0x7ff;
    int bits = (hi & 0x80000000) | (((hi & 0x7fffffff) - (896 << 20)) << 3);
    float r = __int_as_float(bits);
    return e <= 896 ? 0.0f : (e >= 1151 ? __int_as_float(0x7fc00000) : r);
}

// ---------------------------------------------------------------- liquid fraction
// EEBM (Algorithm 2): temperature of an enthalpy, Theta(H) = H below 0, 0 on
// the melting plateau [0, 1/Ste], H - 1/Ste above it.
__device__ __forceinline__ double eebm_theta(double H, double inv_ste)
{
    return H < 0.0 ? H : (H > inv_ste ? H - inv_ste : 0.0);
}
__device__ __forceinline__ float eebm_theta(float H, float inv_ste)
{
    return H < 0.0f ? H : (H > inv_ste ? H - inv_ste : 0.0f);
}

// phi(x) = (1 + tanh(x/delta))/2 (Sec. 4.1) and phi' = (1 - t)(1 + t)/(2 delta).
__device__ __forceinline__ double phi_of(double x, double inv_delta) { return 0.5 + 0.5 * tanh(x * inv_delta); }

// Local Newton solve of Eq. (14): the root of
//   F(x) = (x - m0) + (phi(x) - phi(theta))/Ste,   F' = 1 + phi'(x)/Ste >= 1,
// from x = theta (Algorithm 3).  Safeguard: the root lies in
// [m0 + (phi(theta) - 1)/Ste, m0 + phi(theta)/Ste]; a Newton iterate that
// leaves the current bracket, or does not at least halve the update before
// last, is replaced by the bracket midpoint (this also breaks 2-cycles).
// Converged when an update moves x by at most tol*max(1,|x|) (tested before
// the safeguard), when F = 0, or when the bracket is that narrow.
struct NewtonOut {
    double root;
    double phi_root;
    int iters;
    bool ok;
};

__device__ __forceinline__ NewtonOut newton_solve(double m0, double theta, double phi_theta, double inv_ste,
                                                  double inv_delta, double tol, int maxit)
{
    double lo = m0 + (phi_theta - 1.0) * inv_ste, hi = m0 + phi_theta * inv_ste;
    double x = theta;
    double step_old = hi - lo, step = step_old;
    NewtonOut r;
    for (int k = 0; k < maxit; ++k) {
        double t = tanh(x * inv_delta);
        double ph = 0.5 + 0.5 * t;
        double F = (x - m0) + (ph - phi_theta) * inv_ste;
        if (F == 0.0) {
            r.root = x; r.phi_root = ph; r.iters = k; r.ok = true;
            return r;
        }
        if (F < 0.0) lo = fmax(lo, x);
        else hi = fmin(hi, x);
        double dph = 0.5 * (1.0 - t) * (1.0 + t) * inv_delta;
        double xn = x - F / (1.0 + dph * inv_ste);
        double sc = tol * fmax(1.0, fabs(x));
        if (fabs(xn - x) <= sc) {
            // |xn - x| <= ~1e-14: phi(xn) = ph + phi'(x)(xn - x) to far below one ulp
            r.root = xn; r.phi_root = ph + dph * (xn - x); r.iters = k + 1; r.ok = true;
            return r;
        }
        if (!(xn >= lo && xn <= hi) || fabs(xn - x) > 0.5 * step_old) {
            step_old = step;
            step = 0.5 * (hi - lo);
            xn = lo + step;
            if (step <= tol * fmax(1.0, fabs(xn))) {
                r.root = xn; r.phi_root = phi_of(xn, inv_delta); r.iters = k + 1; r.ok = true;
                return r;
            }
        } else {
            step_old = step;
            step = fabs(xn - x);
        }
        x = xn;
    }
    r.root = x; r.phi_root = phi_of(x, inv_delta); r.iters = maxit; r.ok = false;
    return r;
}

// Mixed-precision form of the same solve (same root, same stopping rule).
//  1. FP32 Newton (tanhf) locates the root to FP32 accuracy, x0 (it stops at
//     FP32 precision or once its updates stop halving).
//  2. FP64 step from x0: one FP64 tanh gives t = tanh(x0/delta), F, F', F''
//     and F''' (F^(k) = phi^(k)/Ste, phi2 = -t(1-t^2)/delta^2,
//     phi3 = (1-t^2)(3t^2-1)/delta^3), the Newton update dn = -F/F' (1/F' from
//     an FP32 reciprocal and one FP64 Newton step: relative error ~1e-14) and
//     Halley's update d = dn / (1 + dn F''/(2F')).  Halley's error e is about
//     |F''^2/(4F'^2) - F'''/(6F')| |dn|^3, and theta' = m0 + (phi(theta) -
//     phi(root))/Ste inherits it as (F' - 1) e; when F' e is below
//     0.1 tol max(1,|x|) and |d| <= 3e-5 delta, x0 + d is accepted and
//     phi(x0 + d) comes from the cubic Taylor expansion (the quartic remainder
//     is below (d/delta)^4 / 12 < 1e-19).  From the FP32 start (|dn| ~ 1e-8)
//     one FP64 evaluation suffices; a plain Newton step would leave F' e ~
//     |F''| dn^2 / 2, above the tolerance in the middle of the band, and need a
//     second one.  Otherwise the FP64 iteration goes on.  Iterations of both
//     precisions count against maxit.
//  3. Anything unexpected (no FP32 convergence, an FP64 update larger than
//     1e-3 delta) falls back to newton_solve from theta.
// The FP32 and derived constants come converted in the Problem: on this GPU
// every FP64 instruction, conversions included, shares the narrow FP64 pipe.
__device__ __forceinline__ NewtonOut newton_mixed(double m0, double theta, double phi_theta, const Problem& pb)
{
    const double inv_ste = pb.inv_ste, inv_delta = pb.inv_delta, tol = pb.tol;
    const int maxit = pb.maxit;
    const float mf = (float)m0, pf = (float)phi_theta, isf = pb.inv_ste_f, idf = pb.inv_delta_f;
    float lo = mf + (pf - 1.0f) * isf, hi = mf + pf * isf;
    float x = (float)theta;
    const float xfloor = pb.delta_f;
    float step_prev = hi - lo;
    int k = 0;
    // FP32 stage: plain Newton inside the bracket; it stops at FP32 precision or
    // when the update no longer halves (the FP32 rounding floor of F is reached).
    // Only an iterate that leaves the bracket is replaced by the midpoint.
    for (; k < 16; ++k) {
        const float t = tanhf(x * idf);
        const float F = (x - mf) + (0.5f * t + 0.5f - pf) * isf;
        if (F == 0.0f) break;
        if (F < 0.0f) lo = fmaxf(lo, x);
        else hi = fminf(hi, x);
        const float dph = 0.5f * (1.0f - t) * (1.0f + t) * idf;
        float xn = x - F / (1.0f + dph * isf);
        if (!(xn >= lo && xn <= hi)) {
            xn = 0.5f * (lo + hi);
        } else {
            const float st = fabsf(xn - x);
            if (st <= 1e-7f * fmaxf(fabsf(x), xfloor) || (k >= 2 && st >= 0.5f * step_prev)) {
                x = xn;
                ++k;
                break;
            }
            step_prev = st;
        }
        x = xn;
    }
    const bool conv32 = isfinite(x);
    const double delta = pb.delta;
    if (conv32) {
        double xd = (double)x;
        for (int j = 0; j < 3; ++j) {
            const double t = tanh(xd * inv_delta);
            const double s = (1.0 - t) * (1.0 + t);
            const double ph = 0.5 + 0.5 * t;
            const double F = (xd - m0) + (ph - phi_theta) * inv_ste;
            const double dph = 0.5 * s * inv_delta;
            const double Fp = 1.0 + dph * inv_ste;
            const double r0 = (double)(1.0f / (float)Fp);
            const double rinv = fma(r0, fma(-Fp, r0, 1.0), r0);
            const double dn = -F * rinv;   // Newton update
            const double adn = fabs(dn);
            if (adn > 1e-3 * delta) break;   // FP32 start not close enough: full FP64 solve
            const double p2 = -t * s * pb.inv_delta2;                   // second derivative of phi
            const double p3 = s * (3.0 * t * t - 1.0) * pb.inv_delta3;  // third derivative of phi
            // Halley update d = dn / (1 + dn F''/(2F')), 1/(1 + eps) to second order (accepted only
            // for |eps| <= 1e-4: the neglected eps^3 |dn| is below 1e-12 |dn|)
            const double eps = 0.5 * dn * p2 * inv_ste * rinv;
            const double d = dn * (1.0 - eps + eps * eps);
            const double ad = fabs(d);
            const double x1 = xd + d;
            const double sc = tol * fmax(1.0, fabs(xd));
            // theta' = m0 + (phi(theta) - phi(x))/Ste carries a root error e as (F' - 1) e;
            // after the Halley step F' e ~ |F''^2/(4F') - F'''/6| |dn|^3
            const double g = (0.25 * p2 * p2 * inv_ste * rinv + fabs(p3) * (1.0 / 6.0)) * inv_ste;
            if (ad <= sc || (ad <= 3e-5 * delta && fabs(eps) <= 1e-4 && g * adn * adn * adn <= 0.1 * sc)) {
                NewtonOut r;
                r.root = x1;
                r.phi_root = ph + d * (dph + d * (0.5 * p2 + d * p3 * (1.0 / 6.0)));
                r.iters = k + j + 1;
                r.ok = r.iters <= maxit;
                return r;
            }
            xd = x1;
        }
    }
    NewtonOut r = newton_solve(m0, theta, phi_theta, inv_ste, inv_delta, tol, maxit);
    r.iters += k;
    r.ok = r.ok && r.iters <= maxit;
    return r;
}

// ---------------------------------------------------------------- lane shifts
// A warp-wide row of 32*N values held N per lane, shifted by one element.
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

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ int warp_max_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// 128-bit fixed-point value (scaled by 2^60) as a register pair; adding two of
// them is exact, so sums in this form do not depend on the order of terms.
struct Fx {
    long long hi;
    unsigned long long lo;
};

__device__ __forceinline__ Fx to_fixed(double v)
{
    Fx f;
    const double s = v * 0.0625;   // v * 2^60 / 2^64
    const double h = floor(s);
    const double r = s - h;        // in [0, 1), exact
    f.hi = (long long)h;
    f.lo = __double2ull_rz(r * 18446744073709551616.0);
    return f;
}

__device__ __forceinline__ void fx_add(Fx& a, const Fx& b)
{
    const unsigned long long lo = a.lo + b.lo;
    a.hi += b.hi + (lo < a.lo ? 1 : 0);
    a.lo = lo;
}

__device__ __forceinline__ void acc_add_fx(Acc128* a, const Fx& v)
{
    if (v.hi == 0 && v.lo == 0) return;
    const unsigned long long old = atomicAdd(&a->lo, v.lo);
    const long long carry = (old + v.lo < old) ? 1 : 0;
    atomicAdd(reinterpret_cast<unsigned long long*>(&a->hi), (unsigned long long)(v.hi + carry));
}

// Exact fixed-point value of a float with integer operations only (no FP64
// instruction): v = m * 2^(e-150), scaled by 2^60.  Bits below 2^-60 are dropped.
__device__ __forceinline__ Fx float_to_fixed(float v)
{
    Fx f{0, 0ull};
    const unsigned bits = __float_as_uint(v);
    const int e = (bits >> 23) & 0xff;
    unsigned long long m = bits & 0x7fffffu;
    if (e == 0 && m == 0) return f;
    if (e != 0) m |= 0x800000u;
    const int sh = (e == 0 ? 1 : e) - 90;   // m * 2^(e - 150 + 60)
    unsigned long long lo = 0, hi = 0;
    if (sh >= 0) {
        if (sh < 64) {
            lo = m << sh;
            hi = sh > 40 ? (m >> (64 - sh)) : 0ull;
        } else {
            hi = m << (sh - 64);
        }
    } else if (sh > -64) {
        lo = m >> (-sh);
    }
    if (bits >> 31) {   // two's complement of the 128-bit value
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    f.lo = lo;
    f.hi = (long long)hi;
    return f;
}

// Add v into the 128-bit fixed-point accumulator.
__device__ __forceinline__ void acc_add(Acc128* a, double v)
{
    if (v == 0.0) return;
    acc_add_fx(a, to_fixed(v));
}

__device__ __forceinline__ double acc_read(const Acc128* a)
{
    volatile const Acc128* va = a;
    unsigned long long lo = va->lo;
    long long hi = va->hi;
    return (double)hi * 16.0 + (double)lo * 0x1p-60;
}

__device__ __forceinline__ void acc_clear(Acc128* a)
{
    volatile Acc128* va = a;
    va->lo = 0ull;
    va->hi = 0ll;
}

// The per-step sums (AccSum): return-less additions of the four limbs, so a
// thread never waits for them.
__device__ __forceinline__ void acc_add_fx(AccSum* a, const Fx& v)
{
    const unsigned long long lo = v.lo, hi = (unsigned long long)v.hi;
    if (lo == 0ull && hi == 0ull) return;
    atomicAdd(&a->limb[0], lo & 0xffffffffull);
    atomicAdd(&a->limb[1], lo >> 32);
    atomicAdd(&a->limb[2], hi & 0xffffffffull);
    atomicAdd(&a->limb[3], hi >> 32);
}

__device__ __forceinline__ void acc_add(AccSum* a, double v)
{
    if (v == 0.0) return;
    acc_add_fx(a, to_fixed(v));
}

// sum_k limb[k] 2^(32k) modulo 2^128, as a double
__device__ __forceinline__ double acc_read(const AccSum* a)
{
    volatile const unsigned long long* l = a->limb;
    const unsigned long long s0 = l[0], s1 = l[1], s2 = l[2], s3 = l[3];
    const unsigned long long lo = s0 + (s1 << 32);
    const unsigned long long carry = lo < s0 ? 1ull : 0ull;
    const unsigned long long hi = (s1 >> 32) + s2 + (s3 << 32) + carry;
    return (double)(long long)hi * 16.0 + (double)lo * 0x1p-60;
}

__device__ __forceinline__ void acc_clear(AccSum* a)
{
    volatile unsigned long long* l = a->limb;
    l[0] = l[1] = l[2] = l[3] = 0ull;
}

// The stripe a thread adds into: spread over blocks and warps.
__device__ __forceinline__ StepStripe* my_stripe(DevStats* st)
{
    return &st->cur[(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % kStripes];
}

// Totals of one problem's stripes.
struct StatSums {
    unsigned long long e[4], f[4], dir[4], newton, iters, liquid, shifted;
};

// The shift s of a state (FP32 D2Q9 / D2Q5; 0 for the other forms): its tail.
__device__ __forceinline__ float state_shift(const Problem& pb, int parity)
{
    return __ldg(reinterpret_cast<const float*>(static_cast<const char*>(pb.state[parity]) + pb.tail_off));
}

// Read one stripe into `s` and clear it.
__device__ __forceinline__ void stripe_take(StepStripe* stripe, StatSums& s)
{
    volatile StepStripe* c = stripe;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        s.e[j] += c->energy.limb[j];
        s.f[j] += c->flux.limb[j];
        s.dir[j] += c->dir[j];
    }
    s.newton += c->newton;
    s.iters += c->iters;
    s.liquid += c->liquid;
    s.shifted += c->shifted;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c->energy.limb[j] = 0ull;
        c->flux.limb[j] = 0ull;
        c->dir[j] = 0ull;
    }
    c->newton = 0ull;
    c->iters = 0ull;
    c->liquid = 0ull;
    c->shifted = 0ull;
}

// The published step statistics from the stripe totals.
// E = fixed-point sum + (liquid nodes + sum_w Dirichlet nodes of wall w * phi(theta_w)) / Ste.
__device__ __forceinline__ void publish_totals(DevStats* st, const Problem* pb, const StatSums& s)
{
    // every input first, as independent L2 loads (ld.global.cg), so that the
    // publication waits for about one memory round trip, not one per field
    const int have = __ldcg(&st->have_energy);
    const double e_old = __ldcg(&st->energy), imax = __ldcg(&st->imbalance_max);
    const long long steps = __ldcg(&st->steps);
    const int cmax = __ldcg(&st->cur_maxit);
    double inv_ste = 0.0, wphi[4] = {0.0, 0.0, 0.0, 0.0};
    float shift = 0.0f;
    if (pb) {
        inv_ste = pb->inv_ste;
#pragma unroll
        for (int w = 0; w < 4; ++w) wphi[w] = pb->wall_phi[w];
        if (s.shifted) shift = state_shift(*pb, 0);
    }
    AccSum esum, fsum;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        esum.limb[j] = s.e[j];
        fsum.limb[j] = s.f[j];
    }
    double e = acc_read(&esum);
    const double f = acc_read(&fsum);
    if (pb) {
        double c = (double)s.liquid;
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (s.dir[w]) c += (double)s.dir[w] * wphi[w];
        e += c * inv_ste;
        if (s.shifted) e += (double)s.shifted * (double)shift;
    }
    const double imb = have ? e - e_old - f : 0.0;
    __stcg(&st->imbalance, imb);
    if (have && fabs(imb) > imax) __stcg(&st->imbalance_max, fabs(imb));
    __stcg(&st->energy_prev, e_old);
    __stcg(&st->energy, e);
    __stcg(&st->flux, f);
    __stcg(&st->have_energy, 1);
    __stcg(&st->steps, steps + 1);
    __stcg(&st->newton_nodes, (long long)s.newton);
    __stcg(&st->newton_iters, (long long)s.iters);
    __stcg(&st->newton_max_iter, cmax);
    __stcg(&st->cur_maxit, 0);
}

// Publish one problem's step statistics and clear its stripes (one thread of
// the last block).
__device__ __forceinline__ void publish_stats(DevStats* st, const Problem* pb)
{
    StatSums s = {};
    for (int k = 0; k < kStripes; ++k) stripe_take(&st->cur[k], s);
    publish_totals(st, pb, s);
}

// The same with one warp: lane k takes stripe k, the warp adds the totals
// (integer sums: the result is the one thread's), lane 0 publishes.
__device__ __forceinline__ void publish_stats_warp(DevStats* st, const Problem* pb, int lane)
{
    static_assert(kStripes == 32, "one stripe per lane");
    StatSums s = {};
    stripe_take(&st->cur[lane], s);
    unsigned long long* v = &s.e[0];   // the 16 fields in order
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
    if (lane == 0) publish_totals(st, pb, s);
}

// Last-block pattern: every block calls this after its warps have added their
// partial sums; the block that arrives last publishes the statistics of all
// problems (one thread per problem) and resets the ticket.  No block waits.
__device__ __forceinline__ void finish_launch(DevStats* stats, int nprob, unsigned int* ticket)
{
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        for (int p = threadIdx.x; p < nprob; p += blockDim.x) publish_stats(&stats[p], nullptr);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

}  // namespace lbm
