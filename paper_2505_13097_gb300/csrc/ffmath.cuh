// Float-float arithmetic (a value as the unevaluated sum hi + lo of two
// floats, about 48 significant bits) for the FP32 form's Newton solves.  On
// GB300 an FP64 instruction issues at 1/64 of the FP32 rate, so the solves of
// the front band (Eq. 14) run their refinement on the FP32 pipe instead.
//
// Building blocks (error-free transformations):
//   two_sum (Knuth): s + e = a + b exactly;
//   fast_two_sum (Dekker): the same when |a| >= |b|;
//   two_prod: p + e = a * b exactly, e from one fused multiply-add.
// Sums, products and the quotient follow Dekker's double-length algorithms
// (Dekker 1971; the accurate sum adds the low parts with their own error).
//
// exp(y) for y <= 0: y = k ln2 + r with k = rint(y / ln2), ln2 split into
// three floats (Cody and Waite; the first with 15 significant bits, so k L1 is
// exact for |k| < 512), |r| <= ln2 / 2, then the Taylor series of exp(r):
// orders 7 .. 13 in float by Horner's rule (their sum, about 1/7!, times r^7
// is below 2e-7, so its float rounding stays below 1e-14), orders 0 .. 6 in
// float-float, and the result scaled by 2^k.  The series' remainder after
// order 13 is below (ln2/2)^14 / 14! < 1e-17.  Relative error about 1e-14.
//
// The same source compiles for the host (plain IEEE float operations, no
// contraction) so that a host program can check it against long double.
#pragma once

#ifndef __CUDACC__
#include <cmath>
#define __host__
#define __device__
#define __forceinline__ inline
#endif

#if defined(__CUDA_ARCH__)
#define FF_ADD(a, b) __fadd_rn((a), (b))
#define FF_SUB(a, b) __fsub_rn((a), (b))
#define FF_MUL(a, b) __fmul_rn((a), (b))
#define FF_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#define FF_DIV(a, b) __fdiv_rn((a), (b))
#define FF_RINT(a) rintf(a)
#else
#define FF_ADD(a, b) ((float)((float)(a) + (float)(b)))
#define FF_SUB(a, b) ((float)((float)(a) - (float)(b)))
#define FF_MUL(a, b) ((float)((float)(a) * (float)(b)))
#define FF_FMA(a, b, c) std::fmaf((a), (b), (c))
#define FF_DIV(a, b) ((float)((float)(a) / (float)(b)))
#define FF_RINT(a) std::rintf(a)
#endif

#define FF_HD __host__ __device__ __forceinline__

namespace lbm {

struct ff {
    float hi, lo;
};

FF_HD ff two_sum(float a, float b)
{
    const float s = FF_ADD(a, b);
    const float bb = FF_SUB(s, a);
    const float e = FF_ADD(FF_SUB(a, FF_SUB(s, bb)), FF_SUB(b, bb));
    return ff{s, e};
}

FF_HD ff fast_two_sum(float a, float b)
{
    const float s = FF_ADD(a, b);
    return ff{s, FF_SUB(b, FF_SUB(s, a))};
}

FF_HD ff two_prod(float a, float b)
{
    const float p = FF_MUL(a, b);
    return ff{p, FF_FMA(a, b, -p)};
}

FF_HD ff ff_neg(const ff& a) { return ff{-a.hi, -a.lo}; }

// a + b, both float-float (accurate form: the low parts' sum keeps its error)
FF_HD ff ff_sum(const ff& a, const ff& b)
{
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo = FF_ADD(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = FF_ADD(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

FF_HD ff ff_sum_f(const ff& a, float b)
{
    ff s = two_sum(a.hi, b);
    s.lo = FF_ADD(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

FF_HD ff ff_prod(const ff& a, const ff& b)
{
    ff p = two_prod(a.hi, b.hi);
    p.lo = FF_FMA(a.hi, b.lo, FF_FMA(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

FF_HD ff ff_prod_f(const ff& a, float b)
{
    ff p = two_prod(a.hi, b);
    p.lo = FF_FMA(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// a / b: a float quotient, the float-float remainder a - q b, one correction
FF_HD ff ff_quot(const ff& a, const ff& b)
{
    const float q1 = FF_DIV(a.hi, b.hi);
    const ff r = ff_sum(a, ff_neg(ff_prod_f(b, q1)));
    const float q2 = FF_DIV(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

FF_HD float ff_float(const ff& a) { return FF_ADD(a.hi, a.lo); }

// exp(y) for y <= 0 (see the header); 0 below y = -80 (exp < 2e-35).
FF_HD ff ff_exp_nonpos(const ff& y)
{
    if (!(y.hi > -80.0f)) return ff{0.0f, 0.0f};
    const float kL1 = 0x1.62e4p-1f, kL2 = 0x1.7f7d1cp-20f, kL3 = 0x1.ef357ap-45f;
    const float k = FF_RINT(FF_MUL(y.hi, 0x1.715476p+0f));
    // r = y - k ln2: y.hi - k L1 is exact (k L1 exact; Sterbenz), then the rest
    const float t1 = FF_SUB(y.hi, FF_MUL(k, kL1));
    const ff p2 = two_prod(k, kL2);
    ff r = two_sum(t1, -p2.hi);
    r.lo = FF_ADD(r.lo, FF_SUB(FF_SUB(y.lo, p2.lo), FF_MUL(k, kL3)));
    r = fast_two_sum(r.hi, r.lo);
    // orders 13 .. 7 in float
    float s = 0x1.612462p-33f;
    s = FF_FMA(s, r.hi, 0x1.1eed8ep-29f);
    s = FF_FMA(s, r.hi, 0x1.ae6456p-26f);
    s = FF_FMA(s, r.hi, 0x1.27e4fcp-22f);
    s = FF_FMA(s, r.hi, 0x1.71de3ap-19f);
    s = FF_FMA(s, r.hi, 0x1.a01a02p-16f);
    s = FF_FMA(s, r.hi, 0x1.a01a02p-13f);
    // orders 6 .. 0 in float-float: p = ((s r + c6) r + c5) r ... + 1
    ff p = ff_sum(ff_prod_f(r, s), ff{0x1.6c16c2p-10f, -0x1.27d27ep-35f});
    p = ff_sum(ff_prod(p, r), ff{0x1.111112p-7f, -0x1.dddddep-32f});
    p = ff_sum(ff_prod(p, r), ff{0x1.555556p-5f, -0x1.555556p-30f});
    p = ff_sum(ff_prod(p, r), ff{0x1.555556p-3f, -0x1.555556p-28f});
    p = ff_sum_f(ff_prod(p, r), 0.5f);
    p = ff_sum_f(ff_prod(p, r), 1.0f);
    p = ff_sum_f(ff_prod(p, r), 1.0f);
    // times 2^k (k >= -116: a normal power of two)
    const int ki = (int)k;
#if defined(__CUDA_ARCH__)
    const float sc = __int_as_float((ki + 127) << 23);
#else
    const float sc = std::ldexp(1.0f, ki);
#endif
    return ff{FF_MUL(p.hi, sc), FF_MUL(p.lo, sc)};
}

// phi(x) = (1 + tanh(x/delta))/2 = 1/(1 + exp(-2x/delta)) (Sec. 4.1) and
// 1 - phi, both in float-float: with E = exp(-2|x|/delta) <= 1, the larger of
// the two is 1/(1 + E) and the smaller E/(1 + E), so neither cancels.
struct PhiFF {
    ff phi;    // phi(x)
    ff phic;   // 1 - phi(x)
};

FF_HD PhiFF ff_phi(const ff& x, const ff& inv_delta)
{
    const ff z = ff_prod(x, inv_delta);
    const bool pos = z.hi >= 0.0f;
    const ff y = pos ? ff{-2.0f * z.hi, -2.0f * z.lo} : ff{2.0f * z.hi, 2.0f * z.lo};
    const ff e = ff_exp_nonpos(y);
    const ff big = ff_quot(ff{1.0f, 0.0f}, ff_sum_f(e, 1.0f));
    const ff small = ff_prod(e, big);
    PhiFF r;
    r.phi = pos ? big : small;
    r.phic = pos ? small : big;
    return r;
}

}  // namespace lbm
