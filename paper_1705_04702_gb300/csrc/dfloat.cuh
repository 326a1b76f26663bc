// Double-float arithmetic for the exact dust-emission solve: a value is an
// unevaluated sum hi + lo of two IEEE binary32 numbers (|lo| <= ulp(hi)/2),
// about 48 significant bits, computed on the FP32 pipe.  GB300 retires an
// FP64 warp instruction far more slowly than an FP32 one, so the per-term
// work of the solve (the Planck factor 1/expm1(x) of every wavelength and
// population) runs in this arithmetic and only the per-population steps stay
// in FP64.
//
// Methods (all published, none taken from a math library):
//  * error-free transformations: Knuth's two-sum, Dekker's fast two-sum (for
//    |a| >= |b|), and the exact product a*b = p + e with e = fma(a, b, -p)
//    (Dekker 1971; Ogita, Rump and Oishi 2005);
//  * double-float sums and products built on them in the usual way
//    (Dekker 1971; Hida, Li and Bailey 2001);
//  * expm1(x), 0 <= x <= 88: Cody-Waite reduction x = k ln 2 + r, |r| <= ln 2 / 2,
//    with ln 2 split into three binary32 pieces; expm1(r) = r P(r) from the
//    Taylor series P(r) = sum_n r^n / (n+1)! through n = 12 (the first omitted
//    term is below 2e-17 of the sum), terms n >= 7 in binary32 (they add less
//    than 1.6e-8 of the sum); then e^x - 1 = 2^k (1 + expm1(r)) - 1;
//  * 1/a: the binary32 reciprocal refined by one Newton step,
//    y' = y + y (1 - a y), with the residual formed exactly.
//
// The operations are spelled with round-to-nearest intrinsics on the device
// (nothing may be contracted into an FMA); on the host the same code is plain
// binary32 arithmetic and gives identical results when compiled without
// floating-point contraction (-ffp-contract=off).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define DF_FN __host__ __device__ __forceinline__
#else
#define DF_FN static inline
#endif

#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn((a), (b))
#define DF_SUB(a, b) __fsub_rn((a), (b))
#define DF_MUL(a, b) __fmul_rn((a), (b))
#define DF_RCP(a) __frcp_rn(a)
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#define DF_RCP(a) (1.0f / (a))
#endif

namespace dfl {

struct df2 {
    float hi, lo;
};

DF_FN df2 make(float hi, float lo)
{
    df2 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

// s + e = a + b exactly
DF_FN void two_sum(float a, float b, float& s, float& e)
{
    s = DF_ADD(a, b);
    const float bb = DF_SUB(s, a);
    e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
}

// s + e = a + b exactly, for |a| >= |b| (or a == 0)
DF_FN void fast_two_sum(float a, float b, float& s, float& e)
{
    s = DF_ADD(a, b);
    e = DF_SUB(b, DF_SUB(s, a));
}

// p + e = a * b exactly (barring underflow)
DF_FN void two_prod(float a, float b, float& p, float& e)
{
    p = DF_MUL(a, b);
    e = fmaf(a, b, -p);
}

DF_FN df2 renorm(float hi, float lo)
{
    df2 r;
    fast_two_sum(hi, lo, r.hi, r.lo);
    return r;
}

// a + b, for operands of the same sign (no cancellation between the high parts)
DF_FN df2 add(df2 a, df2 b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = DF_ADD(e, DF_ADD(a.lo, b.lo));
    return renorm(s, e);
}

DF_FN df2 mul(df2 a, df2 b)
{
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return renorm(p, e);
}

// 2^k a for an integer 0 <= k <= 127 (exact)
DF_FN df2 scale2(df2 a, int k)
{
    union {
        unsigned u;
        float v;
    } c;
    c.u = (unsigned)(127 + k) << 23;
    return make(DF_MUL(a.hi, c.v), DF_MUL(a.lo, c.v));
}

// 1/a for a > 0 (binary32 normal range)
DF_FN df2 recip(df2 a)
{
    const float y = DF_RCP(a.hi);
    float p, e;
    two_prod(a.hi, y, p, e);            // a.hi y = p + e, p within an ulp of 1
    float r = DF_SUB(1.0f, p);          // exact
    r = DF_SUB(r, e);
    r = fmaf(-a.lo, y, r);              // r = 1 - a y to ~2^-48
    return renorm(y, DF_MUL(y, r));
}

// p r + (ch + cl) for |p r| < ch / 2 (one double-float Horner step)
DF_FN df2 horner_step(df2 p, df2 r, float ch, float cl)
{
    p = mul(p, r);
    float s, e;
    two_sum(p.hi, ch, s, e);
    e = DF_ADD(e, DF_ADD(p.lo, cl));
    return renorm(s, e);
}

// ln 2 in three binary32 pieces, and 1/ln 2 rounded to binary32
#define DF_LN2_0 0x1.62e430p-1f
#define DF_LN2_1 -0x1.05c610p-29f
#define DF_LN2_2 -0x1.950d88p-54f
#define DF_INV_LN2 0x1.715476p+0f

// e^x - 1 for 0 <= x.hi <= 88
DF_FN df2 expm1(df2 x)
{
    const float kf = rintf(DF_MUL(x.hi, DF_INV_LN2));
    df2 r = x;
    if (kf != 0.0f) {
        // r = x - k ln 2: k LN2_0 and k LN2_1 exactly as (p, e) pairs, the
        // leading difference exact (x.hi lies within a factor 2 of k ln 2)
        float p0, e0, p1, e1;
        two_prod(kf, DF_LN2_0, p0, e0);
        two_prod(kf, DF_LN2_1, p1, e1);
        const float s = DF_SUB(x.hi, p0);
        float a_hi, a_lo, b_hi, b_lo, r_hi, r_lo;
        two_sum(x.lo, -e0, a_hi, a_lo);
        two_sum(a_hi, -p1, b_hi, b_lo);
        const float rest = DF_SUB(DF_SUB(DF_ADD(a_lo, b_lo), e1), DF_MUL(kf, DF_LN2_2));
        two_sum(s, b_hi, r_hi, r_lo);
        r = renorm(r_hi, DF_ADD(r_lo, rest));
    }
    // P(r) = sum_n r^n / (n+1)!: the binary32 tail n = 12..7, then n = 6..0 in
    // double-float (coefficients 1/(n+1)! as hexadecimal literals of their
    // correctly rounded binary32 pieces)
    float t = 0x1.612462p-33f;            // 1/13!
    t = fmaf(t, r.hi, 0x1.1eed8ep-29f);   // 1/12!
    t = fmaf(t, r.hi, 0x1.ae6456p-26f);   // 1/11!
    t = fmaf(t, r.hi, 0x1.27e4fcp-22f);   // 1/10!
    t = fmaf(t, r.hi, 0x1.71de3ap-19f);   // 1/9!
    t = fmaf(t, r.hi, 0x1.a01a02p-16f);   // 1/8!
    df2 p = make(t, 0.0f);
    p = horner_step(p, r, 0x1.a01a02p-13f, -0x1.7f97fap-39f);  // 1/7!
    p = horner_step(p, r, 0x1.6c16c2p-10f, -0x1.27d27ep-35f);  // 1/6!
    p = horner_step(p, r, 0x1.111112p-7f, -0x1.dddddep-32f);   // 1/5!
    p = horner_step(p, r, 0x1.555556p-5f, -0x1.555556p-30f);   // 1/4!
    p = horner_step(p, r, 0x1.555556p-3f, -0x1.555556p-28f);   // 1/3!
    p = horner_step(p, r, 0x1p-1f, 0.0f);                       // 1/2!
    p = horner_step(p, r, 0x1p+0f, 0.0f);                       // 1/1!
    const df2 em1 = mul(r, p);  // expm1(r)
    if (kf == 0.0f) return em1;
    // 2^k (1 + expm1(r)) - 1
    float s, e;
    two_sum(1.0f, em1.hi, s, e);
    df2 f = scale2(renorm(s, DF_ADD(e, em1.lo)), (int)kf);
    two_sum(f.hi, -1.0f, s, e);
    return renorm(s, DF_ADD(e, f.lo));
}

}  // namespace dfl
