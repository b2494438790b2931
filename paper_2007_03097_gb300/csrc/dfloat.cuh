// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits.  The error-free
// transformations (Dekker 1971, Knuth TAOCP vol. 2, Sec. 4.2.2) use the
// round-to-nearest intrinsics so the compiler never fuses or reorders them.
//
// GB300 issues FP64 at 2 lanes per clock per SM against 128 for FP32, so the
// pair sums of the FP64 precision mode are evaluated in this representation
// on the FP32 pipes (relative error about 2^-44 per pair term) and only the
// neighbour decisions near the support radius fall back to exact FP64.
#pragma once

#include <cuda_runtime.h>

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) { return df{hi, lo}; }

// s + e == a + b exactly
__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

// s + e == a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

// p + e == a * b exactly (fused multiply-add gives the rounding error)
__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return df{p, e};
}

__device__ __forceinline__ df df_add(df a, df b)
{
    const df s = two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_add_f(df a, float b)
{
    const df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    const df p = two_prod(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b)
{
    const df p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// Products without the final renormalisation: hi + lo with |lo| up to a few
// ulp(hi) keeps the same ~2^-46 relative accuracy and is a valid operand of
// every operation here (a product cancels nothing), so chains of products
// skip the fast_two_sum of each step.  A result is renormalised (df_norm, or
// any df_add / df_sub) before a comparison or a store.
__device__ __forceinline__ df df_mul_u(df a, df b)
{
    const df p = two_prod(a.hi, b.hi);
    return df{p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo))};
}

__device__ __forceinline__ df df_mul_f_u(df a, float b)
{
    const df p = two_prod(a.hi, b);
    return df{p.hi, __fmaf_rn(a.lo, b, p.lo)};
}

__device__ __forceinline__ df df_sqr_u(df a)
{
    const df p = two_prod(a.hi, a.hi);
    return df{p.hi, __fmaf_rn(__fmul_rn(2.f, a.hi), a.lo, p.lo)};
}

// multiplication by a power of two is exact
__device__ __forceinline__ df df_scale(df a, float pow2) { return df{__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)}; }

__device__ __forceinline__ df df_sqr(df a)
{
    const df p = two_prod(a.hi, a.hi);
    const float e = __fmaf_rn(__fmul_rn(2.f, a.hi), a.lo, p.lo);
    return fast_two_sum(p.hi, e);
}

// one Newton step on the FP32 square root: sqrt(a) = y + (a - y^2) / (2y)
__device__ __forceinline__ df df_sqrt(df a)
{
    if (!(a.hi > 0.f)) return df{0.f, 0.f};
    const float y = __fsqrt_rn(a.hi);
    const df y2 = two_prod(y, y);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, y2.hi), y2.lo), a.lo);
    return fast_two_sum(y, __fdiv_rn(r, __fmul_rn(2.f, y)));
}

// one Newton step on the FP32 reciprocal: 1/a = y + y (1 - a y)
__device__ __forceinline__ df df_rcp(df a)
{
    const float y = __frcp_rn(a.hi);
    const df ay = two_prod(a.hi, y);
    const float r = __fsub_rn(__fsub_rn(__fsub_rn(1.f, ay.hi), ay.lo), __fmul_rn(a.lo, y));
    return fast_two_sum(y, __fmul_rn(y, r));
}

__device__ __forceinline__ bool df_lt0(df a) { return a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f); }

__device__ __forceinline__ bool df_gt(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// Faster variants for the pair loops: hardware approximations (about 22
// correct bits) refined by one correction step, about 2^-44 relative error.
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ df df_sqrt_fast(df a)
{
    if (!(a.hi > 0.f)) return df{0.f, 0.f};
    const float t = rsqrt_approx(a.hi);
    const float y = __fmul_rn(a.hi, t);
    const df y2 = two_prod(y, y);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, y2.hi), y2.lo), a.lo);
    return fast_two_sum(y, __fmul_rn(r, __fmul_rn(0.5f, t)));
}

__device__ __forceinline__ df df_rcp_fast(df a)
{
    const float y = rcp_approx(a.hi);
    const float e = __fmaf_rn(-a.lo, y, __fmaf_rn(-a.hi, y, 1.f));     // 1 - a y
    return fast_two_sum(y, __fmul_rn(y, e));
}

// dx^2 + dy^2 + dz^2: exact squares of the high parts, cross terms in FP32
__device__ __forceinline__ df df_norm2(df x, df y, df z)
{
    const df px = two_prod(x.hi, x.hi), py = two_prod(y.hi, y.hi), pz = two_prod(z.hi, z.hi);
    const df s1 = two_sum(px.hi, py.hi);
    const df s2 = two_sum(s1.hi, pz.hi);
    float lo = __fadd_rn(__fadd_rn(px.lo, py.lo), pz.lo);
    lo = __fmaf_rn(__fmul_rn(2.f, x.hi), x.lo, lo);
    lo = __fmaf_rn(__fmul_rn(2.f, y.hi), y.lo, lo);
    lo = __fmaf_rn(__fmul_rn(2.f, z.hi), z.lo, lo);
    lo = __fadd_rn(lo, __fadd_rn(s1.lo, s2.lo));
    return fast_two_sum(s2.hi, lo);
}

// accumulator update acc += x without renormalising acc (lo collects the
// rounding errors of hi; renormalise with fast_two_sum when done)
__device__ __forceinline__ void df_acc(df &acc, df x)
{
    const df s = two_sum(acc.hi, x.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, x.lo));
}

__device__ __forceinline__ df df_norm(df a) { return fast_two_sum(a.hi, a.lo); }

// conversions (FP64 pipe; keep them out of inner loops)
__device__ __forceinline__ df df_from_double(double d)
{
    const float hi = __double2float_rn(d);
    return df{hi, __double2float_rn(d - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// the same split on the host (kernel arguments)
inline df df_host(double d)
{
    const float hi = (float)d;
    return df{hi, (float)(d - (double)hi)};
}

// x_a - x_b from two-float positions with a minimum-image shift: the exact
// difference of the high parts plus the difference of the low parts
__device__ __forceinline__ df df_sep_fast(float ah, float al, float bh, float bl, int wrap, df L)
{
    df d = two_sum(ah, -bh);
    d = fast_two_sum(d.hi, __fadd_rn(d.lo, __fsub_rn(al, bl)));
    if (wrap > 0) d = df_add(d, L);
    else if (wrap < 0) d = df_sub(d, L);
    return d;
}

// ------------------------------------------------------------------ pair helpers
// Separation x_a - x_b from two-float positions as a double-float, with the
// minimum image decided by the caller (wrap = -1, 0, +1 adds wrap * L).
__device__ __forceinline__ df df_sep(float ah, float al, float bh, float bl, int wrap, df L)
{
    df d = two_sum(ah, -bh);
    d = df_add_f(d, __fsub_rn(al, bl));
    if (wrap > 0) d = df_add(d, L);
    else if (wrap < 0) d = df_sub(d, L);
    return d;
}

// Smoothing kernels in double-float (the forms and shapes of
// sph_internal.cuh, q = r/h): w(q) and g(q) = D w(q) + q w'(q) (shapes 0-2:
// D = 3; shapes 3-5: D = 1), or w'(q) alone.
__device__ __forceinline__ void df_kern_w_g3(int k, df q, df &w, df &g3)
{
    const df one = df{1.f, 0.f};
    if (k >= 3) {
        const df s = df_add_f(df_scale(q, -0.5f), 1.f);
        const df q2 = df_sqr_u(q);
        if (k == 3) {                                          // M4, D = 1
            if (q.hi < 1.f) {
                // w = 1 - 1.5 q^2 + 0.75 q^3 ; g = 1 - 4.5 q^2 + 3 q^3
                const df q3 = df_mul_u(q2, q);
                w = df_add(df_add(one, df_mul_f_u(q2, -1.5f)), df_mul_f_u(q3, 0.75f));
                g3 = df_add(df_add(one, df_mul_f_u(q2, -4.5f)), df_mul_f_u(q3, 3.f));
            } else {
                // t = 2 - q ; w = t^3 / 4 ; g = t^2 (2 - 4q) / 4
                const df t = df_add_f(df_neg(q), 2.f);
                const df t2 = df_sqr_u(t);
                w = df_scale(df_mul_u(t2, t), 0.25f);
                g3 = df_scale(df_mul_u(t2, df_add_f(df_scale(q, -4.f), 2.f)), 0.25f);
            }
        } else if (k == 4) {                                   // Wendland C2, D = 1
            // w = s^3 (1 + 1.5 q) ; g = s^2 (s (1 + 1.5 q) - 3 q^2)
            const df s2 = df_sqr_u(s);
            const df p = df_add_f(df_mul_f_u(q, 1.5f), 1.f);
            w = df_mul_u(df_mul_u(s2, s), p);
            g3 = df_mul_u(s2, df_sub(df_mul_u(s, p), df_mul_f_u(q2, 3.f)));
        } else {                                               // Wendland C4, D = 1
            // P = 1 + 2.5 q + 2 q^2 ; w = s^5 P ; g = s^4 (s P - 3.5 q^2 (1 + 2q))
            const df s2 = df_sqr_u(s);
            const df s4 = df_sqr_u(s2);
            const df P = df_add(df_add_f(df_mul_f_u(q, 2.5f), 1.f), df_scale(q2, 2.f));
            w = df_mul_u(df_mul_u(s4, s), P);
            g3 = df_mul_u(s4, df_sub(df_mul_u(s, P), df_mul_f_u(df_mul_u(q2, df_add_f(df_scale(q, 2.f), 1.f)), 3.5f)));
        }
        return;
    }
    if (k == 0) {                                              // M4
        const df q2 = df_sqr_u(q);
        if (q.hi < 1.f) {
            // w = 1 - 1.5 q^2 + 0.75 q^3 ; g3 = 3 - 7.5 q^2 + 4.5 q^3
            const df q3 = df_mul_u(q2, q);
            w = df_add(df_add(one, df_mul_f_u(q2, -1.5f)), df_mul_f_u(q3, 0.75f));
            g3 = df_add(df_add(df{3.f, 0.f}, df_mul_f_u(q2, -7.5f)), df_mul_f_u(q3, 4.5f));
        } else {
            // t = 2 - q ; w = t^3 / 4 ; g3 = 0.75 t^2 (2 - 2q)
            const df t = df_add_f(df_neg(q), 2.f);
            const df t2 = df_sqr_u(t);
            w = df_scale(df_mul_u(t2, t), 0.25f);
            g3 = df_mul_f_u(df_mul_u(t2, df_add_f(df_scale(q, -2.f), 2.f)), 0.75f);
        }
    } else if (k == 1) {                                       // Wendland C2
        // s = 1 - q/2 ; w = s^4 (1 + 2q) ; g3 = s^3 (3 s (1 + 2q) - 5 q^2)
        const df s = df_add_f(df_scale(q, -0.5f), 1.f);
        const df s2 = df_sqr_u(s);
        const df s3 = df_mul_u(s2, s);
        const df p = df_add_f(df_scale(q, 2.f), 1.f);
        w = df_mul_u(df_sqr_u(s2), p);
        g3 = df_mul_u(s3, df_sub(df_mul_f_u(df_mul_u(s, p), 3.f), df_mul_f_u(df_sqr_u(q), 5.f)));
    } else {                                                   // Wendland C4
        // P = 1 + 3q + 35/12 q^2 ; w = s^6 P ;
        // g3 = s^5 (3 s P - 14/3 q^2 (1 + 2.5 q))
        const df c35_12 = df{2.91666674613952637f, -7.94728621e-08f};
        const df c14_3 = df{4.66666650772094727f, 1.58945724e-07f};
        const df s = df_add_f(df_scale(q, -0.5f), 1.f);
        const df s2 = df_sqr_u(s);
        const df s5 = df_mul_u(df_sqr_u(s2), s);
        const df q2 = df_sqr_u(q);
        const df P = df_add(df_add_f(df_mul_f_u(q, 3.f), 1.f), df_mul_u(q2, c35_12));
        w = df_mul_u(df_mul_u(s5, s), P);
        const df t = df_mul_u(df_mul_u(q2, c14_3), df_add_f(df_mul_f_u(q, 2.5f), 1.f));
        g3 = df_mul_u(s5, df_sub(df_mul_f_u(df_mul_u(s, P), 3.f), t));
    }
}

__device__ __forceinline__ df df_kern_dw(int k, df q)
{
    if (k >= 4) {
        const df s = df_add_f(df_scale(q, -0.5f), 1.f);
        const df s2 = df_sqr_u(s);
        if (k == 4) return df_mul_f_u(df_mul_u(q, s2), -3.f);                       // -3 q s^2
        return df_mul_f_u(df_mul_u(df_mul_u(q, df_add_f(df_scale(q, 2.f), 1.f)), df_sqr_u(s2)), -3.5f);  // -3.5 q (1 + 2q) s^4
    }
    if (k == 0 || k == 3) {
        if (q.hi < 1.f) return df_mul_u(q, df_add_f(df_mul_f_u(q, 2.25f), -3.f));    // q (-3 + 2.25 q)
        const df t = df_add_f(df_neg(q), 2.f);
        return df_mul_f_u(df_sqr_u(t), -0.75f);                                      // -0.75 (2 - q)^2
    }
    const df s = df_add_f(df_scale(q, -0.5f), 1.f);
    const df s2 = df_sqr_u(s);
    if (k == 1) return df_mul_f_u(df_mul_u(q, df_mul_u(s2, s)), -5.f);                 // -5 q s^3
    const df c14_3 = df{4.66666650772094727f, 1.58945724e-07f};
    const df s5 = df_mul_u(df_sqr_u(s2), s);                                         // -14/3 q (1 + 2.5q) s^5
    return df_neg(df_mul_u(df_mul_u(df_mul_u(q, c14_3), df_add_f(df_mul_f_u(q, 2.5f), 1.f)), s5));
}
