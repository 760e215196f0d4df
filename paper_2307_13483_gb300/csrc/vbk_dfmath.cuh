// Double-float evaluation of the level shift F[Gamma/2pi](eps) (Eq. IntF with the widths of
// Sec. II.B) on the FP32 pipes, host and device alike.  A double-float number is the
// unevaluated sum hi + lo of two floats; the operations below are built from error-free
// transformations (Knuth's TwoSum, Dekker's product with a fused multiply-add; the algorithms
// of Dekker 1971 and of Hida, Li and Bailey's double-double library restated for float pairs)
// and keep ~2^-47 relative accuracy per operation.  GB300 executes FP32 about 64 times faster
// than FP64, so the energy tables of the FP32 refinement path, which needs the diagonal of A to
// ~1e-14, are cheaper this way than with the FP64 closed form.
//
// Host code that includes this file must be compiled without contraction of a * b + c (the
// build passes -ffp-contract=off to the host compiler); device code uses the round-to-nearest
// intrinsics, which the compiler never contracts.
#pragma once

#include <cmath>

struct dflt {
    float h, l;
};

#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn((a), (b))
#define DF_SUB(a, b) __fsub_rn((a), (b))
#define DF_MUL(a, b) __fmul_rn((a), (b))
#define DF_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#define DF_DIV(a, b) __fdiv_rn((a), (b))
#define DF_SQRT(a) __fsqrt_rn(a)
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#define DF_FMA(a, b, c) std::fmaf((a), (b), (c))
#define DF_DIV(a, b) ((a) / (b))
#define DF_SQRT(a) std::sqrt(a)
#endif

__host__ __device__ inline dflt dfv(float h, float l = 0.f) {
    dflt r;
    r.h = h;
    r.l = l;
    return r;
}
// s + e = a + b exactly (Knuth)
__host__ __device__ inline dflt df_sum(float a, float b) {
    const float s = DF_ADD(a, b);
    const float bb = DF_SUB(s, a);
    const float e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
    return dfv(s, e);
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__host__ __device__ inline dflt df_fast(float a, float b) {
    const float s = DF_ADD(a, b);
    return dfv(s, DF_SUB(b, DF_SUB(s, a)));
}
// p + e = a * b exactly
__host__ __device__ inline dflt df_prod(float a, float b) {
    const float p = DF_MUL(a, b);
    return dfv(p, DF_FMA(a, b, -p));
}
__host__ __device__ inline dflt dd_add(dflt x, dflt y) {
    dflt s = df_sum(x.h, y.h);
    const dflt t = df_sum(x.l, y.l);
    s = df_fast(s.h, DF_ADD(s.l, t.h));
    return df_fast(s.h, DF_ADD(s.l, t.l));
}
__host__ __device__ inline dflt dd_neg(dflt x) { return dfv(-x.h, -x.l); }
__host__ __device__ inline dflt dd_sub(dflt x, dflt y) { return dd_add(x, dd_neg(y)); }
__host__ __device__ inline dflt dd_add_f(dflt x, float f) {
    const dflt s = df_sum(x.h, f);
    return df_fast(s.h, DF_ADD(s.l, x.l));
}
__host__ __device__ inline dflt dd_mul(dflt x, dflt y) {
    const dflt p = df_prod(x.h, y.h);
    return df_fast(p.h, DF_ADD(p.l, DF_FMA(x.h, y.l, DF_MUL(x.l, y.h))));
}
__host__ __device__ inline dflt dd_mul_f(dflt x, float f) {
    const dflt p = df_prod(x.h, f);
    return df_fast(p.h, DF_FMA(x.l, f, p.l));
}
// x / y: two correction steps
__host__ __device__ inline dflt dd_div(dflt x, dflt y) {
    const float q1 = DF_DIV(x.h, y.h);
    dflt r = dd_sub(x, dd_mul_f(y, q1));
    const float q2 = DF_DIV(r.h, y.h);
    r = dd_sub(r, dd_mul_f(y, q2));
    const float q3 = DF_DIV(r.h, y.h);
    const dflt q = df_fast(q1, q2);
    return dd_add_f(q, q3);
}
// sqrt(x), x >= 0: one Newton correction of the FP32 root
__host__ __device__ inline dflt dd_sqrt(dflt x) {
    if (!(x.h > 0.f)) return dfv(0.f);
    const float s = DF_SQRT(x.h);
    const dflt p = df_prod(s, s);
    const float r = DF_ADD(DF_SUB(DF_SUB(x.h, p.h), p.l), x.l);  // x - s^2 (x.h - p.h is exact)
    return df_fast(s, DF_DIV(r, DF_ADD(s, s)));
}
// the double-float pair nearest a double (host set-up of tables and constants)
inline dflt dd_from(double v) {
    const float h = (float)v;
    return dfv(h, (float)(v - (double)h));
}
__host__ __device__ inline double dd_to_double(dflt x) { return (double)x.h + (double)x.l; }

// Polynomial sum_p c[p] t^p of degree DEG by Horner's rule, coefficients as float pairs.
template <int DEG>
__host__ __device__ inline dflt dd_horner(const float2* c, dflt t) {
    dflt r = dfv(c[DEG].x, c[DEG].y);
    for (int p = DEG - 1; p >= 0; --p) r = dd_add(dd_mul(r, t), dfv(c[p].x, c[p].y));
    return r;
}

// Constants of the closed form as float pairs, rounded at compile time.
#define VBK_DF_CONST(name, v)                                        \
    constexpr float name##_h = (float)(v);                           \
    constexpr float name##_l = (float)((v) - (double)(float)(v));
VBK_DF_CONST(kDfPi, 3.14159265358979323846)
VBK_DF_CONST(kDfSqrtPi, 1.7724538509055160273)
VBK_DF_CONST(kDfInvSqrtPi, 0.56418958354775628695)
VBK_DF_CONST(kDfHalfOverPi, 0.15915494309189533577)
#undef VBK_DF_CONST

// Dawson's integral D(x) (the pieces of vbk_dawson): x < 1/2 Taylor series in x^2 (14 terms),
// 1/2 <= x < 16 the piecewise degree-12 interpolants (table dws, pairs), beyond the asymptotic
// series (9 terms).  x >= 0.
__host__ __device__ inline dflt dd_dawson(dflt x, const float2* dws, int nint, const float2* taylor) {
    if (x.h < 0.5f) {
        const dflt u = dd_mul(x, x);
        return dd_mul(dd_horner<13>(taylor, u), x);
    }
    if (x.h < 0.5f * nint) {
        const int k = (int)(2.f * x.h);
        const dflt t = dd_add_f(dd_mul_f(x, 4.f), -(float)(2 * k + 1));  // 4 x exact; 2k + 1 exact
        return dd_horner<12>(dws + k * 13, t);
    }
    const dflt u = dd_div(dfv(0.5f), dd_mul(x, x));  // 1 / (2 x^2)
    dflt sum = dfv(1.f), term = dfv(1.f);
    for (int k = 1; k <= 8; ++k) {
        term = dd_mul(dd_mul_f(term, (float)(2 * k - 1)), u);
        sum = dd_add(sum, term);
    }
    return dd_mul(dd_div(dfv(0.5f), x), sum);
}
// erfcx(y) = exp(y^2) erfc(y), y >= 0 (the pieces of vbk_erfcx)
__host__ __device__ inline dflt dd_erfcx(dflt y, const float2* erx, int nint) {
    if (y.h < 0.5f * nint) {
        const int k = y.h > 0.f ? (int)(2.f * y.h) : 0;
        const dflt t = dd_add_f(dd_mul_f(y, 4.f), -(float)(2 * k + 1));
        return dd_horner<12>(erx + k * 13, t);
    }
    const dflt u = dd_div(dfv(0.5f), dd_mul(y, y));
    dflt sum = dfv(1.f), term = dfv(1.f);
    for (int k = 1; k <= 8; ++k) {
        term = dd_neg(dd_mul(dd_mul_f(term, (float)(2 * k - 1)), u));
        sum = dd_add(sum, term);
    }
    return dd_mul(dd_div(dfv(kDfInvSqrtPi_h, kDfInvSqrtPi_l), y), sum);
}
// exp(x) for x <= 0: x = n ln2 + r with ln2 split in three parts (the first two exact in float
// with 12 significant bits, so n ln2_1 and n ln2_2 are exact), exp(r) by its Taylor series to
// r^12 / 12! (|r| <= ln2 / 2), then the binary exponent; zero below -87.
__host__ __device__ inline dflt dd_exp_neg(dflt x) {
    if (x.h < -87.f) return dfv(0.f);
    const float n = rintf(DF_MUL(x.h, 1.44269504088896341f));
    dflt r = dd_add_f(x, -n * 0.693115234375f);
    r = dd_add_f(r, -n * 3.1948089599609375e-05f);
    r = dd_add_f(r, -n * -1.9046542121259336e-09f);
    // Taylor coefficients 1 / k!, k = 12 .. 0, by Horner
    dflt s = dfv(2.08767569878680990e-09f);  // 1 / 12! (the last terms need no low part)
    const double inv_fact[12] = {1.0, 1.0, 0.5, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320,
                                 1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800};
    for (int k = 11; k >= 0; --k) {
        const float ch = (float)inv_fact[k];
        const float cl = (float)(inv_fact[k] - (double)ch);
        s = dd_add(dd_mul(s, r), dfv(ch, cl));
    }
    const int e = (int)n;
    return dfv(ldexpf(s.h, e), ldexpf(s.l, e));
}

// Tables of a model in double-float form: the interpolant coefficients of Dawson's integral
// and erfcx (nint intervals x 13), the Taylor coefficients of Dawson's integral (14), and the
// constants of each channel: a, b, sqrt(b), 1 / sqrt(b), 1 / b.
struct DfLevelShift {
    const float2* dawson;
    const float2* erfcx;
    const float2* taylor;
    int nint;
};

// F[f](eps) of one channel (Eq. IntF; the closed form of vbk_level_shift_core) in double-float:
//   (a/2pi) [P_l(eps) - i pi eps^(l+1/2) exp(-b eps) theta(eps)],
//   P_l = -Gamma(l+1/2) b^-(l+1/2) + eps P_(l-1),
//   eps P_(-1) = 2 sqrt(pi eps) D(sqrt(b eps)) (eps > 0), pi sqrt(-eps) erfcx(sqrt(-b eps)) (eps < 0).
// c = {a, b, sqrt b, 1/sqrt b, 1/b} as pairs.  Returns (Re F, Im F).
__host__ __device__ inline void dd_level_shift(dflt eps, const float2* c, int l, const DfLevelShift& T, dflt* re,
                                               dflt* im) {
    const dflt a = dfv(c[0].x, c[0].y), b = dfv(c[1].x, c[1].y), sb = dfv(c[2].x, c[2].y),
               isb = dfv(c[3].x, c[3].y), ib = dfv(c[4].x, c[4].y);
    const dflt ae = eps.h < 0.f ? dd_neg(eps) : eps;
    const dflt sq = dd_sqrt(ae);
    dflt t = dfv(0.f);
    if (eps.h > 0.f)
        t = dd_mul(dd_mul_f(dd_mul(dfv(kDfSqrtPi_h, kDfSqrtPi_l), sq), 2.f), dd_dawson(dd_mul(sb, sq), T.dawson, T.nint, T.taylor));
    else if (eps.h < 0.f)
        t = dd_mul(dd_mul(dfv(kDfPi_h, kDfPi_l), sq), dd_erfcx(dd_mul(sb, sq), T.erfcx, T.nint));
    dflt g = dfv(kDfSqrtPi_h, kDfSqrtPi_l);  // Gamma(k + 1/2), k = 0
    dflt ibp = isb;                          // b^-(k+1/2)
    dflt p = dd_sub(t, dd_mul(g, ibp));
    for (int k = 1; k <= l; ++k) {
        g = dd_mul_f(g, (float)k - 0.5f);  // (k - 1/2) exact in float
        ibp = dd_mul(ibp, ib);
        p = dd_sub(dd_mul(eps, p), dd_mul(g, ibp));
    }
    *re = dd_mul(dd_mul(a, dfv(kDfHalfOverPi_h, kDfHalfOverPi_l)), p);
    *im = dfv(0.f);
    if (eps.h > 0.f) {
        dflt el = sq;  // eps^(l+1/2)
        for (int k = 0; k < l; ++k) el = dd_mul(el, eps);
        const dflt ex = dd_exp_neg(dd_neg(dd_mul(b, eps)));
        *im = dd_mul_f(dd_mul(dd_mul(a, el), ex), -0.5f);
    }
}
