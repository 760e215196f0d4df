// Device helpers shared by the solver's translation units (sm_103a): mixed-radix decoding of a
// vibrational index, packed FP32x2 fused multiply-add, and double-float arithmetic.
#pragma once

#include "vbk_internal.cuh"

// mode indices n_m of the vibrational index nu (last mode fastest)
template <int M> __device__ __forceinline__ void decode(const DevModel& md, int nu, int (&n)[MAXM]) {
    unsigned rem = (unsigned)nu;
#pragma unroll
    for (int m = M - 1; m >= 0; --m) {
        const unsigned q = fdiv(rem, md.fd_nb[m]);
        n[m] = (int)(rem - q * (unsigned)md.nb[m]);
        rem = q;
    }
#pragma unroll
    for (int m = M; m < MAXM; ++m) n[m] = 0;
}

// a * b + c on both halves of a float pair with one packed FP32x2 instruction
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
          "l"(*reinterpret_cast<unsigned long long*>(&c)));
    return *reinterpret_cast<float2*>(&r);
}

// a + b, a - b, a * b on both halves of a float pair (packed FP32x2, round to nearest)
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&r);
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&r);
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&r);
}

// n[m] for a runtime mode index m without dynamic register indexing
template <int M> __device__ __forceinline__ int nsel(const int (&n)[MAXM], int m) {
    int r = n[0];
#pragma unroll
    for (int k = 1; k < M; ++k) r = (m == k) ? n[k] : r;
    return r;
}

// ------------------------------------------------------------------ double-float arithmetic
// Unevaluated sums hi + lo of two floats (Dekker 1971 products with a fused multiply-add;
// Knuth's TwoSum): the residual b - A x of the FP32 refinement path is formed with ~48-bit
// significands on the FP32 pipes, which GB300 runs ~64x faster than its FP64 pipe.
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// (sh, sl) += (ah + al) (xh + xl), the al xl term (~2^-48 relative) dropped
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
    float sum, t;
    df_two_sum(sh, p, sum, t);
    sh = sum;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}
// df_fma on both halves of float pairs at once (packed FP32x2): (sh, sl) += (a + al) (x + xl)
// lane by lane, with na = -a supplied by the caller (the packed instructions take no negated
// operand).  The same operations in the same order as df_fma, so each lane's result is
// bit-identical to it: p = fl(a x) is formed as -fl((-a) x), the product error a x - p by one
// fused multiply-add, and TwoSum(sh, p) is written with -p.
__device__ __forceinline__ void df_fma2(float2& sh, float2& sl, float2 a, float2 al, float2 na, float2 x, float2 xl) {
    const float2 pn = fmul2(na, x);                  // -p
    float2 e = ffma2(a, x, pn);                      // a x - p, exact
    e = ffma2(a, xl, ffma2(al, x, e));
    const float2 s = fsub2(sh, pn);                  // fl(sh + p)
    const float2 z = fsub2(s, sh);
    const float2 t = fsub2(fsub2(sh, fsub2(s, z)), fadd2(pn, z));  // (sh - (s - z)) + (p - z)
    sh = s;
    sl = fadd2(sl, fadd2(t, e));
}
// renormalised pair (s, l) with s = fl(h + l)
__device__ __forceinline__ float2 df_norm(float h, float l) {
    const float sum = __fadd_rn(h, l);
    return make_float2(sum, __fsub_rn(l, __fsub_rn(sum, h)));
}

// float -> double, exact, by moving the bit fields (integer pipes; GB300's FP64 pipe is the
// scarce one); zeros, subnormals, infinities and NaNs take the conversion instruction
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f), ex = (u >> 23) & 0xffu;
    if (ex == 0u || ex == 0xffu) return (double)f;
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    ((unsigned long long)(ex + (1023u - 127u)) << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}
