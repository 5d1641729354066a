// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2, about 48 significant bits.  It carries the
// per-site part of the FP32-arithmetic step kernels (moment folding, Landau
// frame, equilibrium coefficients) at FP64-class accuracy on the FP32 pipes:
// GB300 executes FP64 at 1/64 of its FP32 rate, and a double-float operation
// costs 3 to 20 FP32 instructions.
//
// The error-free transformations are Knuth's TwoSum, Dekker's FastTwoSum and
// the FMA form of TwoProduct (a * b = p + e exactly with e = fma(a, b, -p)).
// Every operation uses the _rn intrinsics, which the compiler never contracts
// into an FMA, so the transformations stay exact.  Division, square root and
// reciprocal square root take one FP32 approximation and one correction step
// with a double-float residual (Karp and Markstein).
//
// df2 holds two sites as packed pairs (float2 hi, float2 lo) and runs the same
// operations on Blackwell's f32x2 instructions: one instruction for two sites.
#pragma once

#include <cuda_runtime.h>

namespace rlbmk {

struct df64 {
    float hi, lo;
};

__device__ __forceinline__ df64 dd(float a) { return {a, 0.f}; }
__device__ __forceinline__ df64 dd(float h, float l) { return {h, l}; }

__device__ __forceinline__ df64 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return {s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ df64 fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df64 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// Sum with one TwoSum of the high parts and the low parts added in FP32: its
// error is below about 2 u^2 (|x| + |y|) (u = 2^-24), the bound of FP64
// arithmetic on operands that carry rounding errors of their own.
__device__ __forceinline__ df64 operator+(df64 x, df64 y)
{
    const df64 s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df64 operator-(df64 x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }
__device__ __forceinline__ df64 operator+(df64 x, float b)
{
    const df64 s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ df64 operator-(df64 x, float b) { return x + (-b); }

__device__ __forceinline__ df64 operator*(df64 x, df64 y)
{
    const df64 p = two_prod(x.hi, y.hi);
    const float e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ df64 operator*(df64 x, float b)
{
    const df64 p = two_prod(x.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}

// x / y: q1 = x / y in FP32, then q2 from the residual x - q1 y
__device__ __forceinline__ df64 operator/(df64 x, df64 y)
{
    const float r = __frcp_rn(y.hi);
    const float q1 = __fmul_rn(x.hi, r);
    const df64 res = x - y * q1;
    const float q2 = __fmul_rn(res.hi, r);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ df64 dd_sqrt(df64 x)
{
    if (!(x.hi > 0.f)) return {0.f, 0.f};
    const float s = __fsqrt_rn(x.hi);
    const df64 res = x - two_prod(s, s);
    return fast_two_sum(s, __fdividef(res.hi, __fadd_rn(s, s)));
}

// 1 / sqrt(x): y = rsqrt(x) in FP32, then y + y (1 - x y^2) / 2
__device__ __forceinline__ df64 dd_rsqrt(df64 x)
{
    const float y = rsqrtf(x.hi);
    const df64 e = dd(1.f) - x * two_prod(y, y);
    return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), e.hi));
}

__device__ __forceinline__ float to_float(df64 x) { return __fadd_rn(x.hi, x.lo); }

// ---- two sites at once: packed pairs on the f32x2 instructions --------------

__device__ __forceinline__ unsigned long long f2u(float2 v)
{
    unsigned long long u;
    memcpy(&u, &v, 8);
    return u;
}
__device__ __forceinline__ float2 u2f(unsigned long long u)
{
    float2 v;
    memcpy(&v, &u, 8);
    return v;
}
__device__ __forceinline__ float2 padd(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
    return u2f(d);
}
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }

struct df2 {
    float2 hi, lo;
};

__device__ __forceinline__ df2 p_two_sum(float2 a, float2 b)
{
    const float2 s = padd(a, b);
    const float2 v = psub(s, a);
    return {s, padd(psub(a, psub(s, v)), psub(b, v))};
}
__device__ __forceinline__ df2 p_fast_two_sum(float2 a, float2 b)
{
    const float2 s = padd(a, b);
    return {s, psub(b, psub(s, a))};
}
__device__ __forceinline__ df2 operator+(df2 x, df2 y)
{
    const df2 s = p_two_sum(x.hi, y.hi);
    return p_fast_two_sum(s.hi, padd(s.lo, padd(x.lo, y.lo)));
}
__device__ __forceinline__ df2 operator-(df2 x, df2 y) { return x + df2{pneg(y.hi), pneg(y.lo)}; }
// x * (b_hi + b_lo) for a scalar double-float b (the same for both sites)
__device__ __forceinline__ df2 operator*(df2 x, df64 b)
{
    const float2 bh = make_float2(b.hi, b.hi), bl = make_float2(b.lo, b.lo);
    const float2 p = pmul(x.hi, bh);
    const float2 e = pfma(x.hi, bl, pfma(x.lo, bh, pfma(x.hi, bh, pneg(p))));
    return p_fast_two_sum(p, e);
}
// x * b for a small exact float b (a power of two or a small integer)
__device__ __forceinline__ df2 scale(df2 x, float b)
{
    const float2 bb = make_float2(b, b);
    const float2 p = pmul(x.hi, bb);
    return p_fast_two_sum(p, pfma(x.lo, bb, pfma(x.hi, bb, pneg(p))));
}
__device__ __forceinline__ float2 to_float2(df2 x) { return padd(x.hi, x.lo); }

} // namespace rlbmk
