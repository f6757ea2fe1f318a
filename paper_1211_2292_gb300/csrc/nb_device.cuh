// Device-side building blocks shared by the force, energy and adjoint kernels.
//
// Everything here is arithmetic on values already in registers or shared
// memory; the kernels decide layout and scheduling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nb {

// ---------------------------------------------------------------- float32x2
// Blackwell executes one float32x2 instruction (two IEEE round-to-nearest
// float32 operations on a 64-bit register pair) per issue slot, so pairing
// two i-bodies halves the issue cost of the pair arithmetic; the FP32 pipe
// throughput is unchanged.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Hardware reciprocal square root (MUFU), inputs flushed to zero when
// subnormal.  Relative error below 2^-22.
__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Hardware base-2 logarithm and exponential (MUFU), subnormals flushed.
// lg2: absolute error below 2^-22 on [0.5, 2) (relative elsewhere through the
// exact exponent); ex2: relative error below 2^-22.
__device__ __forceinline__ float lg2_mufu(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_mufu(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// float64 reciprocal square root: a float32 MUFU seed y0 (relative error
// e0 < 2^-22) refined by one second-order Householder step for
// f(y) = 1/y^2 - x.  With e = 1 - x*y0^2 the exact answer is
// y0*(1-e)^(-1/2) = y0*(1 + e/2 + 3e^2/8 + ...); keeping two terms leaves a
// relative error of about (5/16)e^3 ~ 1e-20, below float64 rounding.
// Valid for x within the float32 normal range (1.2e-38 .. 3.4e38).
__device__ __forceinline__ double rsqrt_f64(double x)
{
    double y = (double)rsqrt_mufu((float)x);
    double h = x * y;
    double e = fma(-h, y, 1.0);
    double p = fma(e, 0.375, 0.5);
    return fma(y * e, p, y);
}

// Kahan-compensated accumulation of a partial sum p into (s, c); the value
// represented is s - c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float p)
{
    float y = p - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Range of j-tiles [t0, t1) handled by split `js` of `nsplit`.
__device__ __forceinline__ void split_range(int ntiles, int nsplit, int js, int &t0, int &t1)
{
    t0 = (int)(((long long)ntiles * js) / nsplit);
    t1 = (int)(((long long)ntiles * (js + 1)) / nsplit);
}

__device__ __forceinline__ bool finite3(double a, double b, double c)
{
    return isfinite(a) && isfinite(b) && isfinite(c);
}

// Error-word bits (ctx scratch, read by nb_sync / nb_energy).
enum : int { ERR_NONFINITE = 1 };

}  // namespace nb
