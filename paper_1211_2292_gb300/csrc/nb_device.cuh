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
// The seed is taken at x' = x 2^-2k in [1, 4) (2k the even part of x's
// exponent) and scaled back by 2^-k, both exact edits of the exponent field
// on the integer pipe, so every positive normal float64 x gets a normal seed
// (a float32 seed of x itself would overflow or flush to zero outside
// 1.2e-38 .. 3.4e38, e.g. for r^2 = 1e-40 at eps = 0).  Valid for positive
// normal x; x = 0 gives a large finite value (callers mask the self pair).
__device__ __forceinline__ double rsqrt_f64(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int k2 = ((int)(((unsigned)hi >> 20) & 0x7ffu) - 1023) & ~1;  // even part of the exponent
    const double xs = __hiloint2double(hi - k2 * (1 << 20), lo);   // x 2^-k2, in [1, 4)
    const double ys = (double)rsqrt_mufu((float)xs);
    const double y = __hiloint2double(__double2hiint(ys) - (k2 / 2) * (1 << 20), __double2loint(ys));
    double h = x * y;
    double e = fma(-h, y, 1.0);
    double p = fma(e, 0.375, 0.5);
    return fma(y * e, p, y);
}

// Exclusive scan of in[0..total) into out[0..total) (in == out allowed) by
// one block of 1024 threads, in index order, starting from carry0; returns
// carry0 plus the sum (every thread).
// Tiles of 8192 entries pass through shared memory (coalesced loads and
// stores), 8 consecutive entries per thread, a two-level warp scan of the
// thread sums and a carry from tile to tile.  tile: 8192 + 256 entries,
// wsum: 32 entries of shared memory.
constexpr int BSCAN_PER = 8, BSCAN_TILE = 1024 * BSCAN_PER;
__device__ __forceinline__ int bscan_pad(int i) { return i + (i >> 5); }  // no bank conflicts

template <typename T>
__device__ T block_scan_exclusive(const T *in, T *out, int total, T *tile, T *wsum, T carry0 = 0)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T carry = carry0;
    for (int base = 0; base < total; base += BSCAN_TILE) {
        for (int q = threadIdx.x; q < BSCAN_TILE; q += 1024)
            tile[bscan_pad(q)] = base + q < total ? in[base + q] : T(0);
        __syncthreads();
        T v[BSCAN_PER], sum = 0;
#pragma unroll
        for (int q = 0; q < BSCAN_PER; ++q) {
            v[q] = tile[bscan_pad(threadIdx.x * BSCAN_PER + q)];
            sum += v[q];
        }
        T incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            T w = wsum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const T t = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += t;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        T run = carry + (warp ? wsum[warp - 1] : T(0)) + incl - sum;
#pragma unroll
        for (int q = 0; q < BSCAN_PER; ++q) {
            tile[bscan_pad(threadIdx.x * BSCAN_PER + q)] = run;
            run += v[q];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < BSCAN_TILE; q += 1024)
            if (base + q < total) out[base + q] = tile[bscan_pad(q)];
        carry += wsum[31];
        __syncthreads();  // tile and wsum are rewritten by the next tile
    }
    return carry;
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

// Tile-local coordinate of a hi/lo packed component.
__device__ __forceinline__ float rel(float hi, float lo, float c) { return (hi - c) + lo; }

// Centre of the bounding box of the CTA's valid i-bodies (every thread gets
// the same value).  red: shared scratch of 6 x (T/32) floats.
template <int T>
__device__ __forceinline__ float3 block_center(float (&mn)[3], float (&mx)[3], float (*red)[T / 32])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], off));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], off));
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            red[c][warp] = mn[c];
            red[3 + c][warp] = mx[c];
        }
    }
    __syncthreads();
    float a[3], b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a[c] = red[c][0];
        b[c] = red[3 + c][0];
#pragma unroll
        for (int w = 1; w < T / 32; ++w) {
            a[c] = fminf(a[c], red[c][w]);
            b[c] = fmaxf(b[c], red[3 + c][w]);
        }
    }
    __syncthreads();  // red may be reused by the caller afterwards
    float3 o;
    o.x = a[0] <= b[0] ? 0.5f * (a[0] + b[0]) : 0.f;
    o.y = a[1] <= b[1] ? 0.5f * (a[1] + b[1]) : 0.f;
    o.z = a[2] <= b[2] ? 0.5f * (a[2] + b[2]) : 0.f;
    return o;
}

}  // namespace nb
