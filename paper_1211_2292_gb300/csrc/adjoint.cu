// Force vector-Jacobian product (no counterpart in the paper; it follows
// from differentiating the softened force).  For cotangent mu = dL/da, with
// d_kj = x_j - x_k, s = sqrt(|d|^2 + eps^2), K(d) = I/s^3 - 3 d d^T/s^5:
//
//   gx_k = G sum_j K(d_kj) (m_k mu_j - m_j mu_k)
//        = G sum_j [ w/s^3 - 3 d (d.w)/s^5 ],      w = m_k mu_j - m_j mu_k
//   gm_k = G sum_j mu_j . (x_k - x_j) / s^3  =  -G sum_j (mu_j . d_kj)/s^3
//
// The self pair contributes zero (d = 0 and w = 0).  Schedule as in the
// force kernels: i-tile in registers, j-tiles (x,y,z,m),(mu,0) through
// double-buffered shared memory, j-split across CTAs with an ordered
// last-CTA combine.  float32 variant: pair terms in float32, each tile's
// partial added into float64 accumulators.  float64 variant: all float64.
#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

template <typename R>
struct V4;
template <>
struct V4<float> {
    typedef float4 type;
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static float rsq(float x) { return rsqrt_mufu(x); }
};
template <>
struct V4<double> {
    typedef double4 type;
    __device__ static double4 zero() { return make_double4(0.0, 0.0, 0.0, 0.0); }
    __device__ static double rsq(double x) { return rsqrt_f64(x); }
};

template <typename R, int T, int I, int J, bool ZEPS>
__global__ void __launch_bounds__(T) vjp_kernel(const VjpParams p)
{
    typedef typename V4<R>::type V;
    constexpr int TILE_I = T * I;
    constexpr int LPT = J / T;
    __shared__ __align__(16) V tile[2][2 * J];
    __shared__ int s_last;

    const V *PV = static_cast<const V *>(p.PV);
    const int n = p.n;
    const int n_itiles = (n + TILE_I - 1) / TILE_I;
    const int it = blockIdx.x % n_itiles;
    const int js = blockIdx.x / n_itiles;
    const int i0 = it * TILE_I;
    int t0, t1;
    split_range((n + J - 1) / J, p.nsplit, js, t0, t1);
    const R e2 = sizeof(R) == 4 ? (R)p.eps2f : (R)p.eps2;

    R xk[I], yk[I], zk[I], mk[I], lx[I], ly[I], lz[I];
    R px[I], py[I], pz[I], pm[I];       // tile partials
    double gx[I], gy[I], gz[I], gm[I];  // float64 totals
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        const V a = i < n ? PV[2 * (size_t)i] : V4<R>::zero();
        const V b = i < n ? PV[2 * (size_t)i + 1] : V4<R>::zero();
        xk[k] = a.x; yk[k] = a.y; zk[k] = a.z; mk[k] = a.w;
        lx[k] = b.x; ly[k] = b.y; lz[k] = b.z;
        gx[k] = gy[k] = gz[k] = gm[k] = 0.0;
    }

    V buf[2 * LPT];
    auto gload = [&](int t) {
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int j = t * J + l * T + threadIdx.x;
            buf[2 * l] = j < n ? PV[2 * (size_t)j] : V4<R>::zero();
            buf[2 * l + 1] = j < n ? PV[2 * (size_t)j + 1] : V4<R>::zero();
        }
    };
    auto sstore = [&](int b) {
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int jj = l * T + threadIdx.x;
            tile[b][2 * jj] = buf[2 * l];
            tile[b][2 * jj + 1] = buf[2 * l + 1];
        }
    };
    if (t0 < t1) {
        gload(t0);
        sstore(0);
    }
    __syncthreads();
    for (int t = t0; t < t1; ++t) {
        const int b = (t - t0) & 1;
        if (t + 1 < t1) gload(t + 1);
#pragma unroll
        for (int k = 0; k < I; ++k) px[k] = py[k] = pz[k] = pm[k] = (R)0;
        const V *s = tile[b];
#pragma unroll 4
        for (int jj = 0; jj < J; ++jj) {
            const V q = s[2 * jj], u = s[2 * jj + 1];
#pragma unroll
            for (int k = 0; k < I; ++k) {
                const R dx = q.x - xk[k], dy = q.y - yk[k], dz = q.z - zk[k];
                R r2 = dx * dx + e2;
                r2 = dy * dy + r2;
                r2 = dz * dz + r2;
                R ri = V4<R>::rsq(r2);
                if (ZEPS) ri = r2 > (R)0 ? ri : (R)0;
                const R ri2 = ri * ri;
                const R ri3 = ri2 * ri;
                const R q5 = ri3 * ri2;
                const R wx = mk[k] * u.x - q.w * lx[k];
                const R wy = mk[k] * u.y - q.w * ly[k];
                const R wz = mk[k] * u.z - q.w * lz[k];
                const R dw = dx * wx + dy * wy + dz * wz;
                const R c = (R)3 * dw * q5;
                px[k] += wx * ri3 - dx * c;
                py[k] += wy * ri3 - dy * c;
                pz[k] += wz * ri3 - dz * c;
                pm[k] -= (u.x * dx + u.y * dy + u.z * dz) * ri3;
            }
        }
#pragma unroll
        for (int k = 0; k < I; ++k) {
            gx[k] += (double)px[k];
            gy[k] += (double)py[k];
            gz[k] += (double)pz[k];
            gm[k] += (double)pm[k];
        }
        if (t + 1 < t1) sstore(b ^ 1);
        __syncthreads();
    }

    auto emit = [&](int i, double x, double y, double z, double m) {
        x *= p.G; y *= p.G; z *= p.G; m *= p.G;
        double *o = p.gx + 3 * (size_t)i;
        if (p.accumulate) {
            o[0] += x; o[1] += y; o[2] += z;
            p.gm[i] += m;
        } else {
            o[0] = x; o[1] = y; o[2] = z;
            p.gm[i] = m;
        }
        if (!(finite3(x, y, z) && isfinite(m))) atomicOr(p.err, ERR_NONFINITE);
    };
    if (p.nsplit == 1) {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = i0 + threadIdx.x + k * T;
            if (i < n) emit(i, gx[k], gy[k], gz[k], gm[k]);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        if (i < n) {
            double *q = p.partial + ((size_t)js * n + i) * 4;
            q[0] = gx[k]; q[1] = gy[k]; q[2] = gz[k]; q[3] = gm[k];
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(p.counters + it, 1u) == (unsigned)(p.nsplit - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        if (i < n) {
            double x = 0.0, y = 0.0, z = 0.0, m = 0.0;
            for (int q = 0; q < p.nsplit; ++q) {
                const double *r = p.partial + ((size_t)q * n + i) * 4;
                x += __ldcg(r); y += __ldcg(r + 1); z += __ldcg(r + 2); m += __ldcg(r + 3);
            }
            emit(i, x, y, z, m);
        }
    }
    if (threadIdx.x == 0) p.counters[it] = 0u;
}

#define NB_VJP_ENTRY(R, T, I, J)                                       \
    {{T, I, J, (const void *)vjp_kernel<R, T, I, J, false>},           \
     {T, I, J, (const void *)vjp_kernel<R, T, I, J, true>}}

typedef KernelEntry Pair[2];
const Pair kVjp32[] = {
    NB_VJP_ENTRY(float, 128, 2, 128),
    NB_VJP_ENTRY(float, 128, 4, 128),
    NB_VJP_ENTRY(float, 256, 2, 256),
};
const Pair kVjp64[] = {
    NB_VJP_ENTRY(double, 128, 1, 128),
    NB_VJP_ENTRY(double, 128, 2, 128),
};

}  // namespace

int f32_vjp_variants() { return (int)(sizeof(kVjp32) / sizeof(kVjp32[0])); }
const KernelEntry &f32_vjp_kernel(int v, bool zeps) { return kVjp32[v][zeps]; }
int f64_vjp_variants() { return (int)(sizeof(kVjp64) / sizeof(kVjp64[0])); }
const KernelEntry &f64_vjp_kernel(int v, bool zeps) { return kVjp64[v][zeps]; }

}  // namespace nb
