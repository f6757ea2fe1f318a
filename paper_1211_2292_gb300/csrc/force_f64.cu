// float64 force and energy kernels (paper Sec. IV-A/IV-B force calculation
// as the exact all-pairs sum, every operation in float64).
//
// Same schedule as the float32 kernels: an i-tile of T*I bodies per CTA in
// registers, j-bodies streamed through a double-buffered shared tile of J
// double4 (x,y,z,m), the grid split over j with the last arriving CTA adding
// the float64 partials in split order.  The reciprocal square root is a
// float32 MUFU seed refined by one second-order Householder step (see
// nb_device.cuh), since float64 has no MUFU path.
//
// The energy kernel also accumulates the softened potential
// phi_i = sum_{j != i} m_j / s_ij (self pair skipped by index) and reduces,
// per CTA, E_pot = -G/2 sum m_i phi_i, F = G sum m_i a_i and (split 0 only)
// E_kin and P; a single-CTA kernel adds the per-CTA values in order.
#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

constexpr int UNROLL_F64 = 4;

template <int T, int J>
__device__ __forceinline__ void stage_load64(double4 (&buf)[J / T], const double4 *__restrict__ P,
                                             int jbase, int jend)
{
#pragma unroll
    for (int l = 0; l < J / T; ++l) {
        const int j = jbase + l * T + threadIdx.x;
        buf[l] = j < jend ? P[j] : make_double4(0.0, 0.0, 0.0, 0.0);
    }
}

template <int T, int J>
__device__ __forceinline__ void stage_store64(double4 *tile, const double4 (&buf)[J / T])
{
#pragma unroll
    for (int l = 0; l < J / T; ++l) tile[l * T + threadIdx.x] = buf[l];
}

template <bool ZEPS>
__device__ __forceinline__ double pair_rinv(double r2)
{
    double ri = rsqrt_f64(r2);
    if (ZEPS) ri = r2 > 0.0 ? ri : 0.0;
    return ri;
}

template <int T, int I, int J, bool ZEPS, bool ENERGY>
__device__ __forceinline__ void sweep64(const double4 *__restrict__ P, int n, int t0, int t1,
                                        double eps2, const double (&xi)[I], const double (&yi)[I],
                                        const double (&zi)[I], const int (&ii)[I], double (&ax)[I],
                                        double (&ay)[I], double (&az)[I], double (&ph)[I],
                                        double4 (*tile)[J])
{
    double4 buf[J / T];
    if (t0 < t1) {
        stage_load64<T, J>(buf, P, t0 * J, n);
        stage_store64<T, J>(tile[0], buf);
    }
    __syncthreads();
    for (int t = t0; t < t1; ++t) {
        const int b = (t - t0) & 1;
        if (t + 1 < t1) stage_load64<T, J>(buf, P, (t + 1) * J, n);
        const double4 *s = tile[b];
#pragma unroll UNROLL_F64
        for (int jj = 0; jj < J; ++jj) {
            const double4 q = s[jj];
#pragma unroll
            for (int k = 0; k < I; ++k) {
                const double dx = q.x - xi[k], dy = q.y - yi[k], dz = q.z - zi[k];
                double r2 = fma(dx, dx, eps2);
                r2 = fma(dy, dy, r2);
                r2 = fma(dz, dz, r2);
                const double ri = pair_rinv<ZEPS>(r2);
                const double mri = q.w * ri;
                const double sc = mri * (ri * ri);
                ax[k] = fma(dx, sc, ax[k]);
                ay[k] = fma(dy, sc, ay[k]);
                az[k] = fma(dz, sc, az[k]);
                if (ENERGY) ph[k] += (t * J + jj == ii[k]) ? 0.0 : mri;
            }
        }
        if (t + 1 < t1) stage_store64<T, J>(tile[b ^ 1], buf);
        __syncthreads();
    }
}

template <int T, int I, int J, bool ZEPS>
__global__ void __launch_bounds__(T) force_f64_kernel(const ForceParams p)
{
    constexpr int TILE_I = T * I;
    __shared__ __align__(16) double4 tile[2][J];
    __shared__ int s_last;
    const double4 *P = static_cast<const double4 *>(p.P);
    const int n = p.n;
    const int n_itiles = (n + TILE_I - 1) / TILE_I;
    const int it = blockIdx.x % n_itiles;
    const int js = blockIdx.x / n_itiles;
    const int i0 = it * TILE_I;
    int t0, t1;
    split_range((n + J - 1) / J, p.nsplit, js, t0, t1);

    double xi[I], yi[I], zi[I], ax[I], ay[I], az[I], ph[I];
    int ii[I];
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        const double4 b = i < n ? P[i] : make_double4(0.0, 0.0, 0.0, 0.0);
        xi[k] = b.x;
        yi[k] = b.y;
        zi[k] = b.z;
        ii[k] = i;
        ax[k] = ay[k] = az[k] = ph[k] = 0.0;
    }
    sweep64<T, I, J, ZEPS, false>(P, n, t0, t1, p.eps2, xi, yi, zi, ii, ax, ay, az, ph, tile);

    if (p.nsplit == 1) {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = i0 + threadIdx.x + k * T;
            if (i < n) {
                double *a = p.acc + 3 * (size_t)i;
                const double gx = p.G * ax[k], gy = p.G * ay[k], gz = p.G * az[k];
                a[0] = gx;
                a[1] = gy;
                a[2] = gz;
                if (p.vel) {
                    double *v = p.vel + 3 * (size_t)i;
                    v[0] += p.half_dt * gx;
                    v[1] += p.half_dt * gy;
                    v[2] += p.half_dt * gz;
                }
                if (!finite3(gx, gy, gz)) atomicOr(p.err, ERR_NONFINITE);
            }
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        if (i < n) {
            double *q = p.partial + ((size_t)js * n + i) * 3;
            q[0] = ax[k];
            q[1] = ay[k];
            q[2] = az[k];
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
            double x = 0.0, y = 0.0, z = 0.0;
            for (int q = 0; q < p.nsplit; ++q) {
                const double *r = p.partial + ((size_t)q * n + i) * 3;
                x += __ldcg(r);
                y += __ldcg(r + 1);
                z += __ldcg(r + 2);
            }
            double *a = p.acc + 3 * (size_t)i;
            const double gx = p.G * x, gy = p.G * y, gz = p.G * z;
            a[0] = gx;
            a[1] = gy;
            a[2] = gz;
            if (p.vel) {
                double *v = p.vel + 3 * (size_t)i;
                v[0] += p.half_dt * gx;
                v[1] += p.half_dt * gy;
                v[2] += p.half_dt * gz;
            }
            if (!finite3(gx, gy, gz)) atomicOr(p.err, ERR_NONFINITE);
        }
    }
    if (threadIdx.x == 0) p.counters[it] = 0u;
}

// Fixed-order CTA sum of NV doubles per thread (tree over shared memory).
template <int T, int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[T])
{
#pragma unroll
    for (int c = 0; c < NV; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int w = T / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int c = 0; c < NV; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = sh[c][0];
}

// Energy/momentum partials.  red[block][0..7] =
// {E_kin, sum m_i phi_i, P_x, P_y, P_z, sum m_i a_x, sum m_i a_y, sum m_i a_z}
// (G and the -1/2 are applied by the final kernel).
template <int T, int I, int J, bool ZEPS>
__global__ void __launch_bounds__(T) energy_f64_kernel(const EnergyParams p)
{
    constexpr int TILE_I = T * I;
    __shared__ __align__(16) double4 tile[2][J];
    __shared__ double sh[8][T];
    const double4 *P = p.P;
    const int n = p.n;
    const int n_itiles = (n + TILE_I - 1) / TILE_I;
    const int it = blockIdx.x % n_itiles;
    const int js = blockIdx.x / n_itiles;
    const int i0 = it * TILE_I;
    int t0, t1;
    split_range((n + J - 1) / J, p.nsplit, js, t0, t1);

    double xi[I], yi[I], zi[I], mi[I], ax[I], ay[I], az[I], ph[I];
    int ii[I];
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        const double4 b = i < n ? P[i] : make_double4(0.0, 0.0, 0.0, 0.0);
        xi[k] = b.x;
        yi[k] = b.y;
        zi[k] = b.z;
        mi[k] = b.w;  // zero for padding bodies, so they add nothing
        ii[k] = i;
        ax[k] = ay[k] = az[k] = ph[k] = 0.0;
    }
    sweep64<T, I, J, ZEPS, true>(P, n, t0, t1, p.eps2, xi, yi, zi, ii, ax, ay, az, ph, tile);

    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        v[1] += mi[k] * ph[k];
        v[5] += mi[k] * ax[k];
        v[6] += mi[k] * ay[k];
        v[7] += mi[k] * az[k];
        if (js == 0 && i < n) {
            const double *vi = p.vel + 3 * (size_t)i;
            const double vx = vi[0], vy = vi[1], vz = vi[2];
            v[0] += 0.5 * mi[k] * (vx * vx + vy * vy + vz * vz);
            v[2] += mi[k] * vx;
            v[3] += mi[k] * vy;
            v[4] += mi[k] * vz;
        }
    }
    block_sum<T, 8>(v, sh);
    if (threadIdx.x == 0) {
        double *r = p.red + 8 * (size_t)blockIdx.x;
#pragma unroll
        for (int c = 0; c < 8; ++c) r[c] = v[c];
    }
}

#define NB_F64_ENTRY(T, I, J)                                            \
    {{T, I, J, (const void *)force_f64_kernel<T, I, J, false>},          \
     {T, I, J, (const void *)force_f64_kernel<T, I, J, true>}}

typedef KernelEntry Pair[2];
const Pair kF64[] = {
    NB_F64_ENTRY(128, 1, 128),
    NB_F64_ENTRY(128, 2, 128),
    NB_F64_ENTRY(256, 2, 256),
    NB_F64_ENTRY(64, 2, 128),
};
const Pair kEnergy = {{128, 1, 128, (const void *)energy_f64_kernel<128, 1, 128, false>},
                      {128, 1, 128, (const void *)energy_f64_kernel<128, 1, 128, true>}};

}  // namespace

int f64_force_variants() { return (int)(sizeof(kF64) / sizeof(kF64[0])); }
const KernelEntry &f64_force_kernel(int v, bool zeps) { return kF64[v][zeps]; }
const KernelEntry &f64_energy_kernel(bool zeps) { return kEnergy[zeps]; }

}  // namespace nb
