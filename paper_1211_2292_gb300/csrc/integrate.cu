// O(n) kernels around the pair kernels: packing the caller's float64
// (n,3)+(n) arrays into the internal (x,y,z,m) layout, the leapfrog's
// kick+drift (the reading of the paper's "Move_bodies", Sec. IV-B), the
// adjoint's drift/cotangent packing, and the final energy reduction.
//
// All are memory-bound one-thread-per-body kernels (grid-stride loops).
#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

constexpr int TPB = 256;

inline int grid_for(int n)
{
    int g = (n + TPB - 1) / TPB;
    return g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g);
}

__device__ __forceinline__ void put(float4 *P, int i, double x, double y, double z, double m)
{
    P[i] = make_float4((float)x, (float)y, (float)z, (float)m);
}
__device__ __forceinline__ void put(double4 *P, int i, double x, double y, double z, double m)
{
    P[i] = make_double4(x, y, z, m);
}
// float32 hi/lo pair: x = hi + lo with hi = fl(x), lo = fl(x - hi); the lo
// slot's w carries log2 m for the log-domain pair factor.
__device__ __forceinline__ void put_hilo(float4 *P, float4 *Plo, int i, double x, double y,
                                         double z, double m)
{
    const float hx = (float)x, hy = (float)y, hz = (float)z;
    P[i] = make_float4(hx, hy, hz, (float)m);
    Plo[i] = make_float4((float)(x - (double)hx), (float)(y - (double)hy), (float)(z - (double)hz),
                         (float)log2(m));
}

template <typename V>
__global__ void pack_kernel(int n, const double *__restrict__ pos, const double *__restrict__ mass,
                            const int *__restrict__ perm, V *__restrict__ P)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = perm ? perm[k] : k;
        const double *x = pos + 3 * (size_t)i;
        put(P, k, x[0], x[1], x[2], mass[i]);
    }
}

// Opening half-kick and drift of one leapfrog step, then repack:
//   v += half_dt * a;  x += dt * v.
// (x, v) before the update are copied to rec_pos/rec_vel when given.
template <typename V>
__global__ void kdp_kernel(int n, double *__restrict__ pos, double *__restrict__ vel,
                           const double *__restrict__ acc, const double *__restrict__ mass,
                           double half_dt, double dt, V *__restrict__ P, float4 *__restrict__ Plo,
                           double *__restrict__ rec_pos, double *__restrict__ rec_vel)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double *x = pos + 3 * (size_t)i;
        double *v = vel + 3 * (size_t)i;
        const double *a = acc + 3 * (size_t)i;
        double xx = x[0], xy = x[1], xz = x[2];
        double vx = v[0], vy = v[1], vz = v[2];
        if (rec_pos) {
            double *r = rec_pos + 3 * (size_t)i;
            r[0] = xx; r[1] = xy; r[2] = xz;
        }
        if (rec_vel) {
            double *r = rec_vel + 3 * (size_t)i;
            r[0] = vx; r[1] = vy; r[2] = vz;
        }
        vx += half_dt * a[0];
        vy += half_dt * a[1];
        vz += half_dt * a[2];
        xx += dt * vx;
        xy += dt * vy;
        xz += dt * vz;
        v[0] = vx; v[1] = vy; v[2] = vz;
        x[0] = xx; x[1] = xy; x[2] = xz;
        if (Plo)
            put_hilo((float4 *)P, Plo, i, xx, xy, xz, mass[i]);
        else if (P)
            put(P, i, xx, xy, xz, mass[i]);
    }
}

// Adjoint packing: optional drift adjoint lam_v += drift * lam_x, then
// cotangent mu = coef * lam (lam = lam_v when given, else `lam`), packed as
// (x,y,z,m),(mu_x,mu_y,mu_z,0) in float64, or as hi/lo float32 positions plus
// mu in three arrays `stride` float4 apart.
template <typename V>
__global__ void pack_vjp_kernel(int n, const double *__restrict__ pos,
                                const double *__restrict__ mass, const double *__restrict__ lam,
                                double *__restrict__ lam_v, const double *__restrict__ lam_x,
                                double drift, double coef, V *__restrict__ PV, size_t stride)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double *x = pos + 3 * (size_t)i;
        double l0, l1, l2;
        if (lam_v) {
            double *lv = lam_v + 3 * (size_t)i;
            l0 = lv[0]; l1 = lv[1]; l2 = lv[2];
            if (lam_x) {
                const double *lx = lam_x + 3 * (size_t)i;
                l0 += drift * lx[0];
                l1 += drift * lx[1];
                l2 += drift * lx[2];
                lv[0] = l0; lv[1] = l1; lv[2] = l2;
            }
        } else {
            const double *l = lam + 3 * (size_t)i;
            l0 = l[0]; l1 = l[1]; l2 = l[2];
        }
        if (sizeof(V) == sizeof(double4)) {
            put(PV, 2 * i, x[0], x[1], x[2], mass[i]);
            put(PV, 2 * i + 1, coef * l0, coef * l1, coef * l2, 0.0);
        } else {
            float4 *F = reinterpret_cast<float4 *>(PV);
            put_hilo(F, F + stride, i, x[0], x[1], x[2], mass[i]);
            put(F + 2 * stride, i, coef * l0, coef * l1, coef * l2, 0.0);
        }
    }
}

// out[0..8] = {E_kin, E_pot, E_tot, P_x, P_y, P_z, F_x, F_y, F_z} from the
// per-CTA partials, added in a fixed order by one CTA.
__global__ void energy_final_kernel(const double *__restrict__ red, int nparts, double G,
                                    double *__restrict__ out)
{
    __shared__ double sh[8][TPB];
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nparts; b += TPB) {
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] += red[8 * (size_t)b + c];
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int w = TPB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ek = sh[0][0];
        const double ep = -0.5 * G * sh[1][0];
        out[0] = ek;
        out[1] = ep;
        out[2] = ek + ep;
        out[3] = sh[2][0];
        out[4] = sh[3][0];
        out[5] = sh[4][0];
        out[6] = G * sh[5][0];
        out[7] = G * sh[6][0];
        out[8] = G * sh[7][0];
    }
}

}  // namespace

cudaError_t launch_pack_f32(cudaStream_t s, int n, const double *pos, const double *mass, float4 *P)
{
    pack_kernel<float4><<<grid_for(n), TPB, 0, s>>>(n, pos, mass, nullptr, P);
    return cudaGetLastError();
}

cudaError_t launch_pack_f64(cudaStream_t s, int n, const double *pos, const double *mass,
                            double4 *P, const int *perm)
{
    pack_kernel<double4><<<grid_for(n), TPB, 0, s>>>(n, pos, mass, perm, P);
    return cudaGetLastError();
}

cudaError_t launch_kdp(cudaStream_t s, bool f64, int n, double *pos, double *vel,
                       const double *acc, const double *mass, double half_dt, double dt, void *P,
                       float4 *Plo, double *rec_pos, double *rec_vel)
{
    if (f64)
        kdp_kernel<double4><<<grid_for(n), TPB, 0, s>>>(n, pos, vel, acc, mass, half_dt, dt,
                                                         (double4 *)P, nullptr, rec_pos, rec_vel);
    else
        kdp_kernel<float4><<<grid_for(n), TPB, 0, s>>>(n, pos, vel, acc, mass, half_dt, dt,
                                                        (float4 *)P, P ? Plo : nullptr, rec_pos,
                                                        rec_vel);
    return cudaGetLastError();
}

cudaError_t launch_pack_vjp(cudaStream_t s, bool f64, int n, const double *pos, const double *mass,
                            const double *lam, double *lam_v, const double *lam_x, double drift,
                            double coef, void *PV, size_t stride)
{
    if (f64)
        pack_vjp_kernel<double4><<<grid_for(n), TPB, 0, s>>>(n, pos, mass, lam, lam_v, lam_x,
                                                              drift, coef, (double4 *)PV, stride);
    else
        pack_vjp_kernel<float4><<<grid_for(n), TPB, 0, s>>>(n, pos, mass, lam, lam_v, lam_x,
                                                             drift, coef, (float4 *)PV, stride);
    return cudaGetLastError();
}

cudaError_t launch_energy_final(cudaStream_t s, const double *red, int nparts, double G,
                                double *out)
{
    energy_final_kernel<<<1, TPB, 0, s>>>(red, nparts, G, out);
    return cudaGetLastError();
}

}  // namespace nb
