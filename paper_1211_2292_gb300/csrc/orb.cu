// Orthogonal recursive bisection over processors that each hold part of the
// bodies (paper Sec. IV-B: space divided into as many non-overlapping
// subspaces as processors, each with about the same number of bodies).
//
// A part shared by p processors is cut across the longest side of its
// bounding box; the lower part takes floor(p/2) processors and the
// k = floor(count floor(p/2) / p) bodies first in (coordinate, body id)
// order.  The bodies of a part are spread over all processors, so the cut is
// found without moving them: a radix select on the 96-bit key
// (order-preserving image of the coordinate, 32-bit body id), one 8-bit
// digit per round, where every processor histograms its own bodies and the
// caller sums the histograms over processors (a collective) before picking
// the digit that holds the k-th key.  Every part of a level is cut in the
// same rounds; a body's group is the first processor of its part, and after
// the last level it is the body's processor.  Keys are unique, so the cut is
// exact and does not depend on how the bodies are distributed.
//
// These kernels compute one processor's share (box, histogram, cut) and the
// packing of bodies by destination; the host code around them does the
// collectives.
#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

constexpr int OBT = 256;

// Order-preserving 64-bit image of a float64 (for non-NaN values; -0 is
// first made +0 so that it ties with +0 as the comparison does).
__device__ __forceinline__ unsigned long long ord64(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v + 0.0);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

inline int grid_for(int n)
{
    int g = (n + OBT - 1) / OBT;
    return g < 1 ? 1 : (g > 2048 ? 2048 : g);
}

__global__ void __launch_bounds__(OBT) orb_box_kernel(int n, const double *__restrict__ pos,
                                                      const int *__restrict__ group, int ngroups,
                                                      unsigned long long *__restrict__ box)
{
    for (int i = blockIdx.x * OBT + threadIdx.x; i < n; i += gridDim.x * OBT) {
        const int g = group[i];
        if (g < 0 || g >= ngroups) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const unsigned long long k = ord64(pos[3 * (size_t)i + c]);
            atomicMin(box + 6 * (size_t)g + c, k);
            atomicMax(box + 6 * (size_t)g + 3 + c, k);
        }
    }
}

// Whether key (hi, lo) starts with the first `bits` bits of (phi, plo).
__device__ __forceinline__ bool has_prefix(unsigned long long hi, unsigned lo,
                                           unsigned long long phi, unsigned plo, int bits)
{
    if (bits == 0) return true;
    if (bits <= 64) return (hi >> (64 - bits)) == (phi >> (64 - bits));
    if (hi != phi) return false;
    const int lb = bits - 64;  // 8, 16 or 24 of the 32 id bits
    return (lo >> (32 - lb)) == (plo >> (32 - lb));
}

__device__ __forceinline__ unsigned digit_of(unsigned long long hi, unsigned lo, int round)
{
    return round < 8 ? (unsigned)(hi >> (56 - 8 * round)) & 255u
                     : (lo >> (24 - 8 * (round - 8))) & 255u;
}

// Histograms in shared memory (one row of 256 per active part), added into
// the global rows at the end.
__global__ void __launch_bounds__(OBT) orb_hist_kernel(int n, const double *__restrict__ pos,
                                                       const long long *__restrict__ id,
                                                       const int *__restrict__ group, int nactive,
                                                       const OrbTables t, int round,
                                                       unsigned long long *__restrict__ hist)
{
    extern __shared__ unsigned sh[];  // [nactive][256]
    for (int q = threadIdx.x; q < nactive * 256; q += OBT) sh[q] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * OBT + threadIdx.x; i < n; i += gridDim.x * OBT) {
        const int g = group[i];
        const int row = (g >= 0 && g < ORB_MAX_P) ? t.slot[g] : -1;
        if (row < 0) continue;
        const unsigned long long hi = ord64(pos[3 * (size_t)i + t.axis[row]]);
        const unsigned lo = (unsigned)id[i];
        if (!has_prefix(hi, lo, t.key_hi[row], t.key_lo[row], 8 * round)) continue;
        atomicAdd(&sh[row * 256 + digit_of(hi, lo, round)], 1u);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nactive * 256; q += OBT)
        if (sh[q]) atomicAdd(hist + q, (unsigned long long)sh[q]);
}

__global__ void __launch_bounds__(OBT) orb_cut_kernel(int n, const double *__restrict__ pos,
                                                      const long long *__restrict__ id,
                                                      int *__restrict__ group, const OrbTables t)
{
    for (int i = blockIdx.x * OBT + threadIdx.x; i < n; i += gridDim.x * OBT) {
        const int g = group[i];
        const int row = (g >= 0 && g < ORB_MAX_P) ? t.slot[g] : -1;
        if (row < 0) continue;
        const unsigned long long hi = ord64(pos[3 * (size_t)i + t.axis[row]]);
        const unsigned lo = (unsigned)id[i];
        const bool below = hi < t.key_hi[row] || (hi == t.key_hi[row] && lo < t.key_lo[row]);
        if (!below) group[i] = t.upper[row];
    }
}

__global__ void __launch_bounds__(OBT) gather_bodies_kernel(
    int n, const int *__restrict__ perm, const double *__restrict__ pos,
    const double *__restrict__ vel, const double *__restrict__ mass,
    const long long *__restrict__ id, double *__restrict__ pos_out, double *__restrict__ vel_out,
    double *__restrict__ mass_out, long long *__restrict__ id_out)
{
    for (int k = blockIdx.x * OBT + threadIdx.x; k < n; k += gridDim.x * OBT) {
        const int j = perm[k];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (pos_out) pos_out[3 * (size_t)k + c] = pos[3 * (size_t)j + c];
            if (vel_out) vel_out[3 * (size_t)k + c] = vel[3 * (size_t)j + c];
        }
        if (mass_out) mass_out[k] = mass[j];
        if (id_out) id_out[k] = id[j];
    }
}

__global__ void __launch_bounds__(OBT) rank_count_kernel(int n, const int *__restrict__ rank,
                                                         int P, unsigned long long *__restrict__ counts)
{
    __shared__ unsigned sh[ORB_MAX_P];
    for (int q = threadIdx.x; q < P; q += OBT) sh[q] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * OBT + threadIdx.x; i < n; i += gridDim.x * OBT) {
        const int r = rank[i];
        if (r >= 0 && r < P) atomicAdd(&sh[r], 1u);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < P; q += OBT)
        if (sh[q]) atomicAdd(counts + q, (unsigned long long)sh[q]);
}

// Float32 min/max of the packed positions; box holds the order-preserving
// images (as for ord64) of the float32 values, widened to 64 bits.
__device__ __forceinline__ unsigned ord32(float v)
{
    const unsigned b = __float_as_uint(v + 0.0f);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}

__global__ void __launch_bounds__(OBT) hi_box_kernel(int n, const float4 *__restrict__ P,
                                                     unsigned *__restrict__ box)
{
    for (int i = blockIdx.x * OBT + threadIdx.x; i < n; i += gridDim.x * OBT) {
        const float4 h = P[i];
        const float v[3] = {h.x, h.y, h.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicMin(box + c, ord32(v[c]));
            atomicMax(box + 3 + c, ord32(v[c]));
        }
    }
}

__global__ void hi_box_decode_kernel(const unsigned *__restrict__ box, float *__restrict__ out)
{
    const int c = threadIdx.x;
    if (c < 6) {
        const unsigned k = box[c];
        const unsigned b = (k >> 31) ? (k & 0x7fffffffu) : ~k;
        out[c] = __uint_as_float(b);
    }
}

}  // namespace

cudaError_t launch_orb_box(cudaStream_t s, int n, const double *pos, const int *group, int ngroups,
                           unsigned long long *box)
{
    // min rows start at all ones, max rows at zero
    for (int g = 0; g < ngroups; ++g) {
        cudaError_t e = cudaMemsetAsync(box + 6 * (size_t)g, 0xff, 3 * sizeof(unsigned long long), s);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(box + 6 * (size_t)g + 3, 0, 3 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    if (n > 0) orb_box_kernel<<<grid_for(n), OBT, 0, s>>>(n, pos, group, ngroups, box);
    return cudaGetLastError();
}

cudaError_t launch_orb_hist(cudaStream_t s, int n, const double *pos, const long long *id,
                            const int *group, int nactive, const OrbTables &t, int round,
                            unsigned long long *hist)
{
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nactive * 256 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (n > 0 && nactive > 0)
        orb_hist_kernel<<<grid_for(n), OBT, (size_t)nactive * 256 * sizeof(unsigned), s>>>(
            n, pos, id, group, nactive, t, round, hist);
    return cudaGetLastError();
}

cudaError_t launch_orb_cut(cudaStream_t s, int n, const double *pos, const long long *id,
                           int *group, const OrbTables &t)
{
    if (n > 0) orb_cut_kernel<<<grid_for(n), OBT, 0, s>>>(n, pos, id, group, t);
    return cudaGetLastError();
}

cudaError_t launch_gather_bodies(cudaStream_t s, int n, const int *perm, const double *pos,
                                 const double *vel, const double *mass, const long long *id,
                                 double *pos_out, double *vel_out, double *mass_out,
                                 long long *id_out)
{
    if (n > 0)
        gather_bodies_kernel<<<grid_for(n), OBT, 0, s>>>(n, perm, pos, vel, mass, id, pos_out,
                                                         vel_out, mass_out, id_out);
    return cudaGetLastError();
}

cudaError_t launch_rank_counts(cudaStream_t s, int n, const int *rank, int P,
                               unsigned long long *counts)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)P * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (n > 0) rank_count_kernel<<<grid_for(n), OBT, 0, s>>>(n, rank, P, counts);
    return cudaGetLastError();
}

cudaError_t launch_hi_box(cudaStream_t s, int n, const float4 *P, float *box)
{
    // box holds 6 floats of output after 6 unsigned of working space
    unsigned *work = reinterpret_cast<unsigned *>(box + 6);
    cudaError_t e = cudaMemsetAsync(work, 0xff, 3 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(work + 3, 0, 3 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (n > 0) hi_box_kernel<<<grid_for(n), OBT, 0, s>>>(n, P, work);
    hi_box_decode_kernel<<<1, 32, 0, s>>>(work, box);
    return cudaGetLastError();
}

}  // namespace nb
