// Spatial ordering of bodies for the float32 force kernels.
//
// The float32 pair differences d = x_j - x_i are formed in coordinates
// relative to an origin at the centre of the i-tile (see force_f32.cu).  This
// only helps close pairs when an i-tile is spatially compact, so for large N
// the bodies are processed in Morton (Z-curve) order:
//   1. bounding box of all positions (per-block partials, re-reduced by every
//      block of the next kernel: no atomics, deterministic);
//   2. 24-bit Morton key per body (8 bits per axis over the cube that holds
//      the box);
//   3. stable LSD radix sort of (key, body index), three 8-bit passes: per
//      warp-chunk digit histograms, one exclusive scan in (digit, chunk)
//      order, then a stable scatter that ranks equal digits within a warp
//      with __match_any_sync, chunk keys taken strictly in order;
//   4. packing in sorted order as float32 hi/lo pairs:
//      P_hi = (fl(x), fl(y), fl(z), fl(m)),
//      P_lo = (fl(x - fl(x)), ..., fl(log2 m)) (log2 m for the log-domain pairs).
// Every step is deterministic, so the order and the forces are reproducible.
#include <cuda_runtime.h>
#include <float.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

constexpr int OTPB = 256;
constexpr int MAX_BOX_PARTS = 1023;            // box partials; the folded box follows them
constexpr int BOX_FINAL = 6 * MAX_BOX_PARTS;  // {min x,y,z, max x,y,z} in the box scratch

__device__ __forceinline__ unsigned spread8(unsigned v)
{
    v &= 0xffu;
    v = (v | (v << 8)) & 0x00f00fu;
    v = (v | (v << 4)) & 0x0c30c3u;
    v = (v | (v << 2)) & 0x249249u;
    return v;
}

// Per-block min/max of the positions: parts[b] = {minx,miny,minz,maxx,maxy,maxz}.
__global__ void __launch_bounds__(OTPB) bbox_kernel(int n, const double *__restrict__ pos,
                                                     double *__restrict__ parts)
{
    __shared__ double sh[6][OTPB];
    double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int i = blockIdx.x * OTPB + threadIdx.x; i < n; i += gridDim.x * OTPB) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double v = pos[3 * (size_t)i + c];
            mn[c] = fmin(mn[c], v);
            mx[c] = fmax(mx[c], v);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        sh[c][threadIdx.x] = mn[c];
        sh[3 + c][threadIdx.x] = mx[c];
    }
    __syncthreads();
    for (int w = OTPB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sh[c][threadIdx.x] = fmin(sh[c][threadIdx.x], sh[c][threadIdx.x + w]);
                sh[3 + c][threadIdx.x] = fmax(sh[3 + c][threadIdx.x], sh[3 + c][threadIdx.x + w]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) parts[6 * (size_t)blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// One block of 6 warps: warp c folds component c of the box partials into
// parts[BOX_FINAL + c].
__global__ void __launch_bounds__(192) box_fold_kernel(double *__restrict__ parts, int nparts)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool is_min = warp < 3;
    double v = is_min ? DBL_MAX : -DBL_MAX;
    for (int b = lane; b < nparts; b += 32) {
        const double p = parts[6 * (size_t)b + warp];
        v = is_min ? fmin(v, p) : fmax(v, p);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_xor_sync(0xffffffffu, v, off);
        v = is_min ? fmin(v, o) : fmax(v, o);
    }
    if (lane == 0) parts[BOX_FINAL + warp] = v;
}

// Morton keys (8 bits per axis) in the folded box.
__global__ void __launch_bounds__(OTPB) morton_kernel(int n, const double *__restrict__ pos,
                                                       const double *__restrict__ parts,
                                                       unsigned *__restrict__ keys,
                                                       int *__restrict__ vals)
{
    double box[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) box[c] = parts[BOX_FINAL + c];
    const double ext = fmax(fmax(box[3] - box[0], box[4] - box[1]), box[5] - box[2]);
    const double scale = ext > 0.0 ? 256.0 / ext : 0.0;
    for (int i = blockIdx.x * OTPB + threadIdx.x; i < n; i += gridDim.x * OTPB) {
        unsigned q[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double t = (pos[3 * (size_t)i + c] - box[c]) * scale;
            t = fmin(fmax(t, 0.0), 255.0);
            q[c] = (unsigned)t;
        }
        keys[i] = spread8(q[0]) | (spread8(q[1]) << 1) | (spread8(q[2]) << 2);
        vals[i] = i;
    }
}

__device__ __forceinline__ unsigned spread10(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// 30-bit Morton keys for the tree code: q = floor((x - lo) * (1024 / ext)),
// clamped to [0, 1023], with lo the box minimum and ext its longest side, all
// in float64 (the same operations as the tree's cell geometry, so a body's
// key and its cells agree exactly).  Block 0 also stores {lo_x, lo_y, lo_z,
// ext} for the tree kernels.
__global__ void __launch_bounds__(OTPB) morton30_kernel(int n, const double *__restrict__ pos,
                                                         const double *__restrict__ parts,
                                                         unsigned *__restrict__ keys,
                                                         int *__restrict__ vals,
                                                         double *__restrict__ box_out)
{
    double box[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) box[c] = parts[BOX_FINAL + c];
    double ext = box[3] - box[0];
    if (box[4] - box[1] > ext) ext = box[4] - box[1];
    if (box[5] - box[2] > ext) ext = box[5] - box[2];
    if (!(ext > 0.0)) ext = 1.0;
    const double scale = 1024.0 / ext;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        box_out[0] = box[0];
        box_out[1] = box[1];
        box_out[2] = box[2];
        box_out[3] = ext;
    }
    for (int i = blockIdx.x * OTPB + threadIdx.x; i < n; i += gridDim.x * OTPB) {
        unsigned q[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double t = __dmul_rn(__dsub_rn(pos[3 * (size_t)i + c], box[c]), scale);
            q[c] = t >= 1023.0 ? 1023u : (t <= 0.0 ? 0u : (unsigned)t);
        }
        keys[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
        vals[i] = i;
    }
}

// Digit histogram per warp-chunk of SORT_CHUNK keys: hist[d * nchunks + chunk].
__global__ void __launch_bounds__(OTPB) radix_hist_kernel(int n, const unsigned *__restrict__ keys,
                                                           int shift, int nchunks,
                                                           unsigned *__restrict__ hist)
{
    __shared__ unsigned cnt[OTPB / 32][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < 256; d += 32) cnt[warp][d] = 0u;
    __syncwarp();
    const int chunk = blockIdx.x * (OTPB / 32) + warp;
    if (chunk < nchunks) {
        const int base = chunk * SORT_CHUNK;
        const int end = min(base + SORT_CHUNK, n);
        for (int i = base + lane; i < end; i += 32) atomicAdd(&cnt[warp][(keys[i] >> shift) & 255u], 1u);
        __syncwarp();
        for (int d = lane; d < 256; d += 32) hist[(size_t)d * nchunks + chunk] = cnt[warp][d];
    }
}

// In-place exclusive scan of hist[0..total) over several blocks: block b
// sums its segment of BSCAN_TILE entries into part[b] (radix_part_kernel),
// then scans it starting from the sum of the segments before it.
__global__ void __launch_bounds__(1024) radix_part_kernel(const unsigned *__restrict__ hist,
                                                          int total, unsigned *__restrict__ part)
{
    __shared__ unsigned ws[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int base = blockIdx.x * BSCAN_TILE;
    unsigned v = 0u;
    for (int q = threadIdx.x; q < BSCAN_TILE; q += 1024)
        if (base + q < total) v += hist[base + q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = ws[lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) part[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024) radix_scan_kernel(unsigned *__restrict__ hist, int total,
                                                          const unsigned *__restrict__ part)
{
    __shared__ unsigned tile[BSCAN_TILE + BSCAN_TILE / 32];
    __shared__ unsigned wsum[32];
    __shared__ unsigned offset;
    if (threadIdx.x < 32) {
        unsigned v = 0u;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += 32) v += part[b];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) offset = v;
    }
    __syncthreads();
    const int base = blockIdx.x * BSCAN_TILE;
    block_scan_exclusive<unsigned>(hist + base, hist + base, min(BSCAN_TILE, total - base), tile,
                                   wsum, offset);
}

inline void launch_radix_scan(cudaStream_t s, unsigned *hist, int total)
{
    const int blocks = (total + BSCAN_TILE - 1) / BSCAN_TILE;
    radix_part_kernel<<<blocks, 1024, 0, s>>>(hist, total, hist + total);
    radix_scan_kernel<<<blocks, 1024, 0, s>>>(hist, total, hist + total);
}

// Stable scatter: one warp per chunk, keys taken 32 at a time in order.
__global__ void __launch_bounds__(OTPB) radix_scatter_kernel(int n,
                                                              const unsigned *__restrict__ kin,
                                                              const int *__restrict__ vin,
                                                              unsigned *__restrict__ kout,
                                                              int *__restrict__ vout, int shift,
                                                              int nchunks,
                                                              const unsigned *__restrict__ offs)
{
    __shared__ unsigned run[OTPB / 32][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int chunk = blockIdx.x * (OTPB / 32) + warp;
    if (chunk >= nchunks) return;  // whole warp leaves together
    for (int d = lane; d < 256; d += 32) run[warp][d] = offs[(size_t)d * nchunks + chunk];
    __syncwarp();
    const int base = chunk * SORT_CHUNK;
    const int end = min(base + SORT_CHUNK, n);
    const unsigned lt = (1u << lane) - 1u;
    for (int r = base; r < end; r += 32) {
        const int i = r + lane;
        const bool valid = i < end;
        const unsigned k = valid ? kin[i] : 0u;
        const unsigned d = valid ? ((k >> shift) & 255u) : 256u + (unsigned)lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned off = 0u;
        if (valid) off = run[warp][d] + (unsigned)__popc(peers & lt);
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane) run[warp][d] += (unsigned)__popc(peers);
        __syncwarp();
        if (valid) {
            kout[off] = k;
            vout[off] = vin[i];
        }
    }
}

// Keys of a plain integer sort: keys[i] = k32[i] or k64[i] (values below
// 2^31), vals[i] = i.
__global__ void __launch_bounds__(OTPB) key_init_kernel(int n, const int *__restrict__ k32,
                                                         const long long *__restrict__ k64,
                                                         unsigned *__restrict__ keys,
                                                         int *__restrict__ vals)
{
    for (int i = blockIdx.x * OTPB + threadIdx.x; i < n; i += gridDim.x * OTPB) {
        keys[i] = k32 ? (unsigned)k32[i] : (unsigned)k64[i];
        vals[i] = i;
    }
}

// Pack body perm[k] at slot k as float32 hi/lo pairs.
__global__ void __launch_bounds__(OTPB) pack_hilo_kernel(int n, const double *__restrict__ pos,
                                                          const double *__restrict__ mass,
                                                          const int *__restrict__ perm,
                                                          float4 *__restrict__ Phi,
                                                          float4 *__restrict__ Plo)
{
    for (int k = blockIdx.x * OTPB + threadIdx.x; k < n; k += gridDim.x * OTPB) {
        const int i = perm ? perm[k] : k;
        const double *x = pos + 3 * (size_t)i;
        const float hx = (float)x[0], hy = (float)x[1], hz = (float)x[2];
        const double m = mass[i];
        Phi[k] = make_float4(hx, hy, hz, (float)m);
        Plo[k] = make_float4((float)(x[0] - (double)hx), (float)(x[1] - (double)hy),
                             (float)(x[2] - (double)hz), (float)log2(m));
    }
}

inline int grid_for(int n)
{
    int g = (n + OTPB - 1) / OTPB;
    return g < 1 ? 1 : (g > 4096 ? 4096 : g);
}

}  // namespace

int sort_chunks(int n) { return (n + SORT_CHUNK - 1) / SORT_CHUNK; }

size_t sort_hist_entries(int n)
{
    // digit counts, then one partial sum per scan block
    const size_t total = (size_t)256 * sort_chunks(n);
    return total + (total + BSCAN_TILE - 1) / BSCAN_TILE + 32;
}

cudaError_t launch_morton_sort(cudaStream_t s, int n, const double *pos, OrderScratch &o,
                               int *perm_out, int &kernels)
{
    kernels = 0;
    if (n <= 0) return cudaSuccess;
    const int nparts = grid_for(n) < MAX_BOX_PARTS ? grid_for(n) : MAX_BOX_PARTS;
    bbox_kernel<<<nparts, OTPB, 0, s>>>(n, pos, o.box);
    box_fold_kernel<<<1, 192, 0, s>>>(o.box, nparts);
    morton_kernel<<<grid_for(n), OTPB, 0, s>>>(n, pos, o.box, o.keys[0], o.vals[0]);
    kernels += 3;
    const int nchunks = sort_chunks(n);
    const int blocks = (nchunks + OTPB / 32 - 1) / (OTPB / 32);
    int cur = 0;
    for (int pass = 0; pass < 3; ++pass) {
        const int shift = 8 * pass;
        radix_hist_kernel<<<blocks, OTPB, 0, s>>>(n, o.keys[cur], shift, nchunks, o.hist);
        launch_radix_scan(s, o.hist, 256 * nchunks);
        int *vout = pass == 2 ? perm_out : o.vals[cur ^ 1];
        radix_scatter_kernel<<<blocks, OTPB, 0, s>>>(n, o.keys[cur], o.vals[cur], o.keys[cur ^ 1],
                                                     vout, shift, nchunks, o.hist);
        kernels += 4;
        cur ^= 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_tree_sort(cudaStream_t s, int n, const double *pos, OrderScratch &o,
                             int *perm_out, double *box_out, int &kernels)
{
    kernels = 0;
    if (n <= 0) return cudaSuccess;
    const int nparts = grid_for(n) < MAX_BOX_PARTS ? grid_for(n) : MAX_BOX_PARTS;
    bbox_kernel<<<nparts, OTPB, 0, s>>>(n, pos, o.box);
    box_fold_kernel<<<1, 192, 0, s>>>(o.box, nparts);
    morton30_kernel<<<grid_for(n), OTPB, 0, s>>>(n, pos, o.box, o.keys[0], o.vals[0], box_out);
    kernels += 3;
    const int nchunks = sort_chunks(n);
    const int blocks = (nchunks + OTPB / 32 - 1) / (OTPB / 32);
    int cur = 0;
    for (int pass = 0; pass < 4; ++pass) {  // 30-bit keys: 4 passes, sorted keys end in keys[0]
        const int shift = 8 * pass;
        radix_hist_kernel<<<blocks, OTPB, 0, s>>>(n, o.keys[cur], shift, nchunks, o.hist);
        launch_radix_scan(s, o.hist, 256 * nchunks);
        int *vout = pass == 3 ? perm_out : o.vals[cur ^ 1];
        radix_scatter_kernel<<<blocks, OTPB, 0, s>>>(n, o.keys[cur], o.vals[cur], o.keys[cur ^ 1],
                                                     vout, shift, nchunks, o.hist);
        kernels += 4;
        cur ^= 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_key_sort(cudaStream_t s, int n, const int *k32, const long long *k64,
                            int passes, OrderScratch &o, int *perm_out, int &kernels)
{
    kernels = 0;
    if (n <= 0) return cudaSuccess;
    key_init_kernel<<<grid_for(n), OTPB, 0, s>>>(n, k32, k64, o.keys[0], o.vals[0]);
    ++kernels;
    const int nchunks = sort_chunks(n);
    const int blocks = (nchunks + OTPB / 32 - 1) / (OTPB / 32);
    int cur = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        radix_hist_kernel<<<blocks, OTPB, 0, s>>>(n, o.keys[cur], shift, nchunks, o.hist);
        launch_radix_scan(s, o.hist, 256 * nchunks);
        int *vout = pass == passes - 1 ? perm_out : o.vals[cur ^ 1];
        radix_scatter_kernel<<<blocks, OTPB, 0, s>>>(n, o.keys[cur], o.vals[cur], o.keys[cur ^ 1],
                                                     vout, shift, nchunks, o.hist);
        kernels += 4;
        cur ^= 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_hilo(cudaStream_t s, int n, const double *pos, const double *mass,
                             const int *perm, float4 *Phi, float4 *Plo)
{
    if (n <= 0) return cudaSuccess;
    pack_hilo_kernel<<<grid_for(n), OTPB, 0, s>>>(n, pos, mass, perm, Phi, Plo);
    return cudaGetLastError();
}

}  // namespace nb
