// Barnes-Hut tree code on the GPU (paper Sec. IV-A): the bodies are placed
// in an octree by recursive 8-way division of space until a cell holds few
// enough bodies; the force on a body is the sum over the cells that are
// distant enough (as their total mass at their centre of mass) and over the
// bodies of the nearby leaves.
//
// Readings (the paper gives no opening rule, threshold or grouping):
//  * space is the cube at the bodies' box minimum with edge `ext`, the
//    longest box side; a body's cell at level L is the top 3L bits of its
//    30-bit Morton key (order.cu: launch_tree_sort);
//  * a cell is a leaf when it holds at most `leaf_cap` bodies or is at
//    level 10;
//  * bodies are taken 32 at a time in key order (one warp); the warp walks
//    the tree depth first with a shared stack, and a cell is used as a
//    monopole only when it is distant enough from every body of the warp:
//    distance from the body to the cell's cube >= edge / theta, computed in
//    float32 with the same operations as the oracle (no contraction), so
//    both take the same decisions;
//  * cell moments are float64 (mass, centre of mass).
//
// Build (all on the device, no host synchronisation, so it can be captured
// in a graph): level by level from the root, each node of level L with more
// than leaf_cap bodies finds its octant ranges by binary search on the
// sorted keys; one block scans the child counts of the level; children are
// written contiguously in octant order.  Moments are summed bottom-up.
//
// Walk arithmetic: float32 pair terms in coordinates relative to the warp's
// centre (hi/lo packed positions and centres of mass, as in the direct-sum
// kernel), float32 partial sums folded into Kahan (sum, carry) pairs after
// every node.
#include <cuda_runtime.h>
#include <float.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

constexpr int TTPB = 256;
constexpr int WALK_WARPS = 4;
constexpr int STACK_CAP = 96;  // >= 1 + 7 * 10 entries of a depth-first walk

enum { META_COUNT = 0, META_BASE = 12, META_OVERFLOW = 24, META_INTS = 32 };

inline int grid_cap(int64_t work)
{
    int64_t g = (work + TTPB - 1) / TTPB;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

__global__ void tree_init_kernel(TreeView t, int n)
{
    if (threadIdx.x < META_INTS) t.meta[threadIdx.x] = 0;
    if (threadIdx.x < 4) t.stats[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) {
        t.meta[META_COUNT + 0] = 1;
        t.start[0] = 0;
        t.end[0] = n;
        t.prefix[0] = 0u;
        t.level[0] = 0;
        t.nchild[0] = 0;
        t.first[0] = -1;
    }
}

// First key index in [lo, hi) with key >= v.
__device__ __forceinline__ int lower_bound(const unsigned *__restrict__ keys, int lo, int hi,
                                           unsigned v)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void octant_bounds(const unsigned *__restrict__ keys, int start,
                                              int end, unsigned prefix, int L, int (&b)[9])
{
    const int shift = 3 * (10 - (L + 1));
    b[0] = start;
    b[8] = end;
#pragma unroll
    for (int o = 1; o < 8; ++o) b[o] = lower_bound(keys, start, end, (prefix * 8u + o) << shift);
}

__global__ void __launch_bounds__(TTPB) tree_count_kernel(TreeView t, const unsigned *keys, int L,
                                                          int leaf_cap)
{
    const int cnt = t.meta[META_COUNT + L], base = t.meta[META_BASE + L];
    for (int q = blockIdx.x * TTPB + threadIdx.x; q < cnt; q += gridDim.x * TTPB) {
        const int node = base + q;
        const int s = t.start[node], e = t.end[node];
        int nch = 0;
        if (e - s > leaf_cap) {
            int b[9];
            octant_bounds(keys, s, e, t.prefix[node], L, b);
#pragma unroll
            for (int o = 0; o < 8; ++o) nch += b[o + 1] > b[o];
        }
        t.nchild[node] = nch;
    }
}

// One block: exclusive scan of the child counts of level L into t.offs,
// level L+1's count and base into meta (clipped at the node capacity).
__global__ void __launch_bounds__(1024) tree_scan_kernel(TreeView t, int L)
{
    __shared__ int part[1024];
    const int cnt = t.meta[META_COUNT + L], base = t.meta[META_BASE + L];
    const int seg = (cnt + 1023) / 1024;
    const int b = threadIdx.x * seg, e = min(b + seg, cnt);
    int s = 0;
    for (int q = b; q < e; ++q) s += t.nchild[base + q];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int q = b; q < e; ++q) {
        t.offs[q] = run;
        run += t.nchild[base + q];
    }
    if (threadIdx.x == 1023) {
        const int total = part[1023];
        const int nbase = base + cnt;
        int room = (int)(t.cap - nbase);
        room = room < 0 ? 0 : room;
        // Past the capacity (never, with tree_node_bound) the tree stops at
        // this level: every node of it becomes a leaf and the flag is raised.
        if (total > room) t.meta[META_OVERFLOW] = 1;
        t.meta[META_BASE + L + 1] = nbase;
        t.meta[META_COUNT + L + 1] = total > room ? 0 : total;
    }
}

__global__ void __launch_bounds__(TTPB) tree_emit_kernel(TreeView t, const unsigned *keys, int L)
{
    const int cnt = t.meta[META_COUNT + L], base = t.meta[META_BASE + L];
    const int nbase = t.meta[META_BASE + L + 1];
    const bool stop = t.meta[META_COUNT + L + 1] == 0;
    for (int q = blockIdx.x * TTPB + threadIdx.x; q < cnt; q += gridDim.x * TTPB) {
        const int node = base + q;
        const int nch = t.nchild[node];
        if (nch == 0 || stop) {
            t.nchild[node] = 0;
            t.first[node] = -1;
            continue;
        }
        const int s = t.start[node], e = t.end[node];
        const unsigned pre = t.prefix[node];
        int b[9];
        octant_bounds(keys, s, e, pre, L, b);
        const int first = nbase + t.offs[q];
        t.first[node] = first;
        int k = 0;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            if (b[o + 1] > b[o]) {
                const int c = first + k++;
                t.start[c] = b[o];
                t.end[c] = b[o + 1];
                t.prefix[c] = pre * 8u + o;
                t.level[c] = L + 1;
                t.nchild[c] = 0;
                t.first[c] = -1;
            }
        }
    }
}

// Float64 monopoles of level L (children first: call from level 10 up).
__global__ void __launch_bounds__(TTPB) tree_moments_kernel(TreeView t, const double *__restrict__ pos,
                                                            const double *__restrict__ mass,
                                                            const int *__restrict__ perm, int L)
{
    const int cnt = t.meta[META_COUNT + L], base = t.meta[META_BASE + L];
    for (int q = blockIdx.x * TTPB + threadIdx.x; q < cnt; q += gridDim.x * TTPB) {
        const int node = base + q;
        double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        const int nch = t.nchild[node];
        if (nch == 0) {
            for (int k = t.start[node]; k < t.end[node]; ++k) {
                const int j = perm[k];
                const double m = mass[j];
                M += m;
                sx += m * pos[3 * (size_t)j];
                sy += m * pos[3 * (size_t)j + 1];
                sz += m * pos[3 * (size_t)j + 2];
            }
        } else {
            const int f = t.first[node];
            for (int c = f; c < f + nch; ++c) {
                const double m = t.M[c];
                M += m;
                sx += m * t.com[3 * (size_t)c];
                sy += m * t.com[3 * (size_t)c + 1];
                sz += m * t.com[3 * (size_t)c + 2];
            }
        }
        t.M[node] = M;
        t.com[3 * (size_t)node] = M > 0.0 ? sx / M : 0.0;
        t.com[3 * (size_t)node + 1] = M > 0.0 ? sy / M : 0.0;
        t.com[3 * (size_t)node + 2] = M > 0.0 ? sz / M : 0.0;
    }
}

// Walk data of every node: float32 cube (exactly as the oracle forms it),
// centre of mass as a float32 hi/lo pair and mass.
__global__ void __launch_bounds__(TTPB) tree_walkdata_kernel(TreeView t, const double *__restrict__ box)
{
    const int total = t.meta[META_BASE + 10] + t.meta[META_COUNT + 10];
    const double lo[3] = {box[0], box[1], box[2]};
    const double ext = box[3];
    if (blockIdx.x == 0 && threadIdx.x == 0) t.stats[0] = (unsigned long long)total;
    int leaves = 0;
    for (int node = blockIdx.x * TTPB + threadIdx.x; node < total; node += gridDim.x * TTPB) {
        const int L = t.level[node];
        leaves += t.nchild[node] == 0;
        const unsigned pre = t.prefix[node];
        unsigned ic[3] = {0u, 0u, 0u};
        for (int bb = 0; bb < L; ++bb) {
            const unsigned trip = (pre >> (3 * bb)) & 7u;
#pragma unroll
            for (int c = 0; c < 3; ++c) ic[c] |= ((trip >> c) & 1u) << bb;
        }
        const double cell = __ddiv_rn(ext, (double)(1u << L));
        float blo[3], bhi[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            blo[c] = (float)__dadd_rn(lo[c], __dmul_rn(cell, (double)ic[c]));
            bhi[c] = (float)__dadd_rn(lo[c], __dmul_rn(cell, (double)(ic[c] + 1u)));
        }
        t.box_lo[node] = make_float4(blo[0], blo[1], blo[2], 0.f);
        t.box_hi[node] = make_float4(bhi[0], bhi[1], bhi[2], 0.f);
        const double cx = t.com[3 * (size_t)node], cy = t.com[3 * (size_t)node + 1],
                     cz = t.com[3 * (size_t)node + 2];
        const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
        t.chi[node] = make_float4(hx, hy, hz, (float)t.M[node]);
        t.clo[node] = make_float4((float)(cx - (double)hx), (float)(cy - (double)hy),
                                  (float)(cz - (double)hz), 0.f);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) leaves += __shfl_xor_sync(0xffffffffu, leaves, off);
    if ((threadIdx.x & 31) == 0 && leaves) atomicAdd(t.stats + 1, (unsigned long long)leaves);
}

// Squared opening distance of a level, as the oracle computes it.
__device__ __forceinline__ float open_dist2(double ext, int L, float theta)
{
    const float edge = (float)__ddiv_rn(ext, (double)(1u << L));
    const float d = __fdiv_rn(edge, theta);
    return __fmul_rn(d, d);
}

// Squared distance from p to the cube [lo, hi], no contraction.
__device__ __forceinline__ float cube_dist2(float4 lo, float4 hi, float px, float py, float pz)
{
    float d2 = 0.0f;
    const float pl[3] = {lo.x, lo.y, lo.z}, ph[3] = {hi.x, hi.y, hi.z}, pp[3] = {px, py, pz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a = __fsub_rn(pl[c], pp[c]);
        const float b = __fsub_rn(pp[c], ph[c]);
        float dd = a > b ? a : b;
        dd = dd > 0.0f ? dd : 0.0f;
        d2 = __fadd_rn(d2, __fmul_rn(dd, dd));
    }
    return d2;
}

template <bool ZEPS>
__device__ __forceinline__ void pair1(float dx, float dy, float dz, float m, float e2, float &ax,
                                      float &ay, float &az)
{
    float r2 = fmaf(dx, dx, e2);
    r2 = fmaf(dy, dy, r2);
    r2 = fmaf(dz, dz, r2);
    float ri = rsqrt_mufu(r2);
    if (ZEPS) ri = r2 > 0.f ? ri : 0.f;
    const float s = (m * ri) * (ri * ri);
    ax = fmaf(dx, s, ax);
    ay = fmaf(dy, s, ay);
    az = fmaf(dz, s, az);
}

template <bool ZEPS>
__global__ void __launch_bounds__(32 * WALK_WARPS) tree_walk_kernel(const TreeWalkParams p)
{
    __shared__ int stack[WALK_WARPS][STACK_CAP];
    __shared__ float crit2[11];
    const TreeView t = p.tree;
    if (threadIdx.x < 11) crit2[threadIdx.x] = open_dist2(p.box[3], threadIdx.x, p.theta);
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = p.n;
    const int k = (blockIdx.x * WALK_WARPS + warp) * 32 + lane;
    if ((blockIdx.x * WALK_WARPS + warp) * 32 >= n) return;  // whole warp past the end
    const bool valid = k < n;
    const float4 h = valid ? __ldg(p.P + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 l = valid ? __ldg(p.Plo + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    // warp centre (box midpoint of the valid bodies) as the coordinate origin
    float mn[3] = {valid ? h.x : INFINITY, valid ? h.y : INFINITY, valid ? h.z : INFINITY};
    float mx[3] = {valid ? h.x : -INFINITY, valid ? h.y : -INFINITY, valid ? h.z : -INFINITY};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], off));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], off));
        }
    }
    const float cx = 0.5f * (mn[0] + mx[0]), cy = 0.5f * (mn[1] + mx[1]),
                cz = 0.5f * (mn[2] + mx[2]);
    const float xi = rel(h.x, l.x, cx), yi = rel(h.y, l.y, cy), zi = rel(h.z, l.z, cz);
    const float e2 = p.eps2f;

    float ax = 0.f, ay = 0.f, az = 0.f;
    float sx = 0.f, sy = 0.f, sz = 0.f, qx = 0.f, qy = 0.f, qz = 0.f;
    int nc = 0, nb = 0;
    int *st = stack[warp];
    if (lane == 0) st[0] = 0;
    int sp = 1;
    __syncwarp();
    while (sp > 0) {
        const int node = st[--sp];
        __syncwarp();
        const float4 blo = __ldg(t.box_lo + node), bhi = __ldg(t.box_hi + node);
        const int L = t.level[node];
        const int nch = t.nchild[node];
        const bool ok = !valid || cube_dist2(blo, bhi, h.x, h.y, h.z) >= crit2[L];
        const bool all = __all_sync(0xffffffffu, ok);
        if (all) {
            const float4 ch = __ldg(t.chi + node), cl = __ldg(t.clo + node);
            pair1<ZEPS>(rel(ch.x, cl.x, cx) - xi, rel(ch.y, cl.y, cy) - yi,
                        rel(ch.z, cl.z, cz) - zi, ch.w, e2, ax, ay, az);
            ++nc;
        } else if (nch == 0) {
            const int s = t.start[node], e = t.end[node];
            for (int j = s; j < e; ++j) {
                const float4 bh = __ldg(p.P + j), bl = __ldg(p.Plo + j);
                pair1<ZEPS>(rel(bh.x, bl.x, cx) - xi, rel(bh.y, bl.y, cy) - yi,
                            rel(bh.z, bl.z, cz) - zi, bh.w, e2, ax, ay, az);
            }
            nb += e - s;
        } else {
            const int f = t.first[node];
            if (lane < nch && sp + lane < STACK_CAP) st[sp + lane] = f + nch - 1 - lane;
            sp += nch;
            if (sp > STACK_CAP) {  // cannot happen for 10 levels; keep the walk in bounds
                if (lane == 0) atomicOr(p.err, ERR_TREE);
                sp = STACK_CAP;
            }
            __syncwarp();
            continue;
        }
        kahan_add(sx, qx, ax);
        kahan_add(sy, qy, ay);
        kahan_add(sz, qz, az);
        ax = ay = az = 0.f;
    }
    if (valid) {
        const int i = p.perm[k];
        const double gx = p.G * ((double)sx - (double)qx);
        const double gy = p.G * ((double)sy - (double)qy);
        const double gz = p.G * ((double)sz - (double)qz);
        double *a = p.acc + 3 * (size_t)i;
        a[0] = gx;
        a[1] = gy;
        a[2] = gz;
        if (p.vel) {
            double *v = p.vel + 3 * (size_t)i;
            v[0] += p.half_dt * gx;
            v[1] += p.half_dt * gy;
            v[2] += p.half_dt * gz;
        }
        if (p.counts) {
            p.counts[2 * (size_t)i] = nc;
            p.counts[2 * (size_t)i + 1] = nb;
        }
        if (!finite3(gx, gy, gz)) atomicOr(p.err, ERR_NONFINITE);
    }
    unsigned long long cnt[2] = {valid ? (unsigned long long)nc : 0ull,
                                 valid ? (unsigned long long)nb : 0ull};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        cnt[0] += __shfl_xor_sync(0xffffffffu, cnt[0], off);
        cnt[1] += __shfl_xor_sync(0xffffffffu, cnt[1], off);
    }
    if (lane == 0) {
        atomicAdd(t.stats + 2, cnt[0]);
        atomicAdd(t.stats + 3, cnt[1]);
    }
}

__global__ void tree_flag_kernel(TreeView t, int *err)
{
    if (threadIdx.x == 0 && t.meta[META_OVERFLOW]) atomicOr(err, ERR_TREE);
}

}  // namespace

int tree_meta_ints() { return META_INTS; }

int64_t tree_node_bound(int64_t n, int leaf_cap)
{
    // Nodes of one level are disjoint and non-empty (<= n), at most 8^L, and
    // children of the split nodes of the level above, which hold more than
    // leaf_cap bodies each (<= 8 n / (leaf_cap + 1)).
    if (n <= 0) return 1;
    const int64_t split = leaf_cap >= 1 ? n / ((int64_t)leaf_cap + 1) : n;
    int64_t total = 1, p8 = 1;
    for (int L = 1; L <= 10; ++L) {
        p8 *= 8;
        int64_t c = p8 < n ? p8 : n;
        if (8 * split < c) c = 8 * split;
        total += c;
    }
    return total;
}

cudaError_t launch_tree_build(cudaStream_t s, const TreeView &t, int n, const unsigned *keys,
                              const double *box, const double *pos, const double *mass,
                              const int *perm, int leaf_cap, int *err, int &kernels)
{
    kernels = 0;
    tree_init_kernel<<<1, 32, 0, s>>>(t, n);
    ++kernels;
    const int g = grid_cap(n);
    for (int L = 0; L < 10; ++L) {
        tree_count_kernel<<<g, TTPB, 0, s>>>(t, keys, L, leaf_cap);
        tree_scan_kernel<<<1, 1024, 0, s>>>(t, L);
        tree_emit_kernel<<<g, TTPB, 0, s>>>(t, keys, L);
        kernels += 3;
    }
    for (int L = 10; L >= 0; --L) {
        tree_moments_kernel<<<g, TTPB, 0, s>>>(t, pos, mass, perm, L);
        ++kernels;
    }
    tree_walkdata_kernel<<<grid_cap(t.cap), TTPB, 0, s>>>(t, box);
    tree_flag_kernel<<<1, 32, 0, s>>>(t, err);
    kernels += 2;
    return cudaGetLastError();
}

cudaError_t launch_tree_walk(cudaStream_t s, const TreeWalkParams &p, bool zeps, int &kernels)
{
    kernels = 0;
    if (p.n <= 0) return cudaSuccess;
    const int groups = (p.n + 31) / 32;
    const int blocks = (groups + WALK_WARPS - 1) / WALK_WARPS;
    if (zeps)
        tree_walk_kernel<true><<<blocks, 32 * WALK_WARPS, 0, s>>>(p);
    else
        tree_walk_kernel<false><<<blocks, 32 * WALK_WARPS, 0, s>>>(p);
    kernels = 1;
    return cudaGetLastError();
}

}  // namespace nb
