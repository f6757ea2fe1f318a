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

// One warp per node: lane o (1..7) finds where octant o starts in the
// node's sorted keys, lane 0 holds start and lane 8 end; lane o < 8 then
// sees whether child o is non-empty.  Returns the ballot of non-empty
// children (bit o) and leaves the child's range in [b, nxt) on lane o.
__device__ __forceinline__ unsigned octants(const unsigned *__restrict__ keys, int s, int e,
                                            unsigned prefix, int L, int lane, int &b, int &nxt)
{
    const int shift = 3 * (10 - (L + 1));
    b = lane == 0 ? s : (lane <= 7 ? lower_bound(keys, s, e, (prefix * 8u + lane) << shift) : e);
    nxt = __shfl_down_sync(0xffffffffu, b, 1);
    return __ballot_sync(0xffffffffu, lane < 8 && nxt > b);
}

__global__ void __launch_bounds__(TTPB) tree_count_kernel(TreeView t, const unsigned *keys, int L,
                                                          int leaf_cap)
{
    const int cnt = t.meta[META_COUNT + L], base = t.meta[META_BASE + L];
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (TTPB / 32);
    for (int q = blockIdx.x * (TTPB / 32) + (threadIdx.x >> 5); q < cnt; q += warps) {
        const int node = base + q;
        const int s = t.start[node], e = t.end[node];
        int nch = 0;
        if (e - s > leaf_cap) {
            int b, nxt;
            nch = __popc(octants(keys, s, e, t.prefix[node], L, lane, b, nxt));
        }
        if (lane == 0) t.nchild[node] = nch;
    }
}

// One block: exclusive scan of the child counts of level L into t.offs,
// level L+1's count and base into meta.
__global__ void __launch_bounds__(1024) tree_scan_kernel(TreeView t, int L)
{
    __shared__ int tile[BSCAN_TILE + BSCAN_TILE / 32];
    __shared__ int wsum[32];
    const int cnt = t.meta[META_COUNT + L], base = t.meta[META_BASE + L];
    const int total = block_scan_exclusive<int>(t.nchild + base, t.offs, cnt, tile, wsum);
    if (threadIdx.x == 0) {
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
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int warps = gridDim.x * (TTPB / 32);
    for (int q = blockIdx.x * (TTPB / 32) + (threadIdx.x >> 5); q < cnt; q += warps) {
        const int node = base + q;
        const int nch = t.nchild[node];
        if (nch == 0 || stop) {
            if (lane == 0) {
                t.nchild[node] = 0;
                t.first[node] = -1;
            }
            continue;
        }
        const unsigned pre = t.prefix[node];
        int b, nxt;
        const unsigned ne = octants(keys, t.start[node], t.end[node], pre, L, lane, b, nxt);
        const int first = nbase + t.offs[q];
        if (lane == 0) t.first[node] = first;
        if (lane < 8 && ((ne >> lane) & 1u)) {
            const int c = first + __popc(ne & lt);
            t.start[c] = b;
            t.end[c] = nxt;
            t.prefix[c] = pre * 8u + lane;
            t.level[c] = L + 1;
            t.nchild[c] = 0;
            t.first[c] = -1;
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
        // .w carries the child count and first child for the walk
        t.box_lo[node] = make_float4(blo[0], blo[1], blo[2], __int_as_float(t.nchild[node]));
        t.box_hi[node] = make_float4(bhi[0], bhi[1], bhi[2], __int_as_float(t.first[node]));
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

// Squared distance from the cube [lo, hi] to the box [mn, mx], written as
// cube_dist2 with the box's far corner in each difference.  Rounding is
// monotonic, so for every p inside the box this value is <= cube_dist2(p):
// when it passes the opening test, every body of the box passes it too.
__device__ __forceinline__ float cube_box_dist2(float4 lo, float4 hi, const float (&mn)[3],
                                                const float (&mx)[3])
{
    float d2 = 0.0f;
    const float pl[3] = {lo.x, lo.y, lo.z}, ph[3] = {hi.x, hi.y, hi.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a = __fsub_rn(pl[c], mx[c]);
        const float b = __fsub_rn(mn[c], ph[c]);
        float dd = a > b ? a : b;
        dd = dd > 0.0f ? dd : 0.0f;
        d2 = __fadd_rn(d2, __fmul_rn(dd, dd));
    }
    return d2;
}

// Interaction list of a warp: up to LIST_CAP sources (cells or bodies) as
// (x, y, z, m), coordinates relative to the warp's centre, stored in pairs
// so that one pair is two float4 loads, already in float32x2 order:
// {x0, x1, y0, y1}, {z0, z1, m0, m1}.
constexpr int LIST_CAP = 64;
constexpr int LEVELS = 11;

__device__ __forceinline__ void list_put(float *L, int q, float x, float y, float z, float m)
{
    float *b = L + 8 * (q >> 1) + (q & 1);
    b[0] = x;
    b[2] = y;
    b[4] = z;
    b[6] = m;
}

// Accumulate the first 2 * npairs sources of the list onto this lane's body
// (float32x2 over source pairs: one instruction covers two sources).
template <bool ZEPS>
__device__ __forceinline__ void list_eval(const float4 *L4, int npairs, float2 nx, float2 ny,
                                          float2 nz, float2 e2, float2 &ax, float2 &ay, float2 &az)
{
#pragma unroll 4
    for (int q = 0; q < npairs; ++q) {
        const float4 A = L4[2 * q], B = L4[2 * q + 1];
        const float2 dx = add2(make_float2(A.x, A.y), nx);
        const float2 dy = add2(make_float2(A.z, A.w), ny);
        const float2 dz = add2(make_float2(B.x, B.y), nz);
        float2 r2 = fma2(dx, dx, e2);
        r2 = fma2(dy, dy, r2);
        r2 = fma2(dz, dz, r2);
        float2 ri = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
        if (ZEPS) {
            ri.x = r2.x > 0.f ? ri.x : 0.f;
            ri.y = r2.y > 0.f ? ri.y : 0.f;
        }
        const float2 s = mul2(mul2(make_float2(B.z, B.w), ri), mul2(ri, ri));
        ax = fma2(dx, s, ax);
        ay = fma2(dy, s, ay);
        az = fma2(dz, s, az);
    }
}

// One warp per 32 consecutive bodies in key order.  The warp walks the tree
// level by level, deepest level first, 32 nodes per round (one per lane):
// the opening test against the 32 bodies decides, per node, between the
// interaction list (accepted cell: its monopole; leaf: its bodies) and
// descending (its children, a contiguous range, go on the next level's
// stack).  Each level's stack holds at most 32 ranges, the children of one
// round's nodes, since a level is refilled only once every deeper level is
// empty.  Whenever 32 sources are listed, every lane adds them to its body.
template <bool ZEPS>
__global__ void __launch_bounds__(32 * WALK_WARPS) tree_walk_kernel(const TreeWalkParams p)
{
    __shared__ float4 list_s[WALK_WARPS][LIST_CAP];
    __shared__ int2 ranges_s[WALK_WARPS][LEVELS][32];
    __shared__ int slot_s[WALK_WARPS][32];
    __shared__ float crit2[LEVELS];
    const TreeView t = p.tree;
    if (threadIdx.x < LEVELS) crit2[threadIdx.x] = open_dist2(p.box[3], threadIdx.x, p.theta);
    __syncthreads();

    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = p.n;
    const int base = (blockIdx.x * WALK_WARPS + warp) * 32;
    if (base >= n) return;  // whole warp past the end
    const int k = base + lane;
    const int nvalid = min(32, n - base);
    const bool valid = k < n;
    const float4 h = valid ? __ldg(p.P + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 l = valid ? __ldg(p.Plo + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    float mn[3] = {valid ? h.x : INFINITY, valid ? h.y : INFINITY, valid ? h.z : INFINITY};
    float mx[3] = {valid ? h.x : -INFINITY, valid ? h.y : -INFINITY, valid ? h.z : -INFINITY};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(FULL, mn[c], off));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(FULL, mx[c], off));
        }
    }
    const float cx = 0.5f * (mn[0] + mx[0]), cy = 0.5f * (mn[1] + mx[1]),
                cz = 0.5f * (mn[2] + mx[2]);
    const float xi = rel(h.x, l.x, cx), yi = rel(h.y, l.y, cy), zi = rel(h.z, l.z, cz);
    const float2 nx = make_float2(-xi, -xi), ny = make_float2(-yi, -yi), nz = make_float2(-zi, -zi);
    const float2 e2 = make_float2(p.eps2f, p.eps2f);

    float *L = reinterpret_cast<float *>(list_s[warp]);
    const float4 *L4 = list_s[warp];
    int2(*rs)[32] = ranges_s[warp];
    int *slot = slot_s[warp];
    const unsigned lt = (1u << lane) - 1u;

    float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
    float sx = 0.f, sy = 0.f, sz = 0.f, qx = 0.f, qy = 0.f, qz = 0.f;
    auto fold = [&]() {
        kahan_add(sx, qx, ax.x);
        kahan_add(sx, qx, ax.y);
        kahan_add(sy, qy, ay.x);
        kahan_add(sy, qy, ay.y);
        kahan_add(sz, qz, az.x);
        kahan_add(sz, qz, az.y);
        ax = ay = az = make_float2(0.f, 0.f);
    };
    int cnt = 0;  // listed sources (warp-uniform)
    // 32 sources listed: add them, move the rest (< 32) to the front
    auto flush32 = [&]() {
        __syncwarp();
        list_eval<ZEPS>(L4, 16, nx, ny, nz, e2, ax, ay, az);
        fold();
        __syncwarp();
        list_s[warp][lane] = list_s[warp][LIST_CAP / 2 + lane];
        cnt -= 32;
        __syncwarp();
    };

    int nc = 0, nb = 0;
    int lsize = lane == 0 ? 1 : 0;  // lane L holds the size of level L's stack
    if (lane == 0) rs[0][0] = make_int2(0, 1);
    __syncwarp();
    for (;;) {
        const unsigned nonempty = __ballot_sync(FULL, lane < LEVELS && lsize > 0);
        if (!nonempty) break;
        const int Lv = 31 - __clz(nonempty);
        const int size = __shfl_sync(FULL, lsize, Lv);
        // take up to 32 nodes from the top ranges of level Lv
        const int R = min(size, 32);
        const int2 r = lane < R ? rs[Lv][size - 1 - lane] : make_int2(0, 0);
        int incl = r.y;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += v;
        }
        const int excl = incl - r.y;
        const int take = min(__shfl_sync(FULL, incl, 31), 32);
        if (lane < R)
            for (int q = excl; q < incl && q < 32; ++q) slot[q] = r.x + (q - excl);
        const unsigned done = __ballot_sync(FULL, lane < R && incl <= 32);
        if (lane < R && excl < 32 && incl > 32)
            rs[Lv][size - 1 - lane] = make_int2(r.x + (32 - excl), incl - 32);
        __syncwarp();
        const int node = lane < take ? slot[lane] : -1;
        if (lane == Lv) lsize -= __popc(done);
        __syncwarp();

        // opening test: the warp's box first, then body by body
        const bool has = node >= 0;
        float4 blo = make_float4(0.f, 0.f, 0.f, 0.f), bhi = blo;
        if (has) {
            blo = __ldg(t.box_lo + node);
            bhi = __ldg(t.box_hi + node);
        }
        const float cr = crit2[Lv];
        bool accept = has && cube_box_dist2(blo, bhi, mn, mx) >= cr;
        // undecided nodes one at a time, every lane testing its own body
        unsigned und = __ballot_sync(FULL, has && !accept);
        while (und) {
            const int j = __ffs(und) - 1;
            und &= und - 1;
            const float4 jlo = make_float4(__shfl_sync(FULL, blo.x, j), __shfl_sync(FULL, blo.y, j),
                                           __shfl_sync(FULL, blo.z, j), 0.f);
            const float4 jhi = make_float4(__shfl_sync(FULL, bhi.x, j), __shfl_sync(FULL, bhi.y, j),
                                           __shfl_sync(FULL, bhi.z, j), 0.f);
            const bool all = __all_sync(FULL, !valid || cube_dist2(jlo, jhi, h.x, h.y, h.z) >= cr);
            if (lane == j) accept = all;
        }
        const int nch = has ? __float_as_int(blo.w) : 0;
        const bool open = has && !accept && nch > 0;
        const bool leaf = has && !accept && nch == 0;

        // children ranges onto the next level (Lv < 10 whenever a node opens)
        const unsigned om = __ballot_sync(FULL, open);
        if (om) {
            const int size1 = __shfl_sync(FULL, lsize, Lv + 1);
            const int slot1 = size1 + __popc(om & lt);
            if (open && slot1 < 32) rs[Lv + 1][slot1] = make_int2(__float_as_int(bhi.w), nch);
            if (lane == Lv + 1) lsize = min(size1 + __popc(om), 32);
            if (lane == 0 && size1 + __popc(om) > 32) atomicOr(p.err, ERR_TREE);  // never: see above
        }
        __syncwarp();
        // accepted cells: their monopoles
        const unsigned am = __ballot_sync(FULL, accept);
        if (am) {
            if (accept) {
                const float4 ch = __ldg(t.chi + node), cl = __ldg(t.clo + node);
                list_put(L, cnt + __popc(am & lt), rel(ch.x, cl.x, cx), rel(ch.y, cl.y, cy),
                         rel(ch.z, cl.z, cz), ch.w);
            }
            cnt += __popc(am);
            nc += __popc(am);
            if (cnt >= 32) flush32();
        }
        // leaves: their bodies, 32 at a time
        unsigned lm = __ballot_sync(FULL, leaf);
        int ls = 0, le = 0;
        if (leaf) {
            ls = t.start[node];
            le = t.end[node];
        }
        while (lm) {
            const int src = __ffs(lm) - 1;
            lm &= lm - 1;
            const int s0 = __shfl_sync(FULL, ls, src), e0 = __shfl_sync(FULL, le, src);
            nb += e0 - s0;
            for (int j0 = s0; j0 < e0; j0 += 32) {
                const int kk = min(32, e0 - j0);
                if (lane < kk) {
                    const float4 bh = __ldg(p.P + j0 + lane), bl = __ldg(p.Plo + j0 + lane);
                    list_put(L, cnt + lane, rel(bh.x, bl.x, cx), rel(bh.y, bl.y, cy),
                             rel(bh.z, bl.z, cz), bh.w);
                }
                cnt += kk;
                if (cnt >= 32) flush32();
            }
        }
    }
    if (cnt > 0) {  // the rest, padded to a pair with a massless source
        if (lane == 0 && (cnt & 1)) list_put(L, cnt, 0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        list_eval<ZEPS>(L4, (cnt + 1) >> 1, nx, ny, nz, e2, ax, ay, az);
        fold();
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
    if (lane == 0) {  // nc, nb are the same for the group's nvalid bodies
        atomicAdd(t.stats + 2, (unsigned long long)nc * nvalid);
        atomicAdd(t.stats + 3, (unsigned long long)nb * nvalid);
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
