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
//  * bodies are taken 32 or 64 at a time in key order (one warp per
//    group); a cell is used as a monopole only when it is distant enough
//    from every body of the group: distance from the body to the cell's
//    cube >= edge / theta, computed in float32 with the same operations as
//    the oracle (no contraction), so both take the same decisions;
//  * cell moments are float64 (mass, centre of mass).
//
// Build (all on the device, no host synchronisation, so it can be captured
// in a graph): level by level from the root, each node of level L with more
// than leaf_cap bodies finds its octant ranges by binary search on the
// sorted keys (one warp per node); one block scans the child counts of the
// level; children are written contiguously in octant order.  Moments are
// summed bottom-up.
//
// Walk arithmetic: float32 pair terms in coordinates relative to the
// group's centre (hi/lo packed positions and centres of mass, as in the
// direct-sum kernel), float32 partial sums over every NB_WALK_FOLD_EVERY
// flushes of FLUSH listed sources folded into Kahan (sum, carry) pairs.
#include <cuda_runtime.h>
#include <float.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

constexpr int TTPB = 256;
// Walk launch shape: warps per block, and the resident blocks per SM the
// register allocation is sized for (one and two bodies per lane).
#ifndef NB_WALK_WARPS
#define NB_WALK_WARPS 4
#endif
#ifndef NB_WALK_MINB1
#define NB_WALK_MINB1 8
#endif
#ifndef NB_WALK_MINB2
#define NB_WALK_MINB2 5
#endif
constexpr int WALK_WARPS = NB_WALK_WARPS;

enum { META_COUNT = 0, META_BASE = 12, META_OVERFLOW = 24, META_QUEUE = 25, META_INTS = 32 };
static_assert(META_COUNT == TREE_META_COUNT && META_BASE == TREE_META_BASE &&
                  META_QUEUE == TREE_META_QUEUE, "meta layout shared with nb_internal.h");

inline int grid_cap(int64_t work)
{
    int64_t g = (work + TTPB - 1) / TTPB;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

// 2^-L exactly (0 <= L <= 10), from its bit pattern.
__device__ __forceinline__ double pow2_neg(int L)
{
    return __longlong_as_double((long long)(1023 - L) << 52);
}

// Float32 cube of the level-L cell with key prefix `pre`, exactly as the
// oracle forms it (float64 lo + edge * index, rounded); .w of the corners
// carries the child count (0) and first child (-1) until the node's own
// level is built.
__device__ __forceinline__ void cube_corners(const double *__restrict__ box, int L, unsigned pre,
                                             float4 &lo4, float4 &hi4)
{
    unsigned ic[3] = {0u, 0u, 0u};
    for (int bb = 0; bb < L; ++bb) {
        const unsigned trip = (pre >> (3 * bb)) & 7u;
#pragma unroll
        for (int c = 0; c < 3; ++c) ic[c] |= ((trip >> c) & 1u) << bb;
    }
    // ext / 2^L: the product with the exact power 2^-L rounds the same real
    // value as the quotient, so it is the same number, without a division
    const double cell = __dmul_rn(box[3], pow2_neg(L));
    float blo[3], bhi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        blo[c] = (float)__dadd_rn(box[c], __dmul_rn(cell, (double)ic[c]));
        bhi[c] = (float)__dadd_rn(box[c], __dmul_rn(cell, (double)(ic[c] + 1u)));
    }
    lo4 = make_float4(blo[0], blo[1], blo[2], __int_as_float(0));
    hi4 = make_float4(bhi[0], bhi[1], bhi[2], __int_as_float(-1));
}

__global__ void tree_init_kernel(TreeView t, int n, const double *box)
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
        t.parent[0] = -1;
        t.arrive[0] = 0;
        cube_corners(box, 0, 0u, t.box_lo[0], t.box_hi[0]);
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

__global__ void __launch_bounds__(TTPB) tree_emit_kernel(TreeView t, const unsigned *keys,
                                                         const double *__restrict__ box, int L)
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
        if (lane == 0) {
            t.first[node] = first;
            reinterpret_cast<int *>(t.box_lo + node)[3] = nch;  // the walk's child count
            reinterpret_cast<int *>(t.box_hi + node)[3] = first;
        }
        if (lane < 8 && ((ne >> lane) & 1u)) {
            const int c = first + __popc(ne & lt);
            t.start[c] = b;
            t.end[c] = nxt;
            t.prefix[c] = pre * 8u + lane;
            t.level[c] = L + 1;
            t.nchild[c] = 0;
            t.first[c] = -1;
            t.parent[c] = node;
            t.arrive[c] = 0;
            cube_corners(box, L + 1, pre * 8u + lane, t.box_lo[c], t.box_hi[c]);
        }
    }
}

// Walk data of a node whose float64 moments are final: mass and centre of
// mass as a float32 hi/lo pair.
__device__ __forceinline__ void put_walk_moments(const TreeView &t, int node, double M, double cx,
                                                 double cy, double cz)
{
    t.M[node] = M;
    t.com[3 * (size_t)node] = cx;
    t.com[3 * (size_t)node + 1] = cy;
    t.com[3 * (size_t)node + 2] = cz;
    const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
    t.chi[node] = make_float4(hx, hy, hz, (float)M);
    t.clo[node] = make_float4((float)(cx - (double)hx), (float)(cy - (double)hy),
                              (float)(cz - (double)hz), 0.f);
}

// Float64 monopoles of every node in one launch, bottom-up without any wait:
// a thread per leaf sums its bodies, then climbs; at each parent it counts
// itself in with an atomic, and only the last child to arrive goes on to
// sum the parent's children (in child order, so the result does not depend
// on who arrives last).  Fences order the moments before the arrival.
__global__ void __launch_bounds__(TTPB) tree_moments_kernel(TreeView t, const double *__restrict__ pos,
                                                            const double *__restrict__ mass,
                                                            const int *__restrict__ perm)
{
    const int total = t.meta[META_BASE + 10] + t.meta[META_COUNT + 10];
    if (blockIdx.x == 0 && threadIdx.x == 0) t.stats[0] = (unsigned long long)total;
    int leaves = 0;
    for (int leaf = blockIdx.x * TTPB + threadIdx.x; leaf < total; leaf += gridDim.x * TTPB) {
        if (t.nchild[leaf] != 0) continue;
        ++leaves;
        double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int k = t.start[leaf]; k < t.end[leaf]; ++k) {
            const int j = perm[k];
            const double m = mass[j];
            M += m;
            sx += m * pos[3 * (size_t)j];
            sy += m * pos[3 * (size_t)j + 1];
            sz += m * pos[3 * (size_t)j + 2];
        }
        put_walk_moments(t, leaf, M, M > 0.0 ? sx / M : 0.0, M > 0.0 ? sy / M : 0.0,
                         M > 0.0 ? sz / M : 0.0);
        for (int node = t.parent[leaf]; node >= 0; node = t.parent[node]) {
            __threadfence();
            if (atomicAdd(t.arrive + node, 1) != t.nchild[node] - 1) break;
            __threadfence();
            const int f = t.first[node], nch = t.nchild[node];
            M = sx = sy = sz = 0.0;
            for (int c = f; c < f + nch; ++c) {
                const double m = __ldcg(t.M + c);
                M += m;
                sx += m * __ldcg(t.com + 3 * (size_t)c);
                sy += m * __ldcg(t.com + 3 * (size_t)c + 1);
                sz += m * __ldcg(t.com + 3 * (size_t)c + 2);
            }
            put_walk_moments(t, node, M, M > 0.0 ? sx / M : 0.0, M > 0.0 ? sy / M : 0.0,
                             M > 0.0 ? sz / M : 0.0);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) leaves += __shfl_xor_sync(0xffffffffu, leaves, off);
    if ((threadIdx.x & 31) == 0 && leaves) atomicAdd(t.stats + 1, (unsigned long long)leaves);
}

// Squared opening distance of a level, as the oracle computes it.
__device__ __forceinline__ float open_dist2(double ext, int L, float theta)
{
    const float edge = (float)__dmul_rn(ext, pow2_neg(L));  // = ext / 2^L
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

// Interaction list of a warp: a ring of LIST_CAP sources (cells or bodies)
// as (x, y, z, m), coordinates relative to the group's centre, laid out for
// float32x2 arithmetic.  A flush evaluates the FLUSH sources of the half the
// ring's head is in and moves the head to the other half; at most
// FLUSH - 1 + 32 sources are ever listed, so new ones never reach the half
// being evaluated.  Paired layout: two sources share an instruction,
// a pair of sources is {x0, x1, y0, y1}, {z0, z1, m0, m1} (one body per
// lane, or each of a lane's two bodies in turn).  Doubled layout (two
// bodies per lane, NB_WALK_PAIRED 0): one source meets both bodies, stored
// twice over, {x, x, y, y}, {z, z, m, m}.
#ifndef NB_WALK_FLUSH
#define NB_WALK_FLUSH 64
#endif
#ifndef NB_WALK_PAIRED
#define NB_WALK_PAIRED 1
#endif
#ifndef NB_WALK_FOLD_EVERY
#define NB_WALK_FOLD_EVERY 4  // flushes between Kahan folds of the float32 partials
#endif
constexpr int FLUSH = NB_WALK_FLUSH;  // sources evaluated per flush (a multiple of 32)
constexpr int LIST_CAP = 2 * FLUSH;
constexpr int LEVELS = 11;

template <int BPL>
__host__ __device__ constexpr bool paired_list() { return BPL == 1 || NB_WALK_PAIRED; }
// float4 slots of a list of LIST_CAP sources
template <int BPL>
__host__ __device__ constexpr int list_f4() { return paired_list<BPL>() ? LIST_CAP : LIST_CAP * 2; }

template <int BPL>
__device__ __forceinline__ void list_put(float *L, int q, float x, float y, float z, float m)
{
    if (paired_list<BPL>()) {
        float *b = L + 8 * (q >> 1) + (q & 1);
        b[0] = x;
        b[2] = y;
        b[4] = z;
        b[6] = m;
    } else {
        float4 *b = reinterpret_cast<float4 *>(L) + 2 * q;
        b[0] = make_float4(x, x, y, y);
        b[1] = make_float4(z, z, m, m);
    }
}

template <bool ZEPS>
__device__ __forceinline__ void pair_terms(float2 dx, float2 dy, float2 dz, float2 m, float2 e2,
                                           float2 &ax, float2 &ay, float2 &az)
{
    float2 r2 = fma2(dx, dx, e2);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    float2 ri = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
    if (ZEPS) {
        ri.x = r2.x > 0.f ? ri.x : 0.f;
        ri.y = r2.y > 0.f ? ri.y : 0.f;
    }
    const float2 s = mul2(mul2(m, ri), mul2(ri, ri));
    ax = fma2(dx, s, ax);
    ay = fma2(dy, s, ay);
    az = fma2(dz, s, az);
}

// Add the first `cnt` listed sources (cnt even for the paired layout) onto
// this lane's bodies.  Paired layout: nx = (-x_i, -x_i) per body (the second
// body's in nx2, its sums in a2); doubled layout: nx = (-x_i0, -x_i1).
template <bool ZEPS, int BPL>
__device__ __forceinline__ void list_eval(const float4 *L4, int cnt, float2 nx, float2 ny,
                                          float2 nz, float2 e2, float2 &ax, float2 &ay, float2 &az,
                                          float2 nx2, float2 ny2, float2 nz2, float2 &bx,
                                          float2 &by, float2 &bz)
{
    constexpr bool TWO = BPL == 2 && paired_list<BPL>();
    const int steps = paired_list<BPL>() ? cnt >> 1 : cnt;
#pragma unroll 4
    for (int q = 0; q < steps; ++q) {
        const float4 A = L4[2 * q], B = L4[2 * q + 1];
        const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
        const float2 sz = make_float2(B.x, B.y), sm = make_float2(B.z, B.w);
        pair_terms<ZEPS>(add2(sx, nx), add2(sy, ny), add2(sz, nz), sm, e2, ax, ay, az);
        if constexpr (TWO)
            pair_terms<ZEPS>(add2(sx, nx2), add2(sy, ny2), add2(sz, nz2), sm, e2, bx, by, bz);
    }
}

// Inclusive warp scan of v (lanes in order).
__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += u;
    }
    return v;
}

// Given inclusive prefix sums `incl` of per-lane counts (non-decreasing over
// the lanes), the lane whose span holds position pos: the number of lanes
// with incl <= pos (a binary search over the lanes, five shuffles).
__device__ __forceinline__ int warp_span_of(int incl, int pos)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
        if (v <= pos) lo += step;
    }
    return lo;
}

// One warp per group of 32 * BPL consecutive bodies in key order (BPL per
// lane: bodies base + lane and base + 32 + lane).  The warp walks the tree
// level by level, deepest level first, 32 nodes per round (one per lane).
// The opening test against every body of the group decides, per node,
// between the interaction list (accepted cell: its monopole; leaf: its
// bodies) and descending (its children, a contiguous range, go on the next
// level's stack).  The test runs in three exact stages: the group's box
// (passing it implies every body passes), then the group's first and last
// bodies (failing either rejects), then, for the nodes still undecided, every
// body.  Each level's stack holds at most 32 ranges, the children of one
// round's nodes, since a level is refilled only once every deeper level is
// empty.  Whenever FLUSH sources are listed, every lane adds them to its bodies.
template <int BPL, bool MULTI>
struct WalkShared {
    float4 list[WALK_WARPS][list_f4<BPL>()];  // float4 slots of the lists
    int2 ranges[WALK_WARPS][LEVELS][32];
    int lslot[MULTI ? 1 : WALK_WARPS][32];  // a chunk's leaf starts: body index minus position
    float crit2[MULTI ? 1 + WALK_MAX_MORE : 1][LEVELS];  // per walked tree
};

// The walk of group g (bodies [g * 32 * BPL, ...) in key order) by one warp:
// over the one tree (tq_only = -1), or (MULTI) over span tq_only of the trees
// in p.more, the group's last span then writing the sums of all of them.
template <bool ZEPS, int BPL, bool MULTI>
__device__ __forceinline__ void walk_group(const TreeWalkParams &p, WalkShared<BPL, MULTI> &sh,
                                           int g, int tq_only)
{
    constexpr int GROUP = 32 * BPL;
    constexpr int LIST_F4 = list_f4<BPL>();
    constexpr bool TWO = BPL == 2 && paired_list<BPL>();  // a lane's two bodies in turn
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = p.n;
    const int base = g * GROUP;
    if (base >= n) return;  // whole warp past the end
    const int nvalid = min(GROUP, n - base);
    float4(*list_s)[LIST_F4] = sh.list;

    bool valid[BPL];
    float4 h[BPL];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    float4 lo_[BPL];
#pragma unroll
    for (int b = 0; b < BPL; ++b) {
        const int k = base + 32 * b + lane;
        valid[b] = k < n;
        h[b] = valid[b] ? __ldg(p.P + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        lo_[b] = valid[b] ? __ldg(p.Plo + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid[b]) {
            mn[0] = fminf(mn[0], h[b].x);
            mn[1] = fminf(mn[1], h[b].y);
            mn[2] = fminf(mn[2], h[b].z);
            mx[0] = fmaxf(mx[0], h[b].x);
            mx[1] = fmaxf(mx[1], h[b].y);
            mx[2] = fmaxf(mx[2], h[b].z);
        }
    }
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
    float xi[BPL], yi[BPL], zi[BPL];
#pragma unroll
    for (int b = 0; b < BPL; ++b) {
        xi[b] = rel(h[b].x, lo_[b].x, cx);
        yi[b] = rel(h[b].y, lo_[b].y, cy);
        zi[b] = rel(h[b].z, lo_[b].z, cz);
    }
    const bool bc = BPL == 1 || TWO;  // the first body broadcast over a source pair
    const float2 nx = bc ? make_float2(-xi[0], -xi[0]) : make_float2(-xi[0], -xi[BPL - 1]);
    const float2 ny = bc ? make_float2(-yi[0], -yi[0]) : make_float2(-yi[0], -yi[BPL - 1]);
    const float2 nz = bc ? make_float2(-zi[0], -zi[0]) : make_float2(-zi[0], -zi[BPL - 1]);
    const float2 nx2 = make_float2(-xi[BPL - 1], -xi[BPL - 1]);
    const float2 ny2 = make_float2(-yi[BPL - 1], -yi[BPL - 1]);
    const float2 nz2 = make_float2(-zi[BPL - 1], -zi[BPL - 1]);
    const float2 e2 = make_float2(p.eps2f, p.eps2f);
    // the group's first and last bodies, for the quick rejection
    const int lastb = (nvalid - 1) >> 5, lastl = (nvalid - 1) & 31;
    float r0[3], r1[3];
    {
        const float4 hl = lastb == 0 ? h[0] : h[BPL - 1];
        r0[0] = __shfl_sync(FULL, h[0].x, 0);
        r0[1] = __shfl_sync(FULL, h[0].y, 0);
        r0[2] = __shfl_sync(FULL, h[0].z, 0);
        r1[0] = __shfl_sync(FULL, hl.x, lastl);
        r1[1] = __shfl_sync(FULL, hl.y, lastl);
        r1[2] = __shfl_sync(FULL, hl.z, lastl);
    }

    float *L = reinterpret_cast<float *>(list_s[warp]);
    const float4 *L4 = list_s[warp];
    int2(*rs)[32] = sh.ranges[warp];
    const unsigned lt = (1u << lane) - 1u;
    int head = 0;  // the list ring's current half (0 or FLUSH)

    // Each tree's sum per body, G (s - c) from its Kahan pair, added in tree
    // order in float64 (as separate accumulating walks would add them).
    double tg[BPL][3];
    int nc = 0, nb = 0;
    const int ntrees = MULTI ? 1 + p.nmore : 1;
    // split mode: this task walks trees [tq_only * tspan, ... + tspan)
    const int tq_lo = MULTI && tq_only >= 0 ? tq_only * p.tspan : 0;
    const int tq_hi = MULTI && tq_only >= 0 ? min(tq_lo + p.tspan, ntrees) : ntrees;
    for (int tq = tq_lo; tq < tq_hi; ++tq) {
    WalkSource t;
    if (!MULTI) {
        t = WalkSource{p.tree.box_lo, p.tree.box_hi, p.tree.chi, p.tree.clo,
                       p.tree.start,  p.tree.end,    p.sP,      p.sPlo,
                       p.box};
    } else {  // every tree of a multi-tree walk, the first included, from `more`
        t = p.more[tq];
    }
    const float *crit2 = sh.crit2[MULTI ? tq : 0];
    float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax, bx = ax, by = ax, bz = ax;
    // Kahan (sum, carry) per body and axis: the paired layout folds both
    // halves of a body's float32x2 accumulators into it (the second body's
    // are bx..bz); the doubled layout keeps .x and .y apart.
    float sx[BPL], sy[BPL], sz[BPL], qx[BPL], qy[BPL], qz[BPL];
#pragma unroll
    for (int b = 0; b < BPL; ++b) sx[b] = sy[b] = sz[b] = qx[b] = qy[b] = qz[b] = 0.f;
    auto fold = [&]() {
        if (paired_list<BPL>()) {
            kahan_add(sx[0], qx[0], ax.x);
            kahan_add(sx[0], qx[0], ax.y);
            kahan_add(sy[0], qy[0], ay.x);
            kahan_add(sy[0], qy[0], ay.y);
            kahan_add(sz[0], qz[0], az.x);
            kahan_add(sz[0], qz[0], az.y);
            if (TWO) {
                kahan_add(sx[BPL - 1], qx[BPL - 1], bx.x);
                kahan_add(sx[BPL - 1], qx[BPL - 1], bx.y);
                kahan_add(sy[BPL - 1], qy[BPL - 1], by.x);
                kahan_add(sy[BPL - 1], qy[BPL - 1], by.y);
                kahan_add(sz[BPL - 1], qz[BPL - 1], bz.x);
                kahan_add(sz[BPL - 1], qz[BPL - 1], bz.y);
            }
        } else {
            kahan_add(sx[0], qx[0], ax.x);
            kahan_add(sy[0], qy[0], ay.x);
            kahan_add(sz[0], qz[0], az.x);
            kahan_add(sx[BPL - 1], qx[BPL - 1], ax.y);
            kahan_add(sy[BPL - 1], qy[BPL - 1], ay.y);
            kahan_add(sz[BPL - 1], qz[BPL - 1], az.y);
        }
        ax = ay = az = bx = by = bz = make_float2(0.f, 0.f);
    };
    int cnt = 0;  // listed sources (warp-uniform)
    int nflush = 0;
    // FLUSH sources listed from the head on: add them, head to the other half
    auto flush = [&]() {
        __syncwarp();
        list_eval<ZEPS, BPL>(L4 + (paired_list<BPL>() ? head : 2 * head), FLUSH, nx, ny, nz, e2,
                             ax, ay, az, nx2, ny2, nz2, bx, by, bz);
        if (++nflush % NB_WALK_FOLD_EVERY == 0) fold();
        head ^= FLUSH;
        cnt -= FLUSH;
        __syncwarp();
    };

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
        const int incl = warp_incl_scan(r.y, lane);
        const int excl = incl - r.y;
        const int take = min(__shfl_sync(FULL, incl, 31), 32);
        // the range holding this lane's node: the last range starting at or
        // before it (ranges 0..R-1 are non-empty, so their starts increase)
        const unsigned starts = __reduce_or_sync(FULL, lane < R && excl < 32 ? 1u << excl : 0u);
        const int src = __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
        const int first_src = __shfl_sync(FULL, r.x, src), excl_src = __shfl_sync(FULL, excl, src);
        const int node = lane < take ? first_src + (lane - excl_src) : -1;
        const unsigned done = __ballot_sync(FULL, lane < R && incl <= 32);
        if (lane < R && excl < 32 && incl > 32)
            rs[Lv][size - 1 - lane] = make_int2(r.x + (32 - excl), incl - 32);
        if (lane == Lv) lsize -= __popc(done);
        __syncwarp();

        // opening test
        const bool has = node >= 0;
        float4 blo = make_float4(0.f, 0.f, 0.f, 0.f), bhi = blo;
        if (has) {
            blo = __ldg(t.box_lo + node);
            bhi = __ldg(t.box_hi + node);
        }
        const float cr = crit2[Lv];
        bool accept = has && cube_box_dist2(blo, bhi, mn, mx) >= cr;
        unsigned und = __ballot_sync(FULL, has && !accept);
        if (und) {
            const bool rej = cube_dist2(blo, bhi, r0[0], r0[1], r0[2]) < cr ||
                             cube_dist2(blo, bhi, r1[0], r1[1], r1[2]) < cr;
            und = __ballot_sync(FULL, has && !accept && !rej);
        }
        // undecided nodes one at a time, every lane testing its own bodies
        while (und) {
            const int j = __ffs(und) - 1;
            und &= und - 1;
            const float4 jlo = make_float4(__shfl_sync(FULL, blo.x, j), __shfl_sync(FULL, blo.y, j),
                                           __shfl_sync(FULL, blo.z, j), 0.f);
            const float4 jhi = make_float4(__shfl_sync(FULL, bhi.x, j), __shfl_sync(FULL, bhi.y, j),
                                           __shfl_sync(FULL, bhi.z, j), 0.f);
            bool ok = true;
#pragma unroll
            for (int b = 0; b < BPL; ++b)
                ok = ok && (!valid[b] || cube_dist2(jlo, jhi, h[b].x, h[b].y, h[b].z) >= cr);
            const bool all = __all_sync(FULL, ok);
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
                list_put<BPL>(L, (head + cnt + __popc(am & lt)) & (LIST_CAP - 1),
                              rel(ch.x, cl.x, cx), rel(ch.y, cl.y, cy), rel(ch.z, cl.z, cz), ch.w);
            }
            cnt += __popc(am);
            nc += __popc(am);
            if (cnt >= FLUSH) flush();
        }
        // leaves: the bodies of all of this round's leaves, 32 list slots at a
        // time (lane l of a chunk fetches the chunk's l-th body)
        if (__ballot_sync(FULL, leaf)) {
            int ls = 0, lsz = 0;
            if (leaf) {
                ls = t.start[node];
                lsz = t.end[node] - ls;
            }
            const int linc = warp_incl_scan(lsz, lane);
            const int lexc = linc - lsz;
            const int T = __shfl_sync(FULL, linc, 31);
            nb += T;
            int carry = 0;  // the offset of the leaf running into the chunk
            for (int c0 = 0; c0 < T; c0 += 32) {
                const int pos = c0 + lane;
                int body;
                if constexpr (MULTI) {  // (the slots cost this instance spills)
                    const int j = warp_span_of(linc, pos);
                    body = __shfl_sync(FULL, ls, j & 31) + (pos - __shfl_sync(FULL, lexc, j & 31));
                } else {
                    // the leaf holding position pos: the last one starting at
                    // or before it, in this chunk (its slot) or earlier (carry)
                    const bool st = lsz > 0 && lexc >= c0 && lexc < c0 + 32;
                    if (st) sh.lslot[warp][lexc - c0] = ls - lexc;
                    const unsigned S = __reduce_or_sync(FULL, st ? 1u << (lexc - c0) : 0u);
                    __syncwarp();
                    const unsigned below = S & (0xffffffffu >> (31 - lane));
                    const int off = below ? sh.lslot[warp][31 - __clz(below)] : carry;
                    carry = __shfl_sync(FULL, off, 31);
                    body = off + pos;
                }
                const int kk = min(32, T - c0);
                if (lane < kk) {
                    const float4 bh = __ldg(t.sP + body), bl = __ldg(t.sPlo + body);
                    list_put<BPL>(L, (head + cnt + lane) & (LIST_CAP - 1), rel(bh.x, bl.x, cx),
                                  rel(bh.y, bl.y, cy), rel(bh.z, bl.z, cz), bh.w);
                }
                cnt += kk;
                if (cnt >= FLUSH) flush();
                __syncwarp();  // the slots are rewritten for the next chunk
            }
        }
    }
    if (cnt > 0) {  // the rest, within the head's half (paired layout: padded to a
                    // pair with a massless source)
        if (paired_list<BPL>() && lane == 0 && (cnt & 1))
            list_put<BPL>(L, head + cnt, 0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        list_eval<ZEPS, BPL>(L4 + (paired_list<BPL>() ? head : 2 * head),
                             paired_list<BPL>() ? (cnt + 1) & ~1 : cnt, nx, ny, nz, e2, ax, ay,
                             az, nx2, ny2, nz2, bx, by, bz);
    }
    if (nflush % NB_WALK_FOLD_EVERY != 0 || cnt > 0) fold();
    __syncwarp();  // the next tree reuses this warp's list and stacks
#pragma unroll
    for (int b = 0; b < BPL; ++b) {
        const double d[3] = {p.G * ((double)sx[b] - (double)qx[b]),
                             p.G * ((double)sy[b] - (double)qy[b]),
                             p.G * ((double)sz[b] - (double)qz[b])};
#pragma unroll
        for (int c = 0; c < 3; ++c) tg[b][c] = (!MULTI || tq == tq_lo) ? d[c] : __dadd_rn(tg[b][c], d[c]);
    }
    }  // trees
    bool stats_done = false;
    if (MULTI && tq_only >= 0) {
        // this task's sums and counts; the group's last task adds all tasks'
        // in tree order (with one tree per task, as the walk over every tree
        // in turn does) and writes
        const int ngroups = (n + GROUP - 1) / GROUP;
        const size_t npad = (size_t)ngroups * GROUP;
#pragma unroll
        for (int b = 0; b < BPL; ++b) {
            double *q = p.tpart + ((size_t)tq_only * npad + base + 32 * b + lane) * 3;
            q[0] = tg[b][0];
            q[1] = tg[b][1];
            q[2] = tg[b][2];
        }
        if (lane == 0) {
            p.tcnt[((size_t)tq_only * ngroups + g) * 2] = nc;
            p.tcnt[((size_t)tq_only * ngroups + g) * 2 + 1] = nb;
            atomicAdd(p.tree.stats + 2, (unsigned long long)nc * nvalid);
            atomicAdd(p.tree.stats + 3, (unsigned long long)nb * nvalid);
        }
        stats_done = true;
        __threadfence();
        __syncwarp();
        unsigned last = 0;
        const int nspans = (ntrees + p.tspan - 1) / p.tspan;
        if (lane == 0) last = atomicAdd(p.tctr + g, 1u) == (unsigned)(nspans - 1);
        if (!__shfl_sync(FULL, last, 0)) return;
        __threadfence();
        nc = nb = 0;
        for (int tq = 0; tq < nspans; ++tq) {
#pragma unroll
            for (int b = 0; b < BPL; ++b) {
                const double *q = p.tpart + ((size_t)tq * npad + base + 32 * b + lane) * 3;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    tg[b][c] = tq == 0 ? __ldcg(q + c) : __dadd_rn(tg[b][c], __ldcg(q + c));
            }
            nc += __ldcg(p.tcnt + ((size_t)tq * ngroups + g) * 2);
            nb += __ldcg(p.tcnt + ((size_t)tq * ngroups + g) * 2 + 1);
        }
        if (lane == 0) p.tctr[g] = 0u;  // every task of the group has arrived
    }
#pragma unroll
    for (int b = 0; b < BPL; ++b) {
        if (!valid[b]) continue;
        const int i = p.perm[base + 32 * b + lane];
        const double gx = tg[b][0], gy = tg[b][1], gz = tg[b][2];
        double *a = p.acc + 3 * (size_t)i;
        if (p.accumulate) {  // a further tree's share (a received LET)
            a[0] += gx;
            a[1] += gy;
            a[2] += gz;
            if (p.counts) {
                p.counts[2 * (size_t)i] += nc;
                p.counts[2 * (size_t)i + 1] += nb;
            }
        } else {
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
        }
        if (!finite3(gx, gy, gz)) atomicOr(p.err, ERR_NONFINITE);
    }
    if (lane == 0 && !stats_done) {  // nc, nb are the same for the group's nvalid bodies
        atomicAdd(p.tree.stats + 2, (unsigned long long)nc * nvalid);
        atomicAdd(p.tree.stats + 3, (unsigned long long)nb * nvalid);
    }
    __syncwarp();  // the next group reuses this warp's lists and stacks
}

// Scheduling of the groups over the warps (the paper's OpenMP loop
// schedules, Sec. II, applied to the walk): static, one group per warp of a
// grid covering all groups; dynamic, a grid of resident warps taking `chunk`
// groups at a time from an atomic counter; guided, the same with chunks of
// max(chunk, remaining / (2 x warps)).
template <bool ZEPS, int BPL, bool MULTI>
__global__ void __launch_bounds__(32 * WALK_WARPS, BPL == 1 ? NB_WALK_MINB1 : NB_WALK_MINB2)
    tree_walk_kernel(const TreeWalkParams p)
{
    __shared__ WalkShared<BPL, MULTI> sh;
    for (int q = threadIdx.x; q < (MULTI ? 1 + p.nmore : 1) * LEVELS; q += blockDim.x) {
        const int tq = q / LEVELS, L = q % LEVELS;
        sh.crit2[tq][L] = open_dist2(MULTI ? p.more[tq].box[3] : p.box[3], L, p.theta);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * WALK_WARPS + warp;
    const int ngroups = (p.n + 32 * BPL - 1) / (32 * BPL);
    // tasks: the groups, or with further trees (split mode) the (group,
    // tree) pairs, tree-major
    const int ntasks = MULTI ? ngroups * ((1 + p.nmore + p.tspan - 1) / p.tspan) : ngroups;
    auto task = [&](int t) {
        if constexpr (MULTI)
            walk_group<ZEPS, BPL, MULTI>(p, sh, t % ngroups, t / ngroups);
        else
            walk_group<ZEPS, BPL, MULTI>(p, sh, t, -1);
    };
    if (p.sched == 0) {
        if (gw < ntasks) task(gw);
        return;
    }
    const int nwarps = gridDim.x * WALK_WARPS;
    int *queue = p.queue;
    int seen = 0;
    for (;;) {
        int c = p.chunk;
        if (p.sched == 2) c = max(c, (ntasks - seen) / (2 * nwarps));
        int g0 = 0;
        if (lane == 0) g0 = atomicAdd(queue, c);
        g0 = __shfl_sync(0xffffffffu, g0, 0);
        if (g0 >= ntasks) break;
        seen = g0 + c;
        const int g1 = min(g0 + c, ntasks);
        for (int g = g0; g < g1; ++g) task(g);
    }
}

// ---------------------------------------------- locally essential trees
// The LET of this tree for a destination whose bodies lie in the float32
// box [dlo, dhi] (paper Sec. IV-B, the influence-ring test from the
// destination's side): the root is sent; a sent node whose cube is distant
// enough from the box (cube_box_dist2, the walk's own first-stage test, so
// every body inside the box accepts it) is sent alone; otherwise a sent
// leaf goes with its bodies and a sent cell with all its children.
// Level by level, parents first.
__global__ void __launch_bounds__(TTPB) let_kind_kernel(TreeView t, const double *__restrict__ box,
                                                        float theta, float3 dlo, float3 dhi, int L,
                                                        int *__restrict__ kind)
{
    const int cnt = t.meta[META_COUNT + L], base = t.meta[META_BASE + L];
    const float crit2 = open_dist2(box[3], L, theta);
    const float mn[3] = {dlo.x, dlo.y, dlo.z}, mx[3] = {dhi.x, dhi.y, dhi.z};
    for (int q = blockIdx.x * TTPB + threadIdx.x; q < cnt; q += gridDim.x * TTPB) {
        const int u = base + q;
        int k = 0;
        if (L == 0 || kind[t.parent[u]] == 2) {
            if (cube_box_dist2(t.box_lo[u], t.box_hi[u], mn, mx) >= crit2)
                k = 1;
            else
                k = t.nchild[u] == 0 ? 3 : 2;
        }
        kind[u] = k;
    }
}

// One block: each sent node's index in the LET and each sent leaf's first
// body there (exclusive scans in node order); totals = {nodes, bodies}.
__global__ void __launch_bounds__(1024) let_scan_kernel(TreeView t, LetScratch sc)
{
    __shared__ int tile[BSCAN_TILE + BSCAN_TILE / 32];
    __shared__ int wsum[32];
    const int total = t.meta[META_BASE + 10] + t.meta[META_COUNT + 10];
    // flags and body counts first go into the output arrays, scanned in place
    for (int u = threadIdx.x; u < total; u += 1024) {
        const int k = sc.kind[u];
        sc.nidx[u] = k != 0;
        sc.boff[u] = k == 3 ? t.end[u] - t.start[u] : 0;
    }
    __syncthreads();
    const int nn = block_scan_exclusive<int>(sc.nidx, sc.nidx, total, tile, wsum);
    const int nb = block_scan_exclusive<int>(sc.boff, sc.boff, total, tile, wsum);
    if (threadIdx.x == 0) {
        sc.totals[0] = nn;
        sc.totals[1] = nb;
    }
}

__global__ void __launch_bounds__(TTPB) let_emit_kernel(TreeView t, const double *__restrict__ box,
                                                        LetScratch sc, const float4 *__restrict__ P,
                                                        const float4 *__restrict__ Plo,
                                                        unsigned char *__restrict__ out)
{
    const int total = t.meta[META_BASE + 10] + t.meta[META_COUNT + 10];
    const long long nn = sc.totals[0], nb = sc.totals[1];
    const LetLayout lay = let_layout(nn, nb);
    float4 *lo = reinterpret_cast<float4 *>(out + lay.lo);
    float4 *hi = reinterpret_cast<float4 *>(out + lay.hi);
    float4 *chi = reinterpret_cast<float4 *>(out + lay.chi);
    float4 *clo = reinterpret_cast<float4 *>(out + lay.clo);
    int *st = reinterpret_cast<int *>(out + lay.start);
    int *en = reinterpret_cast<int *>(out + lay.end);
    float4 *bP = reinterpret_cast<float4 *>(out + lay.P);
    float4 *bPlo = reinterpret_cast<float4 *>(out + lay.Plo);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        LetHeader h;
        h.magic = LET_MAGIC;
        h.n_nodes = nn;
        h.n_bodies = nb;
        h.reserved = 0;
        for (int c = 0; c < 4; ++c) h.box[c] = box[c];
        *reinterpret_cast<LetHeader *>(out) = h;
    }
    for (int u = blockIdx.x * TTPB + threadIdx.x; u < total; u += gridDim.x * TTPB) {
        const int k = sc.kind[u];
        if (k == 0) continue;
        const int v = sc.nidx[u];
        float4 a = t.box_lo[u], b = t.box_hi[u];
        // children are kept only for an opened cell; they are consecutive
        // in both trees, so the first one's LET index locates them all
        a.w = __int_as_float(k == 2 ? t.nchild[u] : 0);
        b.w = __int_as_float(k == 2 ? sc.nidx[t.first[u]] : -1);
        lo[v] = a;
        hi[v] = b;
        chi[v] = t.chi[u];
        clo[v] = t.clo[u];
        const int b0 = sc.boff[u];
        const int len = k == 3 ? t.end[u] - t.start[u] : 0;
        st[v] = b0;
        en[v] = b0 + len;
        for (int q = 0; q < len; ++q) {
            bP[b0 + q] = P[t.start[u] + q];
            bPlo[b0 + q] = Plo[t.start[u] + q];
        }
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
    tree_init_kernel<<<1, 32, 0, s>>>(t, n, box);
    ++kernels;
    const int g = grid_cap(n);
    for (int L = 0; L < 10; ++L) {
        tree_count_kernel<<<g, TTPB, 0, s>>>(t, keys, L, leaf_cap);
        tree_scan_kernel<<<1, 1024, 0, s>>>(t, L);
        tree_emit_kernel<<<g, TTPB, 0, s>>>(t, keys, box, L);
        kernels += 3;
    }
    tree_moments_kernel<<<grid_cap(t.cap), TTPB, 0, s>>>(t, pos, mass, perm);
    tree_flag_kernel<<<1, 32, 0, s>>>(t, err);
    kernels += 2;
    return cudaGetLastError();
}

cudaError_t launch_let_select(cudaStream_t s, const TreeView &t, const double *box, float theta,
                              float3 dlo, float3 dhi, const LetScratch &sc, int &kernels)
{
    kernels = 0;
    const int g = grid_cap(t.cap);
    for (int L = 0; L < LEVELS; ++L) {
        let_kind_kernel<<<g, TTPB, 0, s>>>(t, box, theta, dlo, dhi, L, sc.kind);
        ++kernels;
    }
    let_scan_kernel<<<1, 1024, 0, s>>>(t, sc);
    ++kernels;
    return cudaGetLastError();
}

cudaError_t launch_let_emit(cudaStream_t s, const TreeView &t, const double *box,
                            const LetScratch &sc, const float4 *P, const float4 *Plo, void *out,
                            int &kernels)
{
    let_emit_kernel<<<grid_cap(t.cap), TTPB, 0, s>>>(t, box, sc, P, Plo,
                                                     static_cast<unsigned char *>(out));
    kernels = 1;
    return cudaGetLastError();
}

cudaError_t launch_tree_walk(cudaStream_t s, const TreeWalkParams &p, bool zeps, int &kernels)
{
    kernels = 0;
    if (p.n <= 0) return cudaSuccess;
    const int G = p.group;
    if (p.nmore > 0 && (!p.tpart || !p.tcnt || !p.tctr || p.tspan < 1))
        return cudaErrorInvalidValue;
    const int groups =  // tasks
        (p.n + G - 1) / G * (p.nmore > 0 ? (1 + p.nmore + p.tspan - 1) / p.tspan : 1);
    // (a separate instance walks further trees: the single-tree walk keeps
    // its own registers and shared memory)
    void (*fn)(const TreeWalkParams) =
        p.nmore > 0
            ? (G == 32 ? (zeps ? tree_walk_kernel<true, 1, true> : tree_walk_kernel<false, 1, true>)
                       : (zeps ? tree_walk_kernel<true, 2, true> : tree_walk_kernel<false, 2, true>))
            : (G == 32 ? (zeps ? tree_walk_kernel<true, 1, false> : tree_walk_kernel<false, 1, false>)
                       : (zeps ? tree_walk_kernel<true, 2, false> : tree_walk_kernel<false, 2, false>));
    int blocks = (groups + WALK_WARPS - 1) / WALK_WARPS;
    if (p.sched != 0) {  // resident blocks only
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * WALK_WARPS, 0);
        if (e != cudaSuccess) return e;
        blocks = min(blocks, max(per_sm, 1) * p.num_sms);
    }
    fn<<<blocks, 32 * WALK_WARPS, 0, s>>>(p);
    kernels = 1;
    return cudaGetLastError();
}

}  // namespace nb
