// Fast multipole method on the GPU: the O(N) method the paper names as the
// successor of its tree code (Sec. VI, after Greengard and Rokhlin).  The
// paper gives no formulation; the readings (shared with the oracle, which
// computes the same sums by their definitions) are:
//  * the tree is the Barnes-Hut tree of tree.cu (same cube, keys, leaves);
//  * each cell carries a Cartesian Taylor expansion of order p about its
//    cube's centre z, for the softened kernel g(r) = (|r|^2 + eps^2)^-1/2;
//  * target A and source B are well separated when
//    |z_A - z_B| >= (r_A + r_B) / theta, r = sqrt(3)/2 edge; in units of
//    h = ext / 2048 the centres are integers, so the test is exact: the
//    integer D2 against 0.75 (e_A + e_B)^2 / theta^2 in float64;
//  * the pairs come from the dual-tree traversal from (root, root): each
//    target takes the candidates its parent handed down; separated -> B's
//    expansion acts on A; both leaves -> direct sum; A a leaf -> B's
//    children; B a leaf or smaller -> B to A's children; else B's children
//    to A's children.
//
// Scaled expansions (all factors exact powers of two, so float32 holds any
// system size; e = cell edge, v = (x - z) / e):
//   moments  Mc_n = sum_j m_j (-v_j)^n / n!
//   locals   Lc_k = e_A^|k| d^k Phi(z_A)   (Phi = sum of the sources' potentials)
//   P2M  from the bodies (positions read in float64, v rounded once);
//   M2M  Mc^P_n = sum_{k<=n} (-s/4)^(n-k)/(n-k)! 2^-|k| Mc^c_k, s = child octant signs;
//   M2L  with rho = h 2^E, E = floor(log2 |c_A - c_B|), q = (c_A - c_B)/2^E
//        (exact, 1 <= |q| < 2), T'_m = d^m g'(q) for eps' = eps / rho,
//        U_m = (e_A/rho)^|m| T'_m / rho:
//        Lc_k += sum_{|n| <= p-|k|} Mc^B_n 2^((L_A - L_B)|n|) U_{n+k};
//   L2L  Lc^c_k = sum_{n>=k} Lc^P_n 2^-|n| (s/2)^(n-k)/(n-k)!;
//   L2P  a = (G/e_A) sum_{|k|<=p-1} Lc_{k+e_c} v^k/k!.
// The derivatives use g = f(|r|^2/2), f^(m) = (-1)^m (2m-1)!! s^-(2m+1) and
// d^n f_m = q_c d^(n-e_c) f_(m+1) + (n_c - 1) d^(n-2e_c) f_(m+1).
//
// Launches: the upward pass (P2M at the leaves in one launch, then M2M one
// launch per level from the deepest up); one list launch per level over the
// non-leaf cells (the candidates' classification, the hand-down lists and
// each cell's list of separated sources), then one over all leaves (each
// walks its candidates' subtrees for its list); one M2L launch over all
// cells (one source per lane); one L2L launch per level below the root; and
// one near-field launch over the leaves (the same walk collecting the
// leaves to sum directly, float32x2 pair terms over sliced lanes, then L2P).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace fmm {

constexpr unsigned FULL = 0xffffffffu;
constexpr int LEVELS = 11;
constexpr int WARPS = 4;  // warps per block of the downward and near-field kernels
constexpr int FLUSH = 256;  // directly summed sources per flush (128 pairs)

// ------------------------------------------------------------ multi-indices
// Slots in graded order: orders below k first, then a descending, b descending.
__host__ __device__ constexpr int nterms(int p) { return p < 0 ? 0 : (p + 1) * (p + 2) * (p + 3) / 6; }
__host__ __device__ constexpr int slot_of(int a, int b, int c)
{
    return nterms(a + b + c - 1) + (b + c) * (b + c + 1) / 2 + c;
}
__host__ __device__ constexpr int ord_of(int q)
{
    int k = 0;
    while (nterms(k) <= q) ++k;
    return k;
}
__host__ __device__ constexpr int mi_of(int q, int axis)
{
    const int k = ord_of(q), r = q - nterms(k - 1);
    int s = 0;
    while ((s + 1) * (s + 2) / 2 <= r) ++s;
    const int c = r - s * (s + 1) / 2, b = s - c, a = k - s;
    return axis == 0 ? a : (axis == 1 ? b : c);
}
__host__ __device__ constexpr double fact(int a) { return a <= 1 ? 1.0 : a * fact(a - 1); }
__host__ __device__ constexpr float inv_fact3(int q)
{
    return (float)(1.0 / (fact(mi_of(q, 0)) * fact(mi_of(q, 1)) * fact(mi_of(q, 2))));
}
__host__ __device__ constexpr int padded(int p) { return (nterms(p) + 3) & ~3; }

template <int I, int E, class F>
__device__ __forceinline__ void sfor(F &&f)
{
    if constexpr (I < E) {
        f(std::integral_constant<int, I>());
        sfor<I + 1, E>(f);
    }
}

// 2^e for -126 <= e <= 127, exactly.
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// ------------------------------------------------------------ kernel parts
// T[q] = c0 sc^|n| d^n g'(q) for the slots of order <= P,
// g' = (|q|^2 + e2)^-1/2, sc a power of two.  The factors ride on the
// recursion: with W'[m][n] = c0 sc^|n| d^n f_m it reads
// W'[m][n] = (sc q_c) W'[m+1][n-e_c] + (n_c - 1) sc^2 W'[m+1][n-2e_c]
// from the seeds W'[m][0] = c0 f^(m).
template <int P>
__device__ __forceinline__ void derivs(float qx, float qy, float qz, float e2, float sc, float c0,
                                       float (&T)[nterms(P)])
{
    constexpr int N = nterms(P);
    float W[P + 1][N];  // W[m][slot] = c0 sc^|n| d^n f_m, only m + |n| <= P
    const float s2 = fmaf(qz, qz, fmaf(qy, qy, fmaf(qx, qx, e2)));
    const float is = rsqrt_mufu(s2);
    const float is2 = is * is;
    const float sx = sc * qx, sy = sc * qy, sz = sc * qz, sc2 = sc * sc;
    W[0][0] = is * c0;
    sfor<1, P + 1>([&](auto mI) {
        constexpr int m = decltype(mI)::value;
        W[m][0] = -(float)(2 * m - 1) * W[m - 1][0] * is2;
    });
    sfor<1, N>([&](auto qI) {
        constexpr int q = decltype(qI)::value;
        constexpr int a = mi_of(q, 0), b = mi_of(q, 1), c = mi_of(q, 2), k = a + b + c;
        constexpr int ax = a > 0 ? 0 : (b > 0 ? 1 : 2);
        constexpr int na = ax == 0 ? a : (ax == 1 ? b : c);
        constexpr int q1 = slot_of(a - (ax == 0), b - (ax == 1), c - (ax == 2));
        constexpr int q2 =
            na >= 2 ? slot_of(a - 2 * (ax == 0), b - 2 * (ax == 1), c - 2 * (ax == 2)) : -1;
        const float r = ax == 0 ? sx : (ax == 1 ? sy : sz);
        sfor<0, P - k + 1>([&](auto mI) {
            constexpr int m = decltype(mI)::value;
            float v = r * W[m + 1][q1];
            if constexpr (q2 >= 0) v = fmaf((float)(na - 1) * sc2, W[m + 1][q2], v);
            W[m][q] = v;
        });
    });
    sfor<0, N>([&](auto qI) {
        constexpr int q = decltype(qI)::value;
        T[q] = W[0][q];
    });
}

struct Consts {
    float inv_h;     // 2048 / ext
    float eps2_h;    // eps^2 (2048 / ext)^2
};

// acc += the scaled local expansion about A of source cell B's moments Mb.
template <int P>
__device__ __forceinline__ void m2l_add(float (&acc)[nterms(P)], const float *__restrict__ Mb,
                                        int4 cA, int4 cB, const Consts &K)
{
    constexpr int N = nterms(P);
    const int dx = cA.x - cB.x, dy = cA.y - cB.y, dz = cA.z - cB.z;
    const int D2 = dx * dx + dy * dy + dz * dz;  // >= 1 for distinct cells
    const int E = (31 - __clz(D2)) >> 1;         // floor(log2 sqrt(D2))
    const float sc = pow2f(-E);
    // U_m = sA^|m| T'_m / rho, sA = e_A / rho = 2^(11 - L_A - E), 1/rho = inv_h sc
    const float sA = pow2f(11 - cA.w - E);
    float T[N];
    derivs<P>((float)dx * sc, (float)dy * sc, (float)dz * sc, K.eps2_h * sc * sc, sA, K.inv_h * sc, T);
    const float g = pow2f(cA.w - cB.w);
    float pg[P + 1];
    pg[0] = 1.0f;
#pragma unroll
    for (int j = 1; j <= P; ++j) pg[j] = pg[j - 1] * g;
    const float4 *Mb4 = reinterpret_cast<const float4 *>(Mb);
    sfor<0, (N + 3) / 4>([&](auto n4I) {
        constexpr int n4 = decltype(n4I)::value;
        const float4 mv = __ldg(Mb4 + n4);
        const float mm[4] = {mv.x, mv.y, mv.z, mv.w};
        sfor<0, 4>([&](auto jI) {
            constexpr int j = decltype(jI)::value;
            constexpr int n = 4 * n4 + j;
            if constexpr (n < N) {
                constexpr int na = mi_of(n, 0), nb = mi_of(n, 1), nc = mi_of(n, 2);
                constexpr int kmax = P - (na + nb + nc);
                const float w = mm[j] * pg[na + nb + nc];
                sfor<0, nterms(kmax)>([&](auto kI) {
                    constexpr int k = decltype(kI)::value;
                    constexpr int m = slot_of(na + mi_of(k, 0), nb + mi_of(k, 1), nc + mi_of(k, 2));
                    acc[k] = fmaf(w, T[m], acc[k]);
                });
            }
        });
    });
}

// out += the child's share of its parent's local coefficients Lp (L2L), or
// (MOMENTS) out += the parent's share of the child's moments (M2M): both
// sum_{k <= n} t(n - k) x_k with per-axis factors t_c(j) = (s_c d)^j / j!,
// d = 1/2 (L2L, x = 2^-|n| Lp_n, into slot k) or d = -1/4 (M2M, x = 2^-|k|
// Mc_k, into slot n).
template <int P, bool MOMENTS>
__device__ __forceinline__ void translate_add(float (&out)[nterms(P)], const float *__restrict__ x,
                                              int octant)
{
    constexpr int N = nterms(P);
    float t[3][P + 1];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float st = ((octant >> c) & 1) ? 1.0f : -1.0f;
        const float d = MOMENTS ? -0.25f * st : 0.5f * st;
        t[c][0] = 1.0f;
#pragma unroll
        for (int j = 1; j <= P; ++j) t[c][j] = t[c][j - 1] * d / (float)j;
    }
    float xs[N];
    sfor<0, N>([&](auto qI) {
        constexpr int q = decltype(qI)::value;
        xs[q] = x[q] * pow2f(-(mi_of(q, 0) + mi_of(q, 1) + mi_of(q, 2)));
    });
    // pairs (hi, lo) with lo <= hi componentwise
    sfor<0, N>([&](auto hI) {
        constexpr int hq = decltype(hI)::value;
        constexpr int ha = mi_of(hq, 0), hb = mi_of(hq, 1), hc = mi_of(hq, 2);
        sfor<0, nterms(ha + hb + hc)>([&](auto lI) {
            constexpr int lq = decltype(lI)::value;
            constexpr int la = mi_of(lq, 0), lb = mi_of(lq, 1), lc = mi_of(lq, 2);
            if constexpr (la <= ha && lb <= hb && lc <= hc) {
                const float coef = t[0][ha - la] * t[1][hb - lb] * t[2][hc - lc];
                if constexpr (MOMENTS)
                    out[hq] = fmaf(coef, xs[lq], out[hq]);
                else
                    out[lq] = fmaf(coef, xs[hq], out[lq]);
            }
        });
    });
}

// Powers v^j / j! of one coordinate, j <= P.
template <int P>
__device__ __forceinline__ void scaled_powers(float v, float (&pw)[P + 1])
{
    pw[0] = 1.0f;
#pragma unroll
    for (int j = 1; j <= P; ++j) pw[j] = pw[j - 1] * v / (float)j;
}

// Double centre of a node from its integer centre.
__device__ __forceinline__ void centre_of(const double *box, int4 ci, double (&z)[3])
{
    const double h = __dmul_rn(box[3], 0x1p-11);
    z[0] = __dadd_rn(box[0], __dmul_rn((double)ci.x, h));
    z[1] = __dadd_rn(box[1], __dmul_rn((double)ci.y, h));
    z[2] = __dadd_rn(box[2], __dmul_rn((double)ci.z, h));
}

// Integer centre and level of a node from its key prefix.
__device__ __forceinline__ int4 icentre(unsigned prefix, int L)
{
    unsigned ic[3] = {0u, 0u, 0u};
    for (int b = 0; b < L; ++b) {
        const unsigned trip = (prefix >> (3 * b)) & 7u;
#pragma unroll
        for (int c = 0; c < 3; ++c) ic[c] |= ((trip >> c) & 1u) << b;
    }
    return make_int4((int)((2u * ic[0] + 1u) << (10 - L)), (int)((2u * ic[1] + 1u) << (10 - L)),
                     (int)((2u * ic[2] + 1u) << (10 - L)), L);
}

template <int P>
__device__ __forceinline__ void store_exp(float *dst, const float (&v)[nterms(P)])
{
    constexpr int N = nterms(P), NP = padded(P);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    sfor<0, NP / 4>([&](auto iI) {
        constexpr int i = decltype(iI)::value;
        float e[4];
        sfor<0, 4>([&](auto jI) {
            constexpr int j = decltype(jI)::value;
            constexpr int q = 4 * i + j;
            if constexpr (q < N)
                e[j] = v[q];
            else
                e[j] = 0.0f;
        });
        d4[i] = make_float4(e[0], e[1], e[2], e[3]);
    });
}

// ------------------------------------------------------------ upward pass
// P2M: a thread per leaf forms its moments from its bodies (the next body's
// position loaded while this one's monomials are added).  M2M: one launch
// per level from the deepest up, a warp per cell with children: a child per
// lane translates the child's moments, and the lanes' terms are totalled in
// a fixed order.
constexpr int UP_WARPS = 4;

template <int P>
__global__ void __launch_bounds__(32 * UP_WARPS) fmm_p2m_kernel(const FmmParams p)
{
    constexpr int N = nterms(P), NP = padded(P);
    const TreeView &t = p.tree;
    const FmmView &f = p.f;
    const int total = t.meta[TREE_META_BASE + 10] + t.meta[TREE_META_COUNT + 10];
    const double ext = p.box[3];
    for (int leaf = blockIdx.x * blockDim.x + threadIdx.x; leaf < total;
         leaf += gridDim.x * blockDim.x) {
        if (t.nchild[leaf] != 0) continue;
        const int L = t.level[leaf];
        const int4 ci = icentre(t.prefix[leaf], L);
        const int k0 = t.start[leaf], k1 = t.end[leaf];
        f.ci[leaf] = ci;
        f.nd[leaf] = make_int4(0, t.first[leaf], k0, k1);
        double z[3];
        centre_of(p.box, ci, z);
        const double inv_e = (double)(1 << L) / ext;
        float Mc[N];
#pragma unroll
        for (int q = 0; q < N; ++q) Mc[q] = 0.0f;
        double x[3] = {0.0, 0.0, 0.0}, mj = 0.0;
        if (k0 < k1) {
            const int j = p.perm[k0];
            x[0] = p.pos[3 * (size_t)j];
            x[1] = p.pos[3 * (size_t)j + 1];
            x[2] = p.pos[3 * (size_t)j + 2];
            mj = p.mass[j];
        }
        for (int k = k0; k < k1; ++k) {
            const float m = (float)mj;
            float pw[3][P + 1];
#pragma unroll
            for (int c = 0; c < 3; ++c) scaled_powers<P>((float)((z[c] - x[c]) * inv_e), pw[c]);
            if (k + 1 < k1) {
                const int j = p.perm[k + 1];
                x[0] = p.pos[3 * (size_t)j];
                x[1] = p.pos[3 * (size_t)j + 1];
                x[2] = p.pos[3 * (size_t)j + 2];
                mj = p.mass[j];
            }
            sfor<0, N>([&](auto qI) {
                constexpr int q = decltype(qI)::value;
                Mc[q] = fmaf(m * pw[0][mi_of(q, 0)], pw[1][mi_of(q, 1)] * pw[2][mi_of(q, 2)], Mc[q]);
            });
        }
        store_exp<P>(f.M + (size_t)leaf * NP, Mc);
    }
}

template <int P>
__global__ void __launch_bounds__(32 * UP_WARPS) fmm_m2m_kernel(const FmmParams p, int L)
{
    constexpr int N = nterms(P), NP = padded(P);
    const TreeView &t = p.tree;
    const FmmView &f = p.f;
    const int lane = threadIdx.x & 31;
    const int cnt = t.meta[TREE_META_COUNT + L], base = t.meta[TREE_META_BASE + L];
    for (int q0 = blockIdx.x * UP_WARPS + (threadIdx.x >> 5); q0 < cnt; q0 += gridDim.x * UP_WARPS) {
        const int node = base + q0;
        const int nch = t.nchild[node];
        if (nch == 0) continue;
        const int c0 = t.first[node];
        float Mc[N];
#pragma unroll
        for (int q = 0; q < N; ++q) Mc[q] = 0.0f;
        if (lane < nch) {
            float xc[N];
            const float *src = f.M + (size_t)(c0 + lane) * NP;
#pragma unroll
            for (int q = 0; q < N; ++q) xc[q] = src[q];
            translate_add<P, true>(Mc, xc, (int)(t.prefix[c0 + lane] & 7u));
        }
#pragma unroll
        for (int q = 0; q < N; ++q) {
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) Mc[q] += __shfl_down_sync(FULL, Mc[q], o);
        }
        if (lane == 0) {
            f.ci[node] = icentre(t.prefix[node], L);
            f.nd[node] = make_int4(nch, c0, t.start[node], t.end[node]);
            store_exp<P>(f.M + (size_t)node * NP, Mc);
        }
    }
}

// ------------------------------------------------------------ the walks
// Per warp: stacks of child ranges per level (each holds at most 32 ranges:
// a level is refilled only from the level above once every deeper level is
// empty, or from the handed-down list once all are empty).
struct WalkSh {
    int2 rs[LEVELS][32];
    int lsz[LEVELS];
};

__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(FULL, v, off);
        if (lane >= off) v += u;
    }
    return v;
}

// The lane whose span of the inclusive sums `incl` holds position pos.
__device__ __forceinline__ int warp_span_of(int incl, int pos)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(FULL, incl, lo + step - 1);
        if (v <= pos) lo += step;
    }
    return lo;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// Next round of up to 32 candidates (one per lane, -1 for none) of a leaf
// target's walk: from the deepest non-empty level stack, else the next 32
// handed-down candidates.  False when the walk is over.
__device__ __forceinline__ bool next_round(WalkSh &w, const int *inh, int ninh, int &cursor,
                                           int lane, int &node)
{
    const int sz = lane < LEVELS ? w.lsz[lane] : 0;
    const unsigned nonempty = __ballot_sync(FULL, sz > 0);
    if (!nonempty) {
        if (cursor >= ninh) return false;
        const int k = cursor + lane;
        node = k < ninh ? __ldg(inh + k) : -1;
        cursor += 32;
        return true;
    }
    const int Lv = 31 - __clz(nonempty);
    const int size = __shfl_sync(FULL, sz, Lv);
    const int R = min(size, 32);
    const int2 r = lane < R ? w.rs[Lv][size - 1 - lane] : make_int2(0, 0);
    const int incl = warp_incl_scan(r.y, lane);
    const int excl = incl - r.y;
    const int take = min(__shfl_sync(FULL, incl, 31), 32);
    const int src = warp_span_of(incl, lane) & 31;
    const int first_src = __shfl_sync(FULL, r.x, src), excl_src = __shfl_sync(FULL, excl, src);
    node = lane < take ? first_src + (lane - excl_src) : -1;
    const unsigned done = __ballot_sync(FULL, lane < R && incl <= 32);
    __syncwarp();
    if (lane < R && excl < 32 && incl > 32)
        w.rs[Lv][size - 1 - lane] = make_int2(r.x + (32 - excl), incl - 32);
    if (lane == 0) w.lsz[Lv] = size - __popc(done);
    __syncwarp();
    return true;
}

// Push the child range (first, nch) of every opening lane onto the stack of
// its node's level + 1.
__device__ __forceinline__ void push_children(WalkSh &w, bool open, int tgt, int first, int nch,
                                              int lane, int *err)
{
    if (!__ballot_sync(FULL, open)) return;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned grp = __match_any_sync(FULL, open ? tgt : -1);
    int slot = 0;
    if (open) slot = w.lsz[tgt] + __popc(grp & lt);
    __syncwarp();
    if (open) {
        if (slot < 32)
            w.rs[tgt][slot] = make_int2(first, nch);
        else
            atomicOr(err, ERR_TREE);  // never: at most 32 pushes onto an empty level
    }
    __syncwarp();
    if (open && (grp & lt) == 0) w.lsz[tgt] = min(w.lsz[tgt] + __popc(grp), 32);
    __syncwarp();
}

// The two tests of a pair of cells, both on the integer squared distance
// D2 of their centres (units of h), as thresholds per pair of levels: D2 is
// an integer and each float64 test is monotone in it, so one integer
// comparison decides exactly as the float64 expression would, without the
// float64 arithmetic in the walks.
struct CritSh {
    int sep[LEVELS][LEVELS];  // separated iff D2 >= sep
    int dir[LEVELS][LEVELS];  // all_direct iff D2 <= dir (-1: never)
};

__device__ __forceinline__ int dist2(int4 a, int4 b)
{
    const int dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ bool separated(int4 a, int4 b, const CritSh &c)
{
    return dist2(a, b) >= c.sep[a.w][b.w];
}

// No descendant of the unseparated candidate B can be separated from target
// A: with k = sqrt(3)/2 and edges in units of h, a descendant C's centre lies
// within k (e_B - e_C) of B's, so |z_A - z_C| < D + k e_B, while separation
// needs more than k e_A / theta.  The margin puts the float64 rounding of
// both this test and the separation test out of play, so walking B's subtree
// would meet exactly B's bodies directly.
__device__ __forceinline__ bool all_direct(int4 a, int4 b, const CritSh &c)
{
    return dist2(a, b) <= c.dir[a.w][b.w];
}

// The float64 form of all_direct for a squared distance D2 between cells of
// levels la (target) and lb.
static __device__ __noinline__ bool all_direct_f64(long long D2, int la, int lb, double theta)
{
    const double D = __dsqrt_rn((double)D2);
    const double k = 0.8660254037844386;
    const double eA = (double)(1 << (11 - la)), eB = (double)(1 << (11 - lb));
    return __dadd_rn(D, __dmul_rn(k, eB)) < __dmul_rn(1.0 - 1e-9, __ddiv_rn(__dmul_rn(k, eA), theta));
}

// Squared distances stay below 3 * 4096^2 (centres lie in [0, 4096)).
constexpr int D2_MAX = 3 * 4096 * 4096;
static_assert(sizeof(CritSh) == FMM_CRIT_INTS * sizeof(int), "threshold table size");

// The thresholds for theta, computed once per evaluation (by
// fmm_init_kernel) into global memory.
__device__ __forceinline__ void crit_compute(CritSh &c, double theta)
{
    for (int i = threadIdx.x; i < LEVELS * LEVELS; i += blockDim.x) {
        const int la = i / LEVELS, lb = i % LEVELS;
        const double s = (double)((1 << (11 - la)) + (1 << (11 - lb)));
        const double crit = __ddiv_rn(__dmul_rn(__dmul_rn(0.75, s), s), __dmul_rn(theta, theta));
        // the least integer >= crit (beyond every distance: never separated)
        c.sep[la][lb] = crit > (double)D2_MAX ? D2_MAX + 1 : (int)ceil(crit);
        // the largest D2 passing all_direct_f64: from the real boundary
        // (sqrt(D2) + k e_B = (1 - 1e-9) k e_A / theta), then stepped to the
        // exact one
        const double k = 0.8660254037844386;
        const double r = (1.0 - 1e-9) * (k * (double)(1 << (11 - la)) / theta) -
                         k * (double)(1 << (11 - lb));
        long long t;
        if (!(r > 0.0))
            t = -1;
        else if (r * r > 2.0 * D2_MAX)
            t = D2_MAX;
        else
            t = (long long)(r * r);
        while (t < D2_MAX && all_direct_f64(t + 1, la, lb, theta)) ++t;
        while (t >= 0 && !all_direct_f64(t, la, lb, theta)) --t;
        c.dir[la][lb] = (int)t;
    }
}

// A block's shared copy of the thresholds (a __syncthreads must follow).
__device__ __forceinline__ void crit_table(CritSh &c, const int *__restrict__ g)
{
    int *d = reinterpret_cast<int *>(&c);
    for (int i = threadIdx.x; i < (int)(sizeof(CritSh) / sizeof(int)); i += blockDim.x) d[i] = g[i];
}

__device__ __forceinline__ Consts consts_of(const FmmParams &p)
{
    Consts K;
    const double ih = 2048.0 / p.box[3];
    K.inv_h = (float)ih;
    K.eps2_h = (float)(p.eps2 * ih * ih);
    return K;
}

// Chunks a warp reserves at a time (one atomic per batch rather than per
// chunk: the atomic's round trip was on every flush's path).
constexpr int CHUNK_BATCH = 16;

// Append the first k entries of a warp's queue q (qcnt entries, at most 64)
// as a chunk of 32 (pad past k) to a linked chunk list: `prev` is the
// list's last chunk so far (-1 for none, then *head is set); the chunk comes
// from the warp's reserved range [cnext, cend), refilled from *ctr; a store
// that is full sets `bit` in *overflow instead and drops the entries.
template <class T>
__device__ __forceinline__ void flush_chunk(T *q, int &qcnt, int k, T pad, T *store, int *next,
                                            int *head, long long cap, int *ctr, int *overflow,
                                            int bit, int &prev, int &cnext, int &cend, int lane)
{
    if (cnext == cend) {
        int r = 0;
        if (lane == 0) r = atomicAdd(ctr, CHUNK_BATCH);
        cnext = __shfl_sync(FULL, r, 0);
        cend = cnext + CHUNK_BATCH;
    }
    const int ch = cnext++;
    if (ch < cap) {
        store[32 * (size_t)ch + lane] = lane < k ? q[lane] : pad;
        if (lane == 0) {
            next[ch] = -1;
            if (prev < 0)
                *head = ch;
            else
                next[prev] = ch;
        }
        prev = ch;
    } else if (lane == 0) {
        atomicOr(overflow, bit);
    }
    __syncwarp();
    if (lane < qcnt - k) q[lane] = q[k + lane];
    qcnt -= k;
    __syncwarp();
}

// ------------------------------------------------------------ downward pass
// Three parts.  (1) Per level L, a warp per cell (dynamic) classifies the
// candidates its parent handed down: a non-leaf hands the unseparated ones
// (or their children) to its own children, a leaf walks their subtrees; the
// separated cells go into the cell's expansion list, in chunks of 32 source
// ids (one per lane of the later evaluation, -1 past the end) linked from
// chunk_head.  (2) One launch over all cells sums each cell's list (M2L, a
// source per lane, the lanes' sums totalled in a fixed order) into L.
// (3) Per level from the top, L2L adds the parent's translated
// coefficients.  The chunks hold the sources in the order the
// classification meets them and each goes to the lane of its position, so
// every lane's sum, and the result, does not depend on scheduling.
template <int P, bool LEAVES>
__global__ void __launch_bounds__(32 * WARPS) fmm_lists_kernel(const FmmParams p, int L)
{
    __shared__ WalkSh wsh[WARPS];
    __shared__ int mq[WARPS][64];
    __shared__ int2 dq[WARPS][LEAVES ? 64 : 1];  // a leaf's directly summed cells: body ranges
    __shared__ CritSh crit;
    crit_table(crit, p.f.crit);
    __syncthreads();
    const TreeView &t = p.tree;
    const FmmView &f = p.f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    // the non-leaves of level L, or all leaves (coarsest first: their walks
    // are the longest)
    const int cnt = LEAVES ? t.meta[TREE_META_BASE + 10] + t.meta[TREE_META_COUNT + 10]
                           : t.meta[TREE_META_COUNT + L];
    const int base = LEAVES ? 0 : t.meta[TREE_META_BASE + L];
    int *queue = f.meta + (LEAVES ? FMM_META_LEAVES_Q : FMM_META_LEVEL + L);
    WalkSh &w = wsh[warp];
    int cnext = 0, cend = 0;    // this warp's reserved expansion-list chunks
    int rcnext = 0, rcend = 0;  // and direct-range chunks
    // one cell: its list (and, for a non-leaf, its hand-down list)
    auto visit = [&](int qi) {
        const int A = base + qi;
        const int nchA = t.nchild[A];
        if ((nchA == 0) != LEAVES) return;  // the other kernel's cell
        const int4 cA = f.ci[A];
        const int par = t.parent[A];
        int inh_off = 0, inh_cnt = 1;  // the root's list: pool[0] = 0
        if (par >= 0) {
            const int2 d = f.down[par];
            inh_off = d.x;
            inh_cnt = d.y;
        }
        const int *inh = f.pool + inh_off;
        int mcnt = 0, own = 0, farb = 0, nearc = 0, prev = -1, dcnt = 0, dprev = -1;
        if (lane == 0) {
            f.chunk_head[A] = -1;
            if (LEAVES) f.rhead[A] = -1;
        }
        // a non-leaf: how many candidates go down (pass 1), and where
        long long off = 0;
        bool fits = true;
        if constexpr (!LEAVES) {
            int total = 0;
            for (int c0 = 0; c0 < inh_cnt; c0 += 32) {
                const int k = c0 + lane;
                const int B = k < inh_cnt ? __ldg(inh + k) : -1;
                int outc = 0;
                if (B >= 0) {
                    const int4 cB = __ldg(f.ci + B), nB = __ldg(f.nd + B);
                    if (!separated(cA, cB, crit)) outc = (nB.x == 0 || cB.w > cA.w) ? 1 : nB.x;
                }
                total += warp_sum(outc);
            }
            if (lane == 0) off = atomicAdd(f.meta + FMM_META_POOL, total);
            off = __shfl_sync(FULL, off, 0);
            fits = off + total <= f.pool_cap;
            if (lane == 0) {
                f.down[A] = make_int2(fits ? (int)off : 0, fits ? total : 0);
                if (!fits) atomicOr(f.meta + FMM_META_OVERFLOW, 1);
            }
        } else {
            if (lane < LEVELS) w.lsz[lane] = 0;
            __syncwarp();
        }
        // Rounds of 32 candidates fill the queue of separated cells; each
        // time it holds 32 (or the candidates are done) the first 32 become
        // a chunk.  A non-leaf classifies its handed-down candidates and
        // writes the others down (pass 2); a leaf walks their subtrees.
        int c0 = 0, cur = 0, cursor = 0;
        bool more = true;
        while (more || mcnt > 0) {
            while (more && mcnt < 32) {
                bool sep = false;
                int B = -1, bodies = 0;
                if constexpr (!LEAVES) {
                    if (c0 >= inh_cnt) {
                        more = false;
                        break;
                    }
                    const int k = c0 + lane;
                    B = k < inh_cnt ? __ldg(inh + k) : -1;
                    c0 += 32;
                    bool self = false;
                    int outc = 0, firstB = 0;
                    if (B >= 0) {
                        const int4 cB = __ldg(f.ci + B), nB = __ldg(f.nd + B);
                        sep = separated(cA, cB, crit);
                        bodies = nB.w - nB.z;
                        if (!sep) {
                            self = nB.x == 0 || cB.w > cA.w;
                            outc = self ? 1 : nB.x;
                            firstB = nB.y;
                            if (!self && cB.w < cA.w) atomicOr(p.err, ERR_TREE);  // never
                        }
                    }
                    const int incl = warp_incl_scan(outc, lane);
                    if (fits && outc) {
                        int *dst = f.pool + off + cur + (incl - outc);
                        if (self)
                            dst[0] = B;
                        else
                            for (int j = 0; j < outc; ++j) dst[j] = firstB + j;
                    }
                    cur += __shfl_sync(FULL, incl, 31);
                } else {
                    if (!next_round(w, inh, inh_cnt, cursor, lane, B)) {
                        more = false;
                        break;
                    }
                    bool open = false, direct = false;
                    int nchB = 0, firstB = 0, lvB = 0;
                    int2 rng = make_int2(0, 0);
                    if (B >= 0) {
                        const int4 cB = __ldg(f.ci + B), nB = __ldg(f.nd + B);
                        sep = separated(cA, cB, crit);
                        nchB = nB.x;
                        bodies = nB.w - nB.z;
                        if (!sep) {
                            open = nchB > 0 && !all_direct(cA, cB, crit);
                            direct = !open;
                            rng = make_int2(nB.z, nB.w);
                            if (direct) nearc += bodies;
                        }
                        firstB = nB.y;
                        lvB = cB.w;
                    }
                    push_children(w, open, lvB + 1, firstB, nchB, lane, p.err);
                    // the directly summed cells, in walk order, for the near field
                    const unsigned dm = __ballot_sync(FULL, direct);
                    if (direct) dq[warp][dcnt + __popc(dm & lt)] = rng;
                    dcnt += __popc(dm);
                    __syncwarp();
                    if (dcnt >= 32)
                        flush_chunk(dq[warp], dcnt, 32, make_int2(0, 0), f.rchunk, f.rnext,
                                    f.rhead + A, f.rchunk_cap, f.meta + FMM_META_RCHUNKS,
                                    f.meta + FMM_META_OVERFLOW, 4, dprev, rcnext, rcend, lane);
                }
                const unsigned sm = __ballot_sync(FULL, sep);
                if (sep) {
                    mq[warp][mcnt + __popc(sm & lt)] = B;
                    farb += bodies;
                }
                mcnt += __popc(sm);
                own += __popc(sm);
                __syncwarp();
            }
            const int k = min(mcnt, 32);
            if (k > 0)
                flush_chunk(mq[warp], mcnt, k, -1, f.chunk_src, f.chunk_next, f.chunk_head + A,
                            f.chunk_cap, f.meta + FMM_META_CHUNKS, f.meta + FMM_META_OVERFLOW, 2,
                            prev, cnext, cend, lane);
        }
        if constexpr (LEAVES) {
            if (dcnt > 0)
                flush_chunk(dq[warp], dcnt, dcnt, make_int2(0, 0), f.rchunk, f.rnext, f.rhead + A,
                            f.rchunk_cap, f.meta + FMM_META_RCHUNKS, f.meta + FMM_META_OVERFLOW,
                            4, dprev, rcnext, rcend, lane);
            nearc = warp_sum(nearc);
            if (lane == 0) {
                f.nearc[A] = nearc;
                f.leaves[atomicAdd(f.meta + FMM_META_NLEAVES, 1)] = A;
            }
        }
        farb = warp_sum(farb);
        if (lane == 0) {
            int2 cum = make_int2(own, farb);
            if (par >= 0) {
                const int2 pc = f.cum[par];
                cum.x += pc.x;
                cum.y += pc.y;
            }
            f.cum[A] = cum;
            if (own) atomicAdd(f.stats + 2, (unsigned long long)own);
        }
        __syncwarp();
    };
    // a block's warps take neighbouring cells together: their candidates
    // (siblings share their parent's hand-down list) and walks meet mostly
    // the same nodes, which the later ones then find in L1
    __shared__ int blk_base;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) blk_base = atomicAdd(queue, WARPS);
        __syncthreads();
        const int b0 = blk_base;
        if (b0 >= cnt) break;
        if (b0 + warp < cnt) visit(b0 + warp);
    }
}

// Resident blocks per SM the expansion-sum kernel's registers are sized
// for: the lane's running sums and the kernel's derivatives of one source
// are both live in its contraction.
template <int P>
constexpr int m2l_min_blocks() { return P <= 5 ? 4 : 2; }

// A warp per cell (dynamic, deepest cells first): the chunks of its list in
// order, a source per lane; lane 0 stores the total (zero for an empty list).
template <int P>
__global__ void __launch_bounds__(32 * WARPS, m2l_min_blocks<P>()) fmm_m2l_kernel(const FmmParams p)
{
    constexpr int N = nterms(P), NP = padded(P);
    const TreeView &t = p.tree;
    const FmmView &f = p.f;
    if (f.meta[FMM_META_OVERFLOW]) return;  // the lists are incomplete: the host reruns
    const Consts K = consts_of(p);
    const int lane = threadIdx.x & 31;
    const int total = t.meta[TREE_META_BASE + 10] + t.meta[TREE_META_COUNT + 10];
    // the next cell's queue ticket is taken while this one's expansions run
    int ticket = 0;
    if (lane == 0) ticket = atomicAdd(f.meta + FMM_META_M2L, 1);
    for (;;) {
        const int qi = __shfl_sync(FULL, ticket, 0);
        if (qi >= total) break;
        if (lane == 0) ticket = atomicAdd(f.meta + FMM_META_M2L, 1);
        const int A = total - 1 - qi;
        float acc[N];
#pragma unroll
        for (int q = 0; q < N; ++q) acc[q] = 0.0f;
        int ch = f.chunk_head[A];
        if (ch >= 0) {
            // the next chunk's sources are loaded before this chunk's expansions
            const int4 cA = f.ci[A];
            int B = f.chunk_src[32 * (size_t)ch + lane];
            while (ch >= 0) {
                const int nx = f.chunk_next[ch];
                const int Bn = nx >= 0 ? f.chunk_src[32 * (size_t)nx + lane] : -1;
                if (B >= 0) m2l_add<P>(acc, f.M + (size_t)B * NP, cA, __ldg(f.ci + B), K);
                ch = nx;
                B = Bn;
            }
#pragma unroll
            for (int q = 0; q < N; ++q) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(FULL, acc[q], o);
            }
        }
        if (lane == 0) store_exp<P>(f.L + (size_t)A * NP, acc);
    }
}

// Cells of level L >= 1, a thread each: L += the parent's coefficients
// translated to the cell's centre.
template <int P>
__global__ void __launch_bounds__(128) fmm_l2l_kernel(const FmmParams p, int L)
{
    constexpr int N = nterms(P), NP = padded(P);
    const TreeView &t = p.tree;
    const FmmView &f = p.f;
    if (f.meta[FMM_META_OVERFLOW]) return;
    const int cnt = t.meta[TREE_META_COUNT + L], base = t.meta[TREE_META_BASE + L];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
        const int A = base + q, par = t.parent[A];
        float acc[N], xp[N];
        const float *dst = f.L + (size_t)A * NP, *src = f.L + (size_t)par * NP;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            acc[k] = dst[k];
            xp[k] = src[k];
        }
        translate_add<P, false>(acc, xp, (int)(t.prefix[A] & 7u));
        store_exp<P>(f.L + (size_t)A * NP, acc);
    }
}

// ------------------------------------------------------------ near field
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

// Source q of a warp's list, in pairs {x0, x1, y0, y1}, {z0, z1, m0, m1}.
__device__ __forceinline__ void list_put(float *Lf, int q, float x, float y, float z, float m)
{
    float *b = Lf + 8 * (q >> 1) + (q & 1);
    b[0] = x;
    b[2] = y;
    b[4] = z;
    b[6] = m;
}

// Work items of the near field: a leaf's bodies 64 at a time (a level-10 leaf
// may hold more), times its directly met sources in up to 64 slices of about
// CHUNK, so that no warp is left alone with a large leaf's sum.
constexpr int CHUNK = 8192, MAX_SLICES = 64;
__device__ __forceinline__ int body_chunks(int nb) { return (nb + 63) >> 6; }
__device__ __forceinline__ int src_slices(int nearc)
{
    return min(MAX_SLICES, max(1, (nearc + CHUNK - 1) / CHUNK));
}

// One block: work items and partial-sum slots per leaf, scanned.
template <int P>
__global__ void __launch_bounds__(1024) fmm_items_kernel(FmmParams p)
{
    __shared__ int tile[BSCAN_TILE + BSCAN_TILE / 32];
    __shared__ int wsum[32];
    const TreeView &t = p.tree;
    const FmmView &f = p.f;
    const int nl = f.meta[FMM_META_NLEAVES];
    for (int q = threadIdx.x; q < nl; q += blockDim.x) {
        const int A = f.leaves[q];
        const int nb = t.end[A] - t.start[A], ns = src_slices(f.nearc[A]);
        f.item_off[q] = body_chunks(nb) * ns;
        f.part_off[q] = ns > 1 ? nb * ns : 0;
    }
    __syncthreads();
    const int items = block_scan_exclusive<int>(f.item_off, f.item_off, nl, tile, wsum);
    __syncthreads();
    const int slots = block_scan_exclusive<int>(f.part_off, f.part_off, nl, tile, wsum);
    if (threadIdx.x == 0) {
        f.item_off[nl] = items;
        f.part_off[nl] = slots;
        f.meta[FMM_META_ITEMS] = items;
        f.meta[FMM_META_PSLOTS] = slots;
    }
}

// G (near + far) into acc for the body at tree rank k of leaf A (centre z,
// inverse edge inv_e); the far field is the gradient of A's local expansion
// (L2P).
template <int P>
__device__ __forceinline__ void write_body(const FmmParams &p, int A, const double (&z)[3],
                                           double inv_e, int k, double nx, double ny, double nz,
                                           int nnear)
{
    constexpr int NP = padded(P);
    const FmmView &f = p.f;
    const float *Lc = f.L + (size_t)A * NP;
    const int i = p.perm[k];
    float pw[3][P + 1];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        scaled_powers<P>((float)((p.pos[3 * (size_t)i + c] - z[c]) * inv_e), pw[c]);
    float fa[3] = {0.f, 0.f, 0.f};
    sfor<0, nterms(P - 1)>([&](auto kI) {
        constexpr int q = decltype(kI)::value;
        constexpr int a = mi_of(q, 0), b = mi_of(q, 1), c = mi_of(q, 2);
        const float wv = pw[0][a] * pw[1][b] * pw[2][c];
        fa[0] = fmaf(__ldg(Lc + slot_of(a + 1, b, c)), wv, fa[0]);
        fa[1] = fmaf(__ldg(Lc + slot_of(a, b + 1, c)), wv, fa[1]);
        fa[2] = fmaf(__ldg(Lc + slot_of(a, b, c + 1)), wv, fa[2]);
    });
    const double gx = p.G * (nx + (double)fa[0] * inv_e);
    const double gy = p.G * (ny + (double)fa[1] * inv_e);
    const double gz = p.G * (nz + (double)fa[2] * inv_e);
    double *a = p.acc + 3 * (size_t)i;
    a[0] = gx;
    a[1] = gy;
    a[2] = gz;
    if (p.vel) {  // a step's closing half-kick
        double *v = p.vel + 3 * (size_t)i;
        v[0] += p.half_dt * gx;
        v[1] += p.half_dt * gy;
        v[2] += p.half_dt * gz;
    }
    if (p.counts) {
        const int2 cm = f.cum[A];
        p.counts[3 * (size_t)i] = cm.x;
        p.counts[3 * (size_t)i + 1] = cm.y;
        p.counts[3 * (size_t)i + 2] = nnear;
    }
    if (!finite3(gx, gy, gz)) atomicOr(p.err, ERR_NONFINITE);
}

// (s, c) += (so, co) for Kahan pairs holding s - c: the sums' rounding
// error goes into the carry (the two-sum of s and so).
__device__ __forceinline__ void kahan_merge(float &s, float &c, float so, float co)
{
    const float t = s + so;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (so - bp);
    s = t;
    c = (c + co) - e;
}

// write_body for a near field held as float32 Kahan pairs (s - c): the L2P
// in float32 from the body's hi/lo position relative to the centre's hi/lo
// pair (zh, zl) times 1/e, the far field added into the pair, one float64
// conversion at the end.
template <int P>
__device__ __forceinline__ void write_body_kahan(const FmmParams &p, int A, const float (&zh)[3],
                                                 const float (&zl)[3], float inv_e, int k,
                                                 float (&ks)[3], float (&kc)[3], int nnear)
{
    constexpr int NP = padded(P);
    const FmmView &f = p.f;
    const float *Lc = f.L + (size_t)A * NP;
    const int i = p.perm[k];
    const float4 h = __ldg(p.P + k), l = __ldg(p.Plo + k);
    const float hx[3] = {h.x, h.y, h.z}, lx[3] = {l.x, l.y, l.z};
    float pw[3][P + 1];
#pragma unroll
    for (int c = 0; c < 3; ++c) scaled_powers<P>(((hx[c] - zh[c]) + (lx[c] - zl[c])) * inv_e, pw[c]);
    float fa[3] = {0.f, 0.f, 0.f};
    sfor<0, nterms(P - 1)>([&](auto kI) {
        constexpr int q = decltype(kI)::value;
        constexpr int a = mi_of(q, 0), b = mi_of(q, 1), c = mi_of(q, 2);
        const float wv = pw[0][a] * pw[1][b] * pw[2][c];
        fa[0] = fmaf(__ldg(Lc + slot_of(a + 1, b, c)), wv, fa[0]);
        fa[1] = fmaf(__ldg(Lc + slot_of(a, b + 1, c)), wv, fa[1]);
        fa[2] = fmaf(__ldg(Lc + slot_of(a, b, c + 1)), wv, fa[2]);
    });
    double g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        kahan_add(ks[c], kc[c], fa[c] * inv_e);
        g[c] = p.G * ((double)ks[c] - (double)kc[c]);
    }
    double *a = p.acc + 3 * (size_t)i;
    a[0] = g[0];
    a[1] = g[1];
    a[2] = g[2];
    if (p.vel) {  // a step's closing half-kick
        double *v = p.vel + 3 * (size_t)i;
        v[0] += p.half_dt * g[0];
        v[1] += p.half_dt * g[1];
        v[2] += p.half_dt * g[2];
    }
    if (p.counts) {
        const int2 cm = f.cum[A];
        p.counts[3 * (size_t)i] = cm.x;
        p.counts[3 * (size_t)i + 1] = cm.y;
        p.counts[3 * (size_t)i + 2] = nnear;
    }
    if (!finite3(g[0], g[1], g[2])) atomicOr(p.err, ERR_NONFINITE);
}

// A warp per work item (dynamic): the body ranges of the cells the leaf's
// walk met directly, in the order the walk recorded them; the item's slice
// of those bodies is
// listed (coordinates relative to the leaf's centre) and every FLUSH of them
// added onto its bodies: two bodies per lane (b and b + T, T = nb / 2 rounded
// up to a power of two), lane = b + T * slice, the 32 / T slices sharing the
// source pairs.  The slices' sums are combined in a fixed
// order; a leaf in one item gets its result written, a split one its
// partial sums stored for fmm_combine_kernel.
template <int P, bool ZEPS>
__global__ void __launch_bounds__(32 * WARPS) fmm_near_kernel(const FmmParams p)
{
    __shared__ __align__(16) float4 lists[WARPS][2 * FLUSH];  // 2 * FLUSH sources as pairs
    const TreeView &t = p.tree;
    const FmmView &f = p.f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nleaves = f.meta[FMM_META_NLEAVES], nitems = f.meta[FMM_META_ITEMS];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        f.stats[0] = (unsigned long long)(t.meta[TREE_META_BASE + 10] + t.meta[TREE_META_COUNT + 10]);
        f.stats[1] = (unsigned long long)nleaves;
    }
    float *Lf = reinterpret_cast<float *>(lists[warp]);
    const float4 *L4 = lists[warp];
    const float2 e2 = make_float2(p.eps2f, p.eps2f);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(f.meta + FMM_META_NEAR, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= nitems) break;
        // the leaf holding item `it`: the last qi with item_off[qi] <= it
        int lo = 0, hi = nleaves;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (f.item_off[mid] <= it)
                lo = mid;
            else
                hi = mid;
        }
        const int qi = lo, A = f.leaves[qi];
        const int4 cA = f.ci[A];
        const int nearc = f.nearc[A], ns = src_slices(nearc);
        const int j = it - f.item_off[qi], bc = j / ns, sc = j % ns;
        const int nbt = t.end[A] - t.start[A];
        const int s0 = t.start[A] + 64 * bc, nb = min(64, t.end[A] - s0);
        const int per = (nearc + ns - 1) / ns;
        const int src_lo = sc * per, src_hi = min(nearc, src_lo + per);
        double z[3];
        centre_of(p.box, cA, z);
        const float cx = (float)z[0], cy = (float)z[1], cz = (float)z[2];
        // two bodies per lane, b0 and b0 + T (T = nb / 2 rounded up to a power
        // of two), and 32 / T slices of the sources
        const int half = (nb + 1) >> 1;
        const int T = half <= 1 ? 1 : 1 << (32 - __clz(half - 1));
        const int S = 32 / T;
        const int slice = lane / T, b0 = lane % T;
        const bool v0 = b0 < nb, v1 = b0 + T < nb;
        float2 nx0 = make_float2(0.f, 0.f), ny0 = nx0, nz0 = nx0, nx1 = nx0, ny1 = nx0, nz1 = nx0;
        if (v0) {
            const float4 h = __ldg(p.P + s0 + b0), l = __ldg(p.Plo + s0 + b0);
            const float x = -rel(h.x, l.x, cx), y = -rel(h.y, l.y, cy), zz = -rel(h.z, l.z, cz);
            nx0 = make_float2(x, x);
            ny0 = make_float2(y, y);
            nz0 = make_float2(zz, zz);
        }
        if (v1) {
            const float4 h = __ldg(p.P + s0 + b0 + T), l = __ldg(p.Plo + s0 + b0 + T);
            const float x = -rel(h.x, l.x, cx), y = -rel(h.y, l.y, cy), zz = -rel(h.z, l.z, cz);
            nx1 = make_float2(x, x);
            ny1 = make_float2(y, y);
            nz1 = make_float2(zz, zz);
        }
        float2 ax0 = make_float2(0.f, 0.f), ay0 = ax0, az0 = ax0, ax1 = ax0, ay1 = ax0, az1 = ax0;
        float ks[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        float kc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        auto fold = [&]() {
            kahan_add(ks[0][0], kc[0][0], ax0.x);
            kahan_add(ks[0][0], kc[0][0], ax0.y);
            kahan_add(ks[0][1], kc[0][1], ay0.x);
            kahan_add(ks[0][1], kc[0][1], ay0.y);
            kahan_add(ks[0][2], kc[0][2], az0.x);
            kahan_add(ks[0][2], kc[0][2], az0.y);
            kahan_add(ks[1][0], kc[1][0], ax1.x);
            kahan_add(ks[1][0], kc[1][0], ax1.y);
            kahan_add(ks[1][1], kc[1][1], ay1.x);
            kahan_add(ks[1][1], kc[1][1], ay1.y);
            kahan_add(ks[1][2], kc[1][2], az1.x);
            kahan_add(ks[1][2], kc[1][2], az1.y);
            ax0 = ay0 = az0 = ax1 = ay1 = az1 = make_float2(0.f, 0.f);
        };
        auto eval = [&](int npairs) {
            for (int q = slice; q < npairs; q += S) {
                const float4 a = L4[2 * q], bq = L4[2 * q + 1];
                const float2 sx = make_float2(a.x, a.y), sy = make_float2(a.z, a.w);
                const float2 sz = make_float2(bq.x, bq.y), sm = make_float2(bq.z, bq.w);
                pair_terms<ZEPS>(add2(sx, nx0), add2(sy, ny0), add2(sz, nz0), sm, e2, ax0, ay0, az0);
                pair_terms<ZEPS>(add2(sx, nx1), add2(sy, ny1), add2(sz, nz1), sm, e2, ax1, ay1, az1);
            }
        };
        int cnt = 0, seen = 0;  // listed sources; direct sources met so far in walk order
        auto flush = [&]() {
            __syncwarp();
            eval(FLUSH / 2);
            fold();
            __syncwarp();
            for (int c = lane; c < FLUSH; c += 32) lists[warp][c] = lists[warp][FLUSH + c];
            cnt -= FLUSH;
            __syncwarp();
        };
        for (int rc = f.rhead[A]; rc >= 0 && seen < src_hi;) {
            const int2 r = f.rchunk[32 * (size_t)rc + lane];  // (0, 0) past the list's end
            rc = f.rnext[rc];
            const int ls = r.x, lsz = r.y - r.x;
            const int linc = warp_incl_scan(lsz, lane);
            const int lexc = linc - lsz;
            const int tot = __shfl_sync(FULL, linc, 31);
            // this chunk's direct sources are [seen, seen + tot) in walk order
            const int a0 = max(src_lo - seen, 0), a1 = min(src_hi - seen, tot);
            for (int c0 = a0; c0 < a1; c0 += 32) {
                const int pos = c0 + lane;
                const int jj = warp_span_of(linc, pos) & 31;
                const int body = __shfl_sync(FULL, ls, jj) + (pos - __shfl_sync(FULL, lexc, jj));
                const int kk = min(32, a1 - c0);
                if (lane < kk) {
                    const float4 bh = __ldg(p.P + body), bl = __ldg(p.Plo + body);
                    list_put(Lf, cnt + lane, rel(bh.x, bl.x, cx), rel(bh.y, bl.y, cy),
                             rel(bh.z, bl.z, cz), bh.w);
                }
                cnt += kk;
                if (cnt >= FLUSH) flush();
            }
            seen += tot;
        }
        if (cnt > 0) {
            if (lane == 0 && (cnt & 1)) list_put(Lf, cnt, 0.f, 0.f, 0.f, 0.f);
            __syncwarp();
            eval((cnt + 1) >> 1);
            fold();
        }
        // combine the slices' Kahan pairs in float32 (lane b0 of slice 0 ends
        // with the total): float64 work is scarce on this part
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                for (int off = 16; off >= T; off >>= 1) {
                    const float so = __shfl_down_sync(FULL, ks[b][c], off);
                    const float co = __shfl_down_sync(FULL, kc[b][c], off);
                    kahan_merge(ks[b][c], kc[b][c], so, co);
                }
        if (slice == 0) {
            // 1/e = (2048 / ext) 2^(L - 11): the float32 1/h scaled exactly
            const float inv_e = (float)(2048.0 / p.box[3]) * pow2f(cA.w - 11);
            float zh[3], zl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                zh[c] = (float)z[c];
                zl[c] = (float)(z[c] - (double)zh[c]);
            }
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                if (!(b == 0 ? v0 : v1)) continue;
                const int k = s0 + b0 + T * b;
                if (ns == 1) {
                    write_body_kahan<P>(p, A, zh, zl, inv_e, k, ks[b], kc[b], nearc);
                } else {
                    double *d = f.part + 3 * ((size_t)f.part_off[qi] + (size_t)sc * nbt +
                                              (size_t)(k - t.start[A]));
#pragma unroll
                    for (int c = 0; c < 3; ++c) d[c] = (double)ks[b][c] - (double)kc[b][c];
                }
            }
        }
        if (lane == 0)
            atomicAdd(f.stats + 3, (unsigned long long)nb * (unsigned long long)(src_hi - src_lo));
        __syncwarp();
    }
}

// Leaves whose direct sum was split: the slices' partial sums added in slice
// order, then the far field, per body (a thread per body of each such leaf).
template <int P>
__global__ void __launch_bounds__(256) fmm_combine_kernel(const FmmParams p)
{
    const TreeView &t = p.tree;
    const FmmView &f = p.f;
    const int nleaves = f.meta[FMM_META_NLEAVES];
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int qi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); qi < nleaves; qi += warps) {
        const int A = f.leaves[qi];
        const int nearc = f.nearc[A], ns = src_slices(nearc);
        if (ns == 1) continue;
        const int4 cA = f.ci[A];
        const int nbt = t.end[A] - t.start[A];
        const double *base = f.part + 3 * (size_t)f.part_off[qi];
        double z[3];
        centre_of(p.box, cA, z);
        const double inv_e = (double)(1 << cA.w) / p.box[3];
        for (int b = lane; b < nbt; b += 32) {
            double s[3] = {0.0, 0.0, 0.0};
            for (int sc = 0; sc < ns; ++sc) {
                const double *d = base + 3 * ((size_t)sc * nbt + b);
                s[0] += d[0];
                s[1] += d[1];
                s[2] += d[2];
            }
            write_body<P>(p, A, z, inv_e, t.start[A] + b, s[0], s[1], s[2], nearc);
        }
    }
}

template <int P>
__global__ void __launch_bounds__(128) fmm_init_kernel(FmmView f, double theta)
{
    crit_compute(*reinterpret_cast<CritSh *>(f.crit), theta);
    if (threadIdx.x < FMM_META_INTS) f.meta[threadIdx.x] = 0;
    if (threadIdx.x < 4) f.stats[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) {
        f.pool[0] = 0;  // the root is its own candidate
        f.meta[FMM_META_POOL] = 1;
    }
}

template <class K>
int resident_grid(K kernel, int threads, int num_sms, cudaError_t &e)
{
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    return std::max(1, per_sm) * num_sms;
}

// near = false: upward pass, downward levels and the near-field work items;
// near = true: the near field and the split leaves' combination.
template <int P>
cudaError_t launch_fmm_order(cudaStream_t s, const FmmParams &p, bool near, int &kernels)
{
    kernels = 0;
    cudaError_t e = cudaSuccess;
    if (!near) {
        fmm_init_kernel<P><<<1, 128, 0, s>>>(p.f, p.theta);
        const int p2m_grid = (int)std::min<long long>(
            8 * p.num_sms, ((long long)p.tree.cap + 32 * UP_WARPS - 1) / (32 * UP_WARPS));
        fmm_p2m_kernel<P><<<p2m_grid, 32 * UP_WARPS, 0, s>>>(p);
        for (int L = LEVELS - 2; L >= 0; --L)
            fmm_m2m_kernel<P><<<8 * p.num_sms, 32 * UP_WARPS, 0, s>>>(p, L);
        const int lists_grid = resident_grid(fmm_lists_kernel<P, true>, 32 * WARPS, p.num_sms, e);
        if (e != cudaSuccess) return e;
        const int m2l_grid = resident_grid(fmm_m2l_kernel<P>, 32 * WARPS, p.num_sms, e);
        if (e != cudaSuccess) return e;
        for (int L = 0; L < LEVELS; ++L)
            fmm_lists_kernel<P, false><<<lists_grid, 32 * WARPS, 0, s>>>(p, L);
        fmm_lists_kernel<P, true><<<lists_grid, 32 * WARPS, 0, s>>>(p, 0);
        fmm_m2l_kernel<P><<<m2l_grid, 32 * WARPS, 0, s>>>(p);
        for (int L = 1; L < LEVELS; ++L) fmm_l2l_kernel<P><<<2 * p.num_sms, 128, 0, s>>>(p, L);
        fmm_items_kernel<P><<<1, 1024, 0, s>>>(p);
        kernels = 5 + 3 * LEVELS - 2;
        return cudaGetLastError();
    }
    const bool zeps = p.eps2f == 0.0f;
    const int near_grid = zeps ? resident_grid(fmm_near_kernel<P, true>, 32 * WARPS, p.num_sms, e)
                               : resident_grid(fmm_near_kernel<P, false>, 32 * WARPS, p.num_sms, e);
    if (e != cudaSuccess) return e;
    if (zeps)
        fmm_near_kernel<P, true><<<near_grid, 32 * WARPS, 0, s>>>(p);
    else
        fmm_near_kernel<P, false><<<near_grid, 32 * WARPS, 0, s>>>(p);
    fmm_combine_kernel<P><<<4 * p.num_sms, 256, 0, s>>>(p);
    kernels = 2;
    return cudaGetLastError();
}

}  // namespace fmm
}  // namespace nb
