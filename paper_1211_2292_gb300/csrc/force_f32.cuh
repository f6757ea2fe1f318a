// float32 softened direct-sum force kernels (paper Sec. IV-A/IV-B: the force
// calculation, here the exact all-pairs sum):
//
//   a_i = G sum_j m_j d_ij / (|d_ij|^2 + eps^2)^{3/2},   d_ij = x_j - x_i.
//
// Design (sm_103a):
//  * An i-tile of T*I bodies per CTA; each thread keeps I bodies in
//    registers, paired into float32x2 lanes so that every pair operation is
//    one issue slot for two bodies.
//  * j-bodies stream through a double-buffered shared-memory tile of J
//    bodies, stored with each component duplicated ((x,x,y,y),(z,z,m,m)) so a
//    broadcast 128-bit shared load yields the float32x2 operands directly.
//    The next tile's global loads are issued before the current tile is
//    consumed.  Out-of-range j slots are zero-mass bodies.
//  * Tile-local origin: positions arrive as float32 hi/lo pairs
//    (x = x_hi + x_lo).  Each CTA takes the centre c of its i-tile's bounding
//    box as origin and forms every coordinate as (x_hi - c) + x_lo, once per
//    body per CTA when staging.  The pair differences then carry the
//    rounding of |x - c| instead of |x|, which for spatially ordered i-tiles
//    (order.cu) keeps close pairs accurate far from the global origin.  The
//    per-pair arithmetic is unchanged.
//  * Per pair: 3 add, 3 fma (r^2), 1 MUFU rsqrt per body, 3 mul, 3 fma;
//    12 float32 operations, i.e. 6 float32x2 issues per body.
//  * NB_FP32_COMP: each tile's float32 partial sum is added into a per-body
//    Kahan (sum, carry) pair, so rounding grows with the tile count, not
//    with N.  NB_FP32: one running float32 sum.
//  * j-split: the grid is (i-tiles x nsplit).  With nsplit > 1, each CTA
//    stores its float64 partial; the last CTA of an i-tile (arrival counter)
//    adds the partials in split order (deterministic) and runs the epilogue.
//    No CTA ever waits for another.
//  * Epilogue: acc = G*sum in float64, optional fused half-kick
//    vel += dt/2 * acc, non-finite outputs flagged in the error word.
#pragma once

#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

constexpr int UNROLL_F32 = 8;

// Final write of one body's acceleration (float64, G applied).
__device__ __forceinline__ void write_acc(const ForceParams &p, int i, double ax, double ay,
                                          double az)
{
    double *a = p.acc + 3 * (size_t)i;
    a[0] = ax;
    a[1] = ay;
    a[2] = az;
    if (p.vel) {
        double *v = p.vel + 3 * (size_t)i;
        v[0] += p.half_dt * ax;
        v[1] += p.half_dt * ay;
        v[2] += p.half_dt * az;
    }
    if (!finite3(ax, ay, az)) atomicOr(p.err, ERR_NONFINITE);
}

// Interaction of one body pair-lane set with j-body (xj,yj,zj,wj) given as
// duplicated float32x2 values.  nx/ny/nz hold the NEGATED i positions.
//
// Two forms of the pair factor s = m_j / (r^2 + eps^2)^{3/2}:
//  * rsqrt (LOGM = false, wj = m_j): r = rsqrt(r^2) on the MUFU pipe, then
//    s = (r*r)*(m_j*r): 12 float32 operations per pair in total.
//  * log domain (LOGM = true, wj = log2 m_j): s = 2^(log2 m_j - 1.5 log2 r^2)
//    with lg2 and ex2 on the MUFU pipe and one fma: 10 float32 operations and
//    2 MUFU per pair.  On GB300 the FMA pipe takes 128 float32 operations per
//    clock per SM, rsqrt and lg2 16 and ex2 32 MUFU operations (as the
//    kernels' own pipe counters show), so the rsqrt form is FMA-bound and
//    the log form MUFU-bound at the same 10.7 pairs/clk/SM; a thread that
//    runs 2/3 of its body pairs in the log form balances both pipes at
//    12 pairs/clk/SM.
//    Needs m_j >= 0 (m_j = 0 gives log2 = -inf, s = 0).
template <bool ZEPS, bool LOGM>
__device__ __forceinline__ void interact2(float2 xj, float2 yj, float2 zj, float2 wj, float2 e2,
                                          float2 nx, float2 ny, float2 nz, float2 &ax, float2 &ay,
                                          float2 &az)
{
    float2 dx = add2(xj, nx);
    float2 dy = add2(yj, ny);
    float2 dz = add2(zj, nz);
    float2 r2 = fma2(dx, dx, e2);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    float2 s;
    if (LOGM) {
        float2 l;
        l.x = lg2_mufu(r2.x);
        l.y = lg2_mufu(r2.y);
        const float2 t = fma2(l, make_float2(-1.5f, -1.5f), wj);
        s.x = ex2_mufu(t.x);
        s.y = ex2_mufu(t.y);
        if (ZEPS) {  // eps == 0: the self pair (r^2 == 0) must contribute nothing
            s.x = r2.x > 0.f ? s.x : 0.f;
            s.y = r2.y > 0.f ? s.y : 0.f;
        }
    } else {
        float2 ri;
        ri.x = rsqrt_mufu(r2.x);
        ri.y = rsqrt_mufu(r2.y);
        if (ZEPS) {
            ri.x = r2.x > 0.f ? ri.x : 0.f;
            ri.y = r2.y > 0.f ? ri.y : 0.f;
        }
        const float2 ri2 = mul2(ri, ri);
        const float2 mri = mul2(wj, ri);
        s = mul2(ri2, mri);
    }
    ax = fma2(dx, s, ax);
    ay = fma2(dy, s, ay);
    az = fma2(dz, s, az);
}


// Shared-tile slots per j-body: (x,x,y,y), (z,z,m,m) and, for kernels with
// log-domain pairs, (log2 m, log2 m, ., .).
template <int LP>
struct Slots {
    static constexpr int W = LP > 0 ? 3 : 2;
};

// Stage this thread's share of a j-tile into the duplicated shared layout,
// in coordinates relative to the tile origin c.
template <int T, int J, int LP>
__device__ __forceinline__ void stage_store(float4 *tile, const float4 (&bh)[J / T],
                                            const float4 (&bl)[J / T], float3 c)
{
    constexpr int W = Slots<LP>::W;
#pragma unroll
    for (int l = 0; l < J / T; ++l) {
        const int jj = l * T + threadIdx.x;
        const float x = rel(bh[l].x, bl[l].x, c.x);
        const float y = rel(bh[l].y, bl[l].y, c.y);
        const float z = rel(bh[l].z, bl[l].z, c.z);
        const float m = bh[l].w;
        tile[W * jj] = make_float4(x, x, y, y);
        tile[W * jj + 1] = make_float4(z, z, m, m);
        if (W == 3) tile[W * jj + 2] = make_float4(bl[l].w, bl[l].w, 0.f, 0.f);
    }
}

// Out-of-range j slots become massless bodies (m = 0, log2 m = -inf).
template <int T, int J>
__device__ __forceinline__ void stage_load(float4 (&bh)[J / T], float4 (&bl)[J / T],
                                           const float4 *__restrict__ P,
                                           const float4 *__restrict__ Plo, int jbase, int jend)
{
#pragma unroll
    for (int l = 0; l < J / T; ++l) {
        const int j = jbase + l * T + threadIdx.x;
        const bool ok = j < jend;
        bh[l] = ok ? __ldg(P + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        bl[l] = ok ? __ldg(Plo + j) : make_float4(0.f, 0.f, 0.f, -INFINITY);
    }
}

// Accumulator state for the I bodies of one thread.  The per-tile partials
// live in registers; with KSM the Kahan (sum, carry) pairs live in shared
// memory instead (touched once per j-tile), which frees 6*I registers for
// occupancy.  ks: this CTA's [6][I][T] float array (KSM only).
template <int T, int I, bool COMP, bool KSM>
struct Acc {
    static constexpr int NP = I / 2;
    static constexpr bool REG = COMP && !KSM;
    float2 ax[NP], ay[NP], az[NP];
    float sx[REG ? I : 1], sy[REG ? I : 1], sz[REG ? I : 1];
    float cx[REG ? I : 1], cy[REG ? I : 1], cz[REG ? I : 1];
    float *ks;

    __device__ __forceinline__ float &ksm(int q, int k) const { return ks[(q * I + k) * T + threadIdx.x]; }

    __device__ __forceinline__ void init(float *ks_)
    {
        ks = ks_;
#pragma unroll
        for (int p = 0; p < NP; ++p) ax[p] = ay[p] = az[p] = make_float2(0.f, 0.f);
        if (REG) {
#pragma unroll
            for (int k = 0; k < I; ++k) sx[k] = sy[k] = sz[k] = cx[k] = cy[k] = cz[k] = 0.f;
        }
        if (COMP && KSM) {
#pragma unroll
            for (int k = 0; k < I; ++k)
#pragma unroll
                for (int q = 0; q < 6; ++q) ksm(q, k) = 0.f;
        }
    }
    __device__ __forceinline__ void fold(int q, int k, float part)
    {
        float sv = ksm(q, k), cv = ksm(q + 3, k);
        kahan_add(sv, cv, part);
        ksm(q, k) = sv;
        ksm(q + 3, k) = cv;
    }
    // End of a j-tile: fold the tile partial into the compensated sums.
    __device__ __forceinline__ void end_tile()
    {
        if (REG) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                kahan_add(sx[2 * p], cx[2 * p], ax[p].x);
                kahan_add(sx[2 * p + 1], cx[2 * p + 1], ax[p].y);
                kahan_add(sy[2 * p], cy[2 * p], ay[p].x);
                kahan_add(sy[2 * p + 1], cy[2 * p + 1], ay[p].y);
                kahan_add(sz[2 * p], cz[2 * p], az[p].x);
                kahan_add(sz[2 * p + 1], cz[2 * p + 1], az[p].y);
                ax[p] = ay[p] = az[p] = make_float2(0.f, 0.f);
            }
        } else if (COMP && KSM) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                fold(0, 2 * p, ax[p].x);
                fold(0, 2 * p + 1, ax[p].y);
                fold(1, 2 * p, ay[p].x);
                fold(1, 2 * p + 1, ay[p].y);
                fold(2, 2 * p, az[p].x);
                fold(2, 2 * p + 1, az[p].y);
                ax[p] = ay[p] = az[p] = make_float2(0.f, 0.f);
            }
        }
    }
    // Value of body k's sum in float64.
    __device__ __forceinline__ void get(int k, double &x, double &y, double &z) const
    {
        if (REG) {
            x = (double)sx[k] - (double)cx[k];
            y = (double)sy[k] - (double)cy[k];
            z = (double)sz[k] - (double)cz[k];
        } else if (COMP && KSM) {
            x = (double)ksm(0, k) - (double)ksm(3, k);
            y = (double)ksm(1, k) - (double)ksm(4, k);
            z = (double)ksm(2, k) - (double)ksm(5, k);
        } else {
            const int p = k >> 1;
            x = (k & 1) ? ax[p].y : ax[p].x;
            y = (k & 1) ? ay[p].y : ay[p].x;
            z = (k & 1) ? az[p].y : az[p].x;
        }
    }
};

// Sweep the j-tiles [t0, t1) of bodies [jlo, jhi) (tile t starts at
// jlo + t*J) for this thread's bodies.  Threads split each tile's j loop in
// `lanes` interleaved parts (lanes == 1 for the solo kernel).  Body pairs
// p < LP use the log-domain pair factor, the others rsqrt.
template <int T, int I, int J, bool COMP, bool ZEPS, int LP, bool LANES, bool KSM, int UNR>
__device__ __forceinline__ void sweep(const float4 *__restrict__ P, const float4 *__restrict__ Plo,
                                      float3 c, int jlo, int jhi, int t0, int t1, int lane,
                                      int lanes, float2 e2, const float2 (&nx)[I / 2],
                                      const float2 (&ny)[I / 2], const float2 (&nz)[I / 2],
                                      Acc<T, I, COMP, KSM> &acc, float4 (*tile)[Slots<LP>::W * J])
{
    constexpr int NP = I / 2;
    constexpr int W = Slots<LP>::W;
    float4 bh[J / T], bl[J / T];
    if (t0 < t1) {
        stage_load<T, J>(bh, bl, P, Plo, jlo + t0 * J, jhi);
        stage_store<T, J, LP>(tile[0], bh, bl, c);
    }
    __syncthreads();
    for (int t = t0; t < t1; ++t) {
        const int b = (t - t0) & 1;
        if (t + 1 < t1) stage_load<T, J>(bh, bl, P, Plo, jlo + (t + 1) * J, jhi);
        const float4 *s = tile[b];
        if (LANES) {
#pragma unroll 4
            for (int jj = lane; jj < J; jj += lanes) {
                const float4 q0 = s[W * jj], q1 = s[W * jj + 1];
                const float2 xj = make_float2(q0.x, q0.y), yj = make_float2(q0.z, q0.w);
                const float2 zj = make_float2(q1.x, q1.y), mj = make_float2(q1.z, q1.w);
                float2 lj = mj;
                if (LP > 0) {
                    const float4 q2 = s[W * jj + 2];
                    lj = make_float2(q2.x, q2.y);
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    if (p < LP)
                        interact2<ZEPS, true>(xj, yj, zj, lj, e2, nx[p], ny[p], nz[p], acc.ax[p],
                                              acc.ay[p], acc.az[p]);
                    else
                        interact2<ZEPS, false>(xj, yj, zj, mj, e2, nx[p], ny[p], nz[p], acc.ax[p],
                                               acc.ay[p], acc.az[p]);
                }
            }
        } else {
#pragma unroll UNR
            for (int jj = 0; jj < J; ++jj) {
                const float4 q0 = s[W * jj], q1 = s[W * jj + 1];
                const float2 xj = make_float2(q0.x, q0.y), yj = make_float2(q0.z, q0.w);
                const float2 zj = make_float2(q1.x, q1.y), mj = make_float2(q1.z, q1.w);
                float2 lj = mj;
                if (LP > 0) {
                    const float4 q2 = s[W * jj + 2];
                    lj = make_float2(q2.x, q2.y);
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    if (p < LP)
                        interact2<ZEPS, true>(xj, yj, zj, lj, e2, nx[p], ny[p], nz[p], acc.ax[p],
                                              acc.ay[p], acc.az[p]);
                    else
                        interact2<ZEPS, false>(xj, yj, zj, mj, e2, nx[p], ny[p], nz[p], acc.ax[p],
                                               acc.ay[p], acc.az[p]);
                }
            }
        }
        acc.end_tile();
        if (t + 1 < t1) stage_store<T, J, LP>(tile[b ^ 1], bh, bl, c);
        __syncthreads();
    }
}

// Load this thread's i-bodies.  Body k of the thread is at packed slot
// `first + k*stride`; slots at or past `end` read as zero.  Returns the tile
// origin; nx/ny/nz receive the NEGATED tile-local positions, paired.
template <int T, int I>
__device__ __forceinline__ float3 load_i(const float4 *__restrict__ P, const float4 *__restrict__ Plo,
                                         int first, int stride, int end, float2 (&nx)[I / 2],
                                         float2 (&ny)[I / 2], float2 (&nz)[I / 2],
                                         float (*red)[T / 32])
{
    float4 h[I], l[I];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = first + k * stride;
        const bool ok = i < end;
        h[k] = ok ? __ldg(P + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        l[k] = ok ? __ldg(Plo + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok) {
            mn[0] = fminf(mn[0], h[k].x); mx[0] = fmaxf(mx[0], h[k].x);
            mn[1] = fminf(mn[1], h[k].y); mx[1] = fmaxf(mx[1], h[k].y);
            mn[2] = fminf(mn[2], h[k].z); mx[2] = fmaxf(mx[2], h[k].z);
        }
    }
    const float3 c = block_center<T>(mn, mx, red);
#pragma unroll
    for (int p = 0; p < I / 2; ++p) {
        const float4 a = h[2 * p], b = h[2 * p + 1], al = l[2 * p], bl = l[2 * p + 1];
        nx[p] = make_float2(-rel(a.x, al.x, c.x), -rel(b.x, bl.x, c.x));
        ny[p] = make_float2(-rel(a.y, al.y, c.y), -rel(b.y, bl.y, c.y));
        nz[p] = make_float2(-rel(a.z, al.z, c.z), -rel(b.z, bl.z, c.z));
    }
    return c;
}

// -------------------------------------------------------------- solo kernel
// MINB > 0 caps registers so that MINB CTAs fit per SM; 0 leaves the choice
// to the compiler.
template <int T, int I, int J, bool COMP, bool ZEPS, int LP, bool KSM, int MINB, int UNR>
__global__ void __launch_bounds__(T, MINB) force_f32_kernel(const ForceParams p)
{
    static_assert(I % 2 == 0 && J % T == 0 && LP <= I / 2, "bad tile shape");
    constexpr int TILE_I = T * I;
    __shared__ __align__(16) float4 tile[2][Slots<LP>::W * J];
    __shared__ float red[6][T / 32];
    __shared__ float ks[(COMP && KSM) ? 6 * I * T : 1];
    __shared__ int s_last;

    const float4 *P = static_cast<const float4 *>(p.P);
    const int n = p.n;
    const int n_itiles = (n + TILE_I - 1) / TILE_I;
    const int it = blockIdx.x % n_itiles;
    const int js = blockIdx.x / n_itiles;
    const int i0 = it * TILE_I;
    int t0, t1;
    split_range((n + J - 1) / J, p.nsplit, js, t0, t1);

    float2 nx[I / 2], ny[I / 2], nz[I / 2];
    const float3 c = load_i<T, I>(P, p.Plo, i0 + threadIdx.x, T, n, nx, ny, nz, red);
    Acc<T, I, COMP, KSM> acc;
    acc.init(ks);
    const float2 e2 = make_float2(p.eps2f, p.eps2f);
    sweep<T, I, J, COMP, ZEPS, LP, false, KSM, UNR>(
        P, p.Plo, c, 0, n, t0, t1, 0, 1, e2, nx, ny, nz, acc, tile);

    if (p.nsplit == 1) {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = i0 + threadIdx.x + k * T;
            if (i < n) {
                double x, y, z;
                acc.get(k, x, y, z);
                write_acc(p, p.perm ? p.perm[i] : i, p.G * x, p.G * y, p.G * z);
            }
        }
        return;
    }
    // Split: publish this CTA's partial, the last arriving CTA combines.
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        if (i < n) {
            double x, y, z;
            acc.get(k, x, y, z);
            double *q = p.partial + ((size_t)js * n + i) * 3;
            q[0] = x;
            q[1] = y;
            q[2] = z;
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
            write_acc(p, p.perm ? p.perm[i] : i, p.G * x, p.G * y, p.G * z);
        }
    }
    if (threadIdx.x == 0) p.counters[it] = 0u;
}

// ----------------------------------------------------------- batched kernel
// Final write of one body's acceleration from its float64 sum (G applied).
__device__ __forceinline__ void batch_write(const BatchParams &p, int i, double x, double y,
                                            double z)
{
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

// Persistent: each CTA pops items (largest cost first) from an atomic
// counter until the queue is empty, the GPU analogue of the paper's dynamic
// loop schedule (Sec. V-C, Table VI).  An item whose piece is split over
// j-chunks stores its float64 partial sums; the last chunk of the piece to
// arrive (arrival counter) adds the chunks in order and writes the result.
// The last CTA to finish resets the queue counters for the next launch;
// nothing waits.
template <int T, int I, int J, bool COMP, bool ZEPS, int LP>
__global__ void __launch_bounds__(T) force_f32_batched_kernel(const BatchParams p)
{
    constexpr int TILE_I = T * I;
    __shared__ __align__(16) float4 tile[2][Slots<LP>::W * J];
    __shared__ float red[6][T / 32];
    __shared__ BatchItem s_item;
    __shared__ int s_idx, s_last;
    const float2 e2 = make_float2(p.eps2f, p.eps2f);

    for (;;) {
        if (threadIdx.x == 0) {
            const int q = (int)atomicAdd(p.queue, 1u);
            s_idx = q;
            if (q < p.n_items) s_item = p.items[q];
        }
        __syncthreads();
        if (s_idx >= p.n_items) break;
        const BatchItem it = s_item;
        __syncthreads();  // everyone has read s_item before thread 0 may overwrite it

        const int lanes = it.lanes;
        const int lane = threadIdx.x & (lanes - 1);
        const int group = threadIdx.x / lanes;
        const int groups = T / lanes;
        float2 nx[I / 2], ny[I / 2], nz[I / 2];
        const float3 c = load_i<T, I>(p.P, p.Plo, it.i0 + group, groups, it.i_end, nx, ny, nz, red);
        Acc<T, I, COMP, false> acc;
        acc.init(nullptr);
        const int ntiles = (it.j1 - it.j0 + J - 1) / J;
        if (lanes == 1)
            sweep<T, I, J, COMP, ZEPS, LP, false, false, UNROLL_F32>(
                p.P, p.Plo, c, it.j0, it.j1, 0, ntiles, 0, 1, e2, nx, ny, nz, acc, tile);
        else
            sweep<T, I, J, COMP, ZEPS, LP, true, false, UNROLL_F32>(
                p.P, p.Plo, c, it.j0, it.j1, 0, ntiles, lane, lanes, e2, nx, ny, nz, acc, tile);
        const bool split = it.nchunks > 1;
        double *slot = split ? p.partial + (size_t)(it.pbase + it.chunk) * TILE_I * 3 : nullptr;
#pragma unroll
        for (int k = 0; k < I; ++k) {
            double x, y, z;
            acc.get(k, x, y, z);
            // lanes of a group are adjacent in one warp: butterfly sum
            for (int off = lanes >> 1; off > 0; off >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, off);
                y += __shfl_xor_sync(0xffffffffu, y, off);
                z += __shfl_xor_sync(0xffffffffu, z, off);
            }
            const int i = it.i0 + group + k * groups;
            if (lane == 0 && i < it.i_end) {
                if (split) {
                    double *q = slot + 3 * (size_t)(i - it.i0);
                    q[0] = x;
                    q[1] = y;
                    q[2] = z;
                } else {
                    batch_write(p, i, x, y, z);
                }
            }
        }
        if (split) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0)
                s_last = atomicAdd(p.counters + it.ctr, 1u) == (unsigned)(it.nchunks - 1);
            __syncthreads();
            if (s_last) {
                __threadfence();
                const double *base = p.partial + (size_t)it.pbase * TILE_I * 3;
                for (int q = threadIdx.x; q < it.i_end - it.i0; q += T) {
                    double x = 0.0, y = 0.0, z = 0.0;
                    for (int ch = 0; ch < it.nchunks; ++ch) {
                        const double *r = base + ((size_t)ch * TILE_I + q) * 3;
                        x += __ldcg(r);
                        y += __ldcg(r + 1);
                        z += __ldcg(r + 2);
                    }
                    batch_write(p, it.i0 + q, x, y, z);
                }
                if (threadIdx.x == 0) p.counters[it.ctr] = 0u;
            }
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(p.queue + 1, 1u) == gridDim.x - 1) {
            p.queue[0] = 0u;
            p.queue[1] = 0u;
            __threadfence();
        }
    }
}

#define NB_F32_KERNEL(T, I, J, C, Z, L, K, M, U) \
    {T, I, J, (const void *)force_f32_kernel<T, I, J, C, Z, L, K, M, U>, (L) > 0}
// [comp][zero_eps]; L = body pairs per thread in the log-domain form;
// K (Kahan state in shared memory) and M (register cap for M CTAs/SM) only
// change the compensated kernels; U = unroll depth of the j loop.
#define NB_F32_ENTRY_XU(T, I, J, L, K, M, U)                                               \
    {{NB_F32_KERNEL(T, I, J, false, false, L, false, 0, U),                                \
      NB_F32_KERNEL(T, I, J, false, true, L, false, 0, U)},                                \
     {NB_F32_KERNEL(T, I, J, true, false, L, K, M, U),                                     \
      NB_F32_KERNEL(T, I, J, true, true, L, K, M, U)}}
#define NB_F32_ENTRY_X(T, I, J, L, K, M) \
    NB_F32_ENTRY_XU(T, I, J, L, K, M, ((M) >= 4 ? 4 : UNROLL_F32))
#define NB_F32_ENTRY(T, I, J, L) NB_F32_ENTRY_X(T, I, J, L, false, 0)

#define NB_F32B_KERNEL(T, I, J, C, Z, L) \
    {T, I, J, (const void *)force_f32_batched_kernel<T, I, J, C, Z, L>, (L) > 0}
#define NB_F32B_ENTRY(T, I, J, L)                                                          \
    {{NB_F32B_KERNEL(T, I, J, false, false, L), NB_F32B_KERNEL(T, I, J, false, true, L)},   \
     {NB_F32B_KERNEL(T, I, J, true, false, L), NB_F32B_KERNEL(T, I, J, true, true, L)}}

typedef KernelEntry Quad[2][2];

}  // namespace
}  // namespace nb
