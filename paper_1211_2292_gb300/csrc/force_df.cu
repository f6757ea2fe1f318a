// Float64-accuracy force kernel on the float32 pipe ("double-float"): the
// exact all-pairs sum of the paper's force calculation (Sec. IV-A/IV-B), with
// every pair term carried as an unevaluated sum hi + lo of two float32
// numbers and formed with error-free transformations:
//   two_sum  (Knuth): s = fl(a + b), e = (a - (s - (s - a))) + (b - (s - a)),
//            s + e == a + b exactly;
//   two_prod (Dekker, with a fused multiply-add): p = fl(a b),
//            e = fma(a, b, -p), p + e == a b exactly.
// A double-float value carries about 48 significant bits (relative rounding
// ~2^-47 per operation) against float64's 53; on this part the float64 pipe
// is about 64x slower than the float32 one, so ~140 float32 operations per
// pair still run several times faster than ~19 float64 ones.
//
// Layout and schedule follow the float64 kernel: an i-tile of T*I bodies per
// CTA, j-bodies streamed through a double-buffered shared tile, the grid
// split over j with the last arriving CTA adding the float64 partials in split
// order.  Positions are float64 (double4 x,y,z,m) in Morton order; each CTA
// takes the centre of its i-tile's bounding box as origin c and forms, in
// float64, x - c for its i-bodies and c - x for the j-bodies before splitting
// them into hi/lo float32 pairs, so that close pairs (whose differences need
// the most digits) are represented to ~2^-48 of the tile's extent.  Two
// i-bodies share each float32x2 instruction.  Per j-tile the double-float sums
// are folded into float64 accumulators.
#include <cuda_runtime.h>
#include <float.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

// Unevaluated sums on float32x2 lanes (two i-bodies).
struct DF2 {
    float2 h, l;
};

// Negation as a sign change of both halves (the compiler can fold it into
// the consuming instruction's operand).
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// b - a, one rounding
__device__ __forceinline__ float2 sub_from(float2 a, float2 b) { return add2(b, neg2(a)); }

// s + e == a + b exactly (six operations, no ordering of |a|, |b| needed)
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = add2(a, b);
    const float2 bb = sub_from(a, s);  // s - a
    const float2 t = sub_from(bb, s);  // s - bb
    e = add2(sub_from(t, a), sub_from(bb, b));
}

// s + e == a + b exactly when |a| >= |b| or a == 0 (three operations)
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = add2(a, b);
    e = sub_from(sub_from(a, s), b);  // b - (s - a)
}

// (h, l) ~= (ah + al)(bh + bl), dropping al bl (at most ~2^-44 of the
// product, for y^3; keeping it, and dl^2 in r^2, changed no measured error)
__device__ __forceinline__ void df_mul2(float2 ah, float2 al, float2 bh, float2 bl, float2 &h,
                                        float2 &l)
{
    h = mul2(ah, bh);
    l = fma2(ah, bh, neg2(h));
    l = fma2(ah, bl, l);
    l = fma2(al, bh, l);
}

// Shared j-tile entry: c - x_j split into hi/lo, and m_j, each duplicated for
// the two float32x2 lanes: {xh,xh,yh,yh}, {zh,zh,mh,mh}, {xl,xl,yl,yl}, {zl,zl,ml,ml}.
template <int T, int J>
__device__ __forceinline__ void df_stage_load(double4 (&buf)[J / T], const double4 *__restrict__ P,
                                              int jbase, int jend)
{
#pragma unroll
    for (int l = 0; l < J / T; ++l) {
        const int j = jbase + l * T + threadIdx.x;
        buf[l] = j < jend ? P[j] : make_double4(0.0, 0.0, 0.0, 0.0);
    }
}

__device__ __forceinline__ void split_df(double v, float &h, float &l)
{
    h = (float)v;
    l = (float)(v - (double)h);
}

template <int T, int J>
__device__ __forceinline__ void df_stage_store(float4 (*tile)[4], const double4 (&buf)[J / T],
                                               double3 c)
{
#pragma unroll
    for (int l = 0; l < J / T; ++l) {
        float xh, xl, yh, yl, zh, zl, mh, ml;
        split_df(c.x - buf[l].x, xh, xl);
        split_df(c.y - buf[l].y, yh, yl);
        split_df(c.z - buf[l].z, zh, zl);
        split_df(buf[l].w, mh, ml);
        float4 *e = tile[l * T + threadIdx.x];
        e[0] = make_float4(xh, xh, yh, yh);
        e[1] = make_float4(zh, zh, mh, mh);
        e[2] = make_float4(xl, xl, yl, yl);
        e[3] = make_float4(zl, zl, ml, ml);
    }
}

// Accumulate m_j (x_i - x_j) / (|x_i - x_j|^2 + eps^2)^{3/2} onto the pair
// of i-bodies (the sign is the opposite of the acceleration; it is flipped
// at the end).
template <bool ZEPS>
__device__ __forceinline__ void df_pair(const float4 &A, const float4 &B, const float4 &C,
                                        const float4 &D, const DF2 (&xi)[3], float2 e2h,
                                        float2 e2l, DF2 (&acc)[3])
{
    const float2 one = make_float2(1.f, 1.f);
    // d = x_i - x_j = x_i + (c - x_j) - c, hi/lo, normalised
    const float2 njh[3] = {make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(B.x, B.y)};
    const float2 njl[3] = {make_float2(C.x, C.y), make_float2(C.z, C.w), make_float2(D.x, D.y)};
    DF2 d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 s, e;
        two_sum2(xi[c].h, njh[c], s, e);
        e = add2(e, add2(xi[c].l, njl[c]));
        fast_two_sum2(s, e, d[c].h, d[c].l);
    }
    // r^2 = |d|^2 + eps^2: exact squares of the hi parts, cross terms, exact
    // sums of the hi parts, then one renormalisation
    float2 p[3], pe[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        p[c] = mul2(d[c].h, d[c].h);
        pe[c] = fma2(d[c].h, d[c].h, neg2(p[c]));
        pe[c] = fma2(add2(d[c].h, d[c].h), d[c].l, pe[c]);
    }
    float2 r, er, t;
    two_sum2(p[0], p[1], r, er);
    two_sum2(r, p[2], r, t);
    er = add2(er, t);
    two_sum2(r, e2h, r, t);
    er = add2(er, add2(t, add2(add2(pe[0], pe[1]), add2(pe[2], e2l))));
    float2 R, E;
    fast_two_sum2(r, er, R, E);
    // y = 1/sqrt(R + E): float32 seed y0, then y = y0 (1 + e/2 + 3e^2/8) with
    // e = 1 - (R + E) y0^2 formed in double-float (error ~ (5/16) e^3)
    const float2 y0 = make_float2(rsqrt_mufu(R.x), rsqrt_mufu(R.y));
    const float2 q = mul2(y0, y0);
    const float2 qe = fma2(y0, y0, neg2(q));
    const float2 th = mul2(R, q);
    float2 tl = fma2(R, q, neg2(th));
    tl = fma2(R, qe, tl);
    tl = fma2(E, q, tl);
    float2 e = sub_from(th, one);  // 1 - th, exact (th ~ 1)
    e = sub_from(tl, e);
    const float2 corr = mul2(fma2(e, make_float2(0.375f, 0.375f), make_float2(0.5f, 0.5f)), e);
    const float2 yl = mul2(y0, corr);
    // y^2 = q + qe + 2 y0 yl + yl^2, then y^3 and s = m y^3
    float2 y2l = fma2(add2(y0, y0), yl, qe);
    y2l = fma2(yl, yl, y2l);
    float2 y3h, y3l;
    df_mul2(q, y2l, y0, yl, y3h, y3l);
    float2 sh, sl;
    df_mul2(make_float2(B.z, B.w), make_float2(D.z, D.w), y3h, y3l, sh, sl);
    if (ZEPS) {  // eps == 0: the self pair (R == 0) contributes nothing
        sh.x = R.x > 0.f ? sh.x : 0.f;
        sh.y = R.y > 0.f ? sh.y : 0.f;
        sl.x = R.x > 0.f ? sl.x : 0.f;
        sl.y = R.y > 0.f ? sl.y : 0.f;
    }
    // acc += s d, the hi parts summed error-free
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 ph, pl;
        df_mul2(sh, sl, d[c].h, d[c].l, ph, pl);
        float2 s2, e2;
        two_sum2(acc[c].h, ph, s2, e2);
        acc[c].h = s2;
        acc[c].l = add2(acc[c].l, add2(e2, pl));
    }
}

template <int T, int I, int J, bool ZEPS>
__global__ void __launch_bounds__(T) force_df_kernel(const ForceParams p)
{
    static_assert(I % 2 == 0, "i-bodies are taken in float32x2 pairs");
    constexpr int NP = I / 2, TILE_I = T * I;
    __shared__ __align__(16) float4 tile[2][J][4];
    __shared__ int s_last;
    const double4 *P = static_cast<const double4 *>(p.P);
    const int n = p.n;
    const int n_itiles = (n + TILE_I - 1) / TILE_I;
    const int it = blockIdx.x % n_itiles;
    const int js = blockIdx.x / n_itiles;
    const int i0 = it * TILE_I;
    int t0, t1;
    split_range((n + J - 1) / J, p.nsplit, js, t0, t1);

    // origin: the centre of the i-tile's bounding box (float64)
    __shared__ double red[6][T / 32];
    double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        if (i < n) {
            const double4 v = P[i];
            mn[0] = fmin(mn[0], v.x), mx[0] = fmax(mx[0], v.x);
            mn[1] = fmin(mn[1], v.y), mx[1] = fmax(mx[1], v.y);
            mn[2] = fmin(mn[2], v.z), mx[2] = fmax(mx[2], v.z);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            mn[k] = fmin(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], off));
            mx[k] = fmax(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], off));
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            red[k][threadIdx.x >> 5] = mn[k];
            red[3 + k][threadIdx.x >> 5] = mx[k];
        }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < T / 32; ++w)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            mn[k] = fmin(mn[k], red[k][w]);
            mx[k] = fmax(mx[k], red[3 + k][w]);
        }
    const double3 c = make_double3(0.5 * (mn[0] + mx[0]), 0.5 * (mn[1] + mx[1]),
                                   0.5 * (mn[2] + mx[2]));
    const double4 c4 = make_double4(c.x, c.y, c.z, 0.0);
    DF2 xi[NP][3];
    double ax[I], ay[I], az[I];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float h[2][3], l[2][3];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + threadIdx.x + (2 * q + b) * T;
            const double4 v = i < n ? P[i] : c4;
            split_df(v.x - c.x, h[b][0], l[b][0]);
            split_df(v.y - c.y, h[b][1], l[b][1]);
            split_df(v.z - c.z, h[b][2], l[b][2]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            xi[q][k].h = make_float2(h[0][k], h[1][k]);
            xi[q][k].l = make_float2(l[0][k], l[1][k]);
        }
    }
#pragma unroll
    for (int k = 0; k < I; ++k) ax[k] = ay[k] = az[k] = 0.0;
    float e2hs, e2ls;
    split_df(p.eps2, e2hs, e2ls);
    const float2 e2h = make_float2(e2hs, e2hs), e2l = make_float2(e2ls, e2ls);

    double4 buf[J / T];
    if (t0 < t1) {
        df_stage_load<T, J>(buf, P, t0 * J, n);
        df_stage_store<T, J>(tile[0], buf, c);
    }
    __syncthreads();
    for (int t = t0; t < t1; ++t) {
        const int bsel = (t - t0) & 1;
        if (t + 1 < t1) df_stage_load<T, J>(buf, P, (t + 1) * J, n);
        DF2 acc[NP][3];
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[q][k].h = acc[q][k].l = make_float2(0.f, 0.f);
        const float4(*s)[4] = tile[bsel];
#pragma unroll 2
        for (int jj = 0; jj < J; ++jj) {
            const float4 A = s[jj][0], B = s[jj][1], C = s[jj][2], D = s[jj][3];
#pragma unroll
            for (int q = 0; q < NP; ++q) df_pair<ZEPS>(A, B, C, D, xi[q], e2h, e2l, acc[q]);
        }
        // fold the tile's double-float sums (of -a) into float64
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            ax[2 * q] -= (double)acc[q][0].h.x + (double)acc[q][0].l.x;
            ay[2 * q] -= (double)acc[q][1].h.x + (double)acc[q][1].l.x;
            az[2 * q] -= (double)acc[q][2].h.x + (double)acc[q][2].l.x;
            ax[2 * q + 1] -= (double)acc[q][0].h.y + (double)acc[q][0].l.y;
            ay[2 * q + 1] -= (double)acc[q][1].h.y + (double)acc[q][1].l.y;
            az[2 * q + 1] -= (double)acc[q][2].h.y + (double)acc[q][2].l.y;
        }
        if (t + 1 < t1) df_stage_store<T, J>(tile[bsel ^ 1], buf, c);
        __syncthreads();
    }

    auto emit = [&](int k, double x, double y, double z) {
        const int slot = i0 + threadIdx.x + k * T;
        const int i = p.perm ? p.perm[slot] : slot;
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
    };
    if (p.nsplit == 1) {
#pragma unroll
        for (int k = 0; k < I; ++k)
            if (i0 + threadIdx.x + k * T < n) emit(k, ax[k], ay[k], az[k]);
        return;
    }
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        if (i < n) {
            double *r = p.partial + ((size_t)js * n + i) * 3;
            r[0] = ax[k];
            r[1] = ay[k];
            r[2] = az[k];
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
            emit(k, x, y, z);
        }
    }
    if (threadIdx.x == 0) p.counters[it] = 0u;
}

#define NB_DF_ENTRY(T, I, J)                                            \
    {{T, I, J, (const void *)force_df_kernel<T, I, J, false>},          \
     {T, I, J, (const void *)force_df_kernel<T, I, J, true>}}

typedef KernelEntry Pair[2];
// Tiles of at most 256 bodies: a close pair's difference is carried to
// ~2^-48 of the tile's extent, so smaller (Morton-compact) tiles are more
// accurate; 512-body tiles reached 2e-12 at N = 3001 and are not offered.
const Pair kDF[] = {
    NB_DF_ENTRY(128, 2, 128),
    NB_DF_ENTRY(64, 4, 128),
    NB_DF_ENTRY(64, 2, 128),
};

}  // namespace

int df_force_variants() { return (int)(sizeof(kDF) / sizeof(kDF[0])); }
const KernelEntry &df_force_kernel(int v, bool zeps) { return kDF[v][zeps]; }

}  // namespace nb
