// Force vector-Jacobian product (no counterpart in the paper; it follows
// from differentiating the softened force).  For cotangent mu = dL/da, with
// d_kj = x_j - x_k, s = sqrt(|d|^2 + eps^2), K(d) = I/s^3 - 3 d d^T/s^5:
//
//   gx_k = G sum_j K(d_kj) (m_k mu_j - m_j mu_k)
//        = G sum_j [ w/s^3 - 3 d (d.w)/s^5 ],      w = m_k mu_j - m_j mu_k
//   gm_k = G sum_j mu_j . (x_k - x_j) / s^3  =  -G sum_j (mu_j . d_kj)/s^3
//
// Schedule as in the force kernels: i-tile in registers, j-tiles through
// double-buffered shared memory, j-split across CTAs with an ordered
// last-CTA combine.
//
// float32 kernel (vjp_f32_kernel): float32x2 lanes over pairs of i-bodies,
// positions as hi/lo pairs in coordinates relative to the i-tile's centre
// (as in the force kernel).  With b = w - 3 d (d.w)/s^2 the lane accumulates
//   B_k = sum_j b/s^3,  gx_k = G B_k,   M_k = sum_j (mu_j . d)/s^3,  gm_k = -G M_k.
// Scaled form: w/m_k = mu_j - m_j v_k with v_k = mu_k/m_k formed once per
// i-body, 26 float32 operations (13 float32x2 issues) and one rsqrt per pair,
// the factor m_k applied to the float64 total.  Direct form (bodies of zero
// mass, or a tile whose scaled sums overflow): w = m_k mu_j - m_j mu_k, 29
// operations.  Both keep the difference per pair; splitting w into
// m_k sum mu_j/s^3 - mu_k sum m_j/s^3 would round against large coherent sums
// when w is small, as for smooth cotangent fields.  The self pair is masked
// out exactly in the j-tiles that overlap the CTA's own bodies, since the
// pair's w is a rounding residue that 1/eps^3 would magnify.  Each tile's
// float32 partials are added into float64 totals; the j-splits divide the
// bodies (not the tiles) evenly.
//
// float64 kernel (vjp_kernel<double>): the direct form above, all float64.
#include <cuda_runtime.h>

#include "nb_device.cuh"
#include "nb_internal.h"

namespace nb {
namespace {

template <typename R>
struct V4;
template <>
struct V4<float> {
    typedef float4 type;
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static float rsq(float x) { return rsqrt_mufu(x); }
};
template <>
struct V4<double> {
    typedef double4 type;
    __device__ static double4 zero() { return make_double4(0.0, 0.0, 0.0, 0.0); }
    __device__ static double rsq(double x) { return rsqrt_f64(x); }
};

template <typename R, int T, int I, int J, bool ZEPS>
__global__ void __launch_bounds__(T) vjp_kernel(const VjpParams p)
{
    typedef typename V4<R>::type V;
    constexpr int TILE_I = T * I;
    constexpr int LPT = J / T;
    __shared__ __align__(16) V tile[2][2 * J];
    __shared__ int s_last;

    const V *PV = static_cast<const V *>(p.PV);
    const int n = p.n;
    const int n_itiles = (n + TILE_I - 1) / TILE_I;
    const int it = blockIdx.x % n_itiles;
    const int js = blockIdx.x / n_itiles;
    const int i0 = it * TILE_I;
    int t0, t1;
    split_range((n + J - 1) / J, p.nsplit, js, t0, t1);
    const R e2 = sizeof(R) == 4 ? (R)p.eps2f : (R)p.eps2;

    R xk[I], yk[I], zk[I], mk[I], lx[I], ly[I], lz[I];
    R px[I], py[I], pz[I], pm[I];       // tile partials
    double gx[I], gy[I], gz[I], gm[I];  // float64 totals
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        const V a = i < n ? PV[2 * (size_t)i] : V4<R>::zero();
        const V b = i < n ? PV[2 * (size_t)i + 1] : V4<R>::zero();
        xk[k] = a.x; yk[k] = a.y; zk[k] = a.z; mk[k] = a.w;
        lx[k] = b.x; ly[k] = b.y; lz[k] = b.z;
        gx[k] = gy[k] = gz[k] = gm[k] = 0.0;
    }

    V buf[2 * LPT];
    auto gload = [&](int t) {
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int j = t * J + l * T + threadIdx.x;
            buf[2 * l] = j < n ? PV[2 * (size_t)j] : V4<R>::zero();
            buf[2 * l + 1] = j < n ? PV[2 * (size_t)j + 1] : V4<R>::zero();
        }
    };
    auto sstore = [&](int b) {
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int jj = l * T + threadIdx.x;
            tile[b][2 * jj] = buf[2 * l];
            tile[b][2 * jj + 1] = buf[2 * l + 1];
        }
    };
    if (t0 < t1) {
        gload(t0);
        sstore(0);
    }
    __syncthreads();
    for (int t = t0; t < t1; ++t) {
        const int b = (t - t0) & 1;
        if (t + 1 < t1) gload(t + 1);
#pragma unroll
        for (int k = 0; k < I; ++k) px[k] = py[k] = pz[k] = pm[k] = (R)0;
        const V *s = tile[b];
#pragma unroll 4
        for (int jj = 0; jj < J; ++jj) {
            const V q = s[2 * jj], u = s[2 * jj + 1];
#pragma unroll
            for (int k = 0; k < I; ++k) {
                const R dx = q.x - xk[k], dy = q.y - yk[k], dz = q.z - zk[k];
                R r2 = dx * dx + e2;
                r2 = dy * dy + r2;
                r2 = dz * dz + r2;
                R ri = V4<R>::rsq(r2);
                if (ZEPS) ri = r2 > (R)0 ? ri : (R)0;
                const R ri2 = ri * ri;
                const R ri3 = ri2 * ri;
                const R q5 = ri3 * ri2;
                const R wx = mk[k] * u.x - q.w * lx[k];
                const R wy = mk[k] * u.y - q.w * ly[k];
                const R wz = mk[k] * u.z - q.w * lz[k];
                const R dw = dx * wx + dy * wy + dz * wz;
                const R c = (R)3 * dw * q5;
                px[k] += wx * ri3 - dx * c;
                py[k] += wy * ri3 - dy * c;
                pz[k] += wz * ri3 - dz * c;
                pm[k] -= (u.x * dx + u.y * dy + u.z * dz) * ri3;
            }
        }
#pragma unroll
        for (int k = 0; k < I; ++k) {
            gx[k] += (double)px[k];
            gy[k] += (double)py[k];
            gz[k] += (double)pz[k];
            gm[k] += (double)pm[k];
        }
        if (t + 1 < t1) sstore(b ^ 1);
        __syncthreads();
    }

    auto emit = [&](int i, double x, double y, double z, double m) {
        x *= p.G; y *= p.G; z *= p.G; m *= p.G;
        double *o = p.gx + 3 * (size_t)i;
        if (p.accumulate) {
            o[0] += x; o[1] += y; o[2] += z;
            p.gm[i] += m;
        } else {
            o[0] = x; o[1] = y; o[2] = z;
            p.gm[i] = m;
        }
        if (!(finite3(x, y, z) && isfinite(m))) atomicOr(p.err, ERR_NONFINITE);
    };
    if (p.nsplit == 1) {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = i0 + threadIdx.x + k * T;
            if (i < n) emit(i, gx[k], gy[k], gz[k], gm[k]);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        if (i < n) {
            double *q = p.partial + ((size_t)js * n + i) * 4;
            q[0] = gx[k]; q[1] = gy[k]; q[2] = gz[k]; q[3] = gm[k];
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
            double x = 0.0, y = 0.0, z = 0.0, m = 0.0;
            for (int q = 0; q < p.nsplit; ++q) {
                const double *r = p.partial + ((size_t)q * n + i) * 4;
                x += __ldcg(r); y += __ldcg(r + 1); z += __ldcg(r + 2); m += __ldcg(r + 3);
            }
            emit(i, x, y, z, m);
        }
    }
    if (threadIdx.x == 0) p.counters[it] = 0u;
}


// ------------------------------------------------------ float32x2 kernel
template <int T, int J>
__device__ __forceinline__ void vjp_stage_load(float4 (&bh)[J / T], float4 (&bl)[J / T],
                                               float4 (&bu)[J / T], const float4 *__restrict__ Ph,
                                               const float4 *__restrict__ Pl,
                                               const float4 *__restrict__ Pu, int jbase, int jend)
{
#pragma unroll
    for (int l = 0; l < J / T; ++l) {
        const int j = jbase + l * T + threadIdx.x;
        const bool ok = j < jend;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        bh[l] = ok ? __ldg(Ph + j) : z;
        bl[l] = ok ? __ldg(Pl + j) : z;
        bu[l] = ok ? __ldg(Pu + j) : z;
    }
}

// Shared layout per j: (x,x,y,y), (z,z,m,m), (ux,ux,uy,uy), (uz,uz,0,0).
template <int T, int J>
__device__ __forceinline__ void vjp_stage_store(float4 *tile, const float4 (&bh)[J / T],
                                                const float4 (&bl)[J / T],
                                                const float4 (&bu)[J / T], float3 c)
{
#pragma unroll
    for (int l = 0; l < J / T; ++l) {
        const int jj = l * T + threadIdx.x;
        const float x = rel(bh[l].x, bl[l].x, c.x);
        const float y = rel(bh[l].y, bl[l].y, c.y);
        const float z = rel(bh[l].z, bl[l].z, c.z);
        tile[4 * jj] = make_float4(x, x, y, y);
        tile[4 * jj + 1] = make_float4(z, z, bh[l].w, bh[l].w);
        tile[4 * jj + 2] = make_float4(bu[l].x, bu[l].x, bu[l].y, bu[l].y);
        tile[4 * jj + 3] = make_float4(bu[l].z, bu[l].z, 0.f, 0.f);
    }
}

// Per-pair-lane state of the float32 VJP: sum b/s^3 (three components) and
// sum (mu_j . d)/s^3.
template <int NP>
struct VjpAcc {
    float2 gx[NP], gy[NP], gz[NP], gm[NP];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int p = 0; p < NP; ++p) gx[p] = gy[p] = gz[p] = gm[p] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ bool finite(int p) const
    {
        const float2 s = add2(add2(gx[p], gy[p]), add2(gz[p], gm[p]));
        return isfinite(s.x) && isfinite(s.y);
    }
};

// One j-body against a float32x2 lane of two i-bodies: with the pair weight w,
// b = w - 3 d (d.w)/s^2 and the lane adds b/s^3 and (mu_j . d)/s^3.
//   GEN (direct form):  w = m_k mu_j - m_j mu_k, from sk = -mu_k
//       (29 float32 operations);
//   else (scaled form): w = mu_j - m_j v_k with v_k = mu_k/m_k, from
//       sk = -v_k: the same weight over m_k, which the caller multiplies
//       back (26 float32 operations).
// Both keep the difference per pair, so a smooth cotangent field (small w)
// loses nothing to cancellation.
template <bool ZEPS, bool MASK, bool GEN>
__device__ __forceinline__ void vjp_pair(float2 xj, float2 yj, float2 zj, float2 mj, float2 ujx,
                                         float2 ujy, float2 ujz, float2 e2, float2 nx, float2 ny,
                                         float2 nz, float2 mk, float2 skx, float2 sky, float2 skz,
                                         bool self_a, bool self_b, float2 &gx, float2 &gy,
                                         float2 &gz, float2 &gm)
{
    const float2 dx = add2(xj, nx), dy = add2(yj, ny), dz = add2(zj, nz);
    float2 r2 = fma2(dx, dx, e2);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    float2 ri;
    ri.x = rsqrt_mufu(r2.x);
    ri.y = rsqrt_mufu(r2.y);
    if (ZEPS) {
        ri.x = r2.x > 0.f ? ri.x : 0.f;
        ri.y = r2.y > 0.f ? ri.y : 0.f;
    }
    if (MASK) {  // the self pair j == k contributes nothing
        ri.x = self_a ? 0.f : ri.x;
        ri.y = self_b ? 0.f : ri.y;
    }
    const float2 ri2 = mul2(ri, ri);
    const float2 ri3 = mul2(ri2, ri);
    const float2 m3ri2 = mul2(ri2, make_float2(-3.f, -3.f));
    float2 wx, wy, wz;
    if (GEN) {
        wx = fma2(mk, ujx, mul2(mj, skx));
        wy = fma2(mk, ujy, mul2(mj, sky));
        wz = fma2(mk, ujz, mul2(mj, skz));
    } else {
        wx = fma2(mj, skx, ujx);
        wy = fma2(mj, sky, ujy);
        wz = fma2(mj, skz, ujz);
    }
    float2 dw = mul2(dx, wx);
    dw = fma2(dy, wy, dw);
    dw = fma2(dz, wz, dw);
    const float2 t = mul2(dw, m3ri2);
    gx = fma2(fma2(dx, t, wx), ri3, gx);
    gy = fma2(fma2(dy, t, wy), ri3, gy);
    gz = fma2(fma2(dz, t, wz), ri3, gz);
    float2 dlj = mul2(dx, ujx);
    dlj = fma2(dy, ujy, dlj);
    dlj = fma2(dz, ujz, dlj);
    gm = fma2(dlj, ri3, gm);
}

// Float64 totals of the four sums per body: in registers, or (TSM) in
// shared memory, touched once per j-tile, which frees 8 * I registers for
// more resident warps.
template <int T, int I, bool TSM>
struct VjpTotals {
    double reg[TSM ? 1 : 4][TSM ? 1 : I];
    double *sh;  // this CTA's [4][I][T] doubles (TSM only)
    __device__ __forceinline__ double &at(int r, int k)
    {
        return TSM ? sh[(r * I + k) * T + threadIdx.x] : reg[TSM ? 0 : r][TSM ? 0 : k];
    }
};

// The CTA takes the scaled form (totals in units of m_k) unless one of its
// bodies has m_k <= 0 or a non-finite mu_k/m_k; then every tile takes the
// direct form (totals in absolute units).  A lane whose scaled tile sums are
// not finite (m_j mu_k/m_k beyond the float32 range) evaluates that tile
// again in the direct form and adds it divided by m_k.
template <int T, int I, int J, bool ZEPS, bool TSM = false, int MINB = 0>
__global__ void __launch_bounds__(T, MINB) vjp_f32_kernel(const VjpParams p)
{
    static_assert(I % 2 == 0 && J % T == 0, "bad tile shape");
    constexpr int NP = I / 2;
    constexpr int TILE_I = T * I;
    constexpr int LPT = J / T;
    __shared__ __align__(16) float4 tile[2][4 * J];
    __shared__ float red[6][T / 32];
    __shared__ double tsh[TSM ? 4 * I * T : 1];
    __shared__ int s_last;

    const float4 *Ph = static_cast<const float4 *>(p.PV);
    const float4 *Pl = p.Plo, *Pu = p.Plam;
    const int n = p.n;
    const int n_itiles = (n + TILE_I - 1) / TILE_I;
    const int it = blockIdx.x % n_itiles;
    const int js = blockIdx.x / n_itiles;
    const int i0 = it * TILE_I;
    // j-split js covers bodies [jbeg, jend): equal shares to the body, so that
    // the CTAs of one wave carry equal work; its last tile is zero-padded to
    // a multiple of the tile loop's step (8 bodies for I = 2, else 4)
    const int jbeg = (int)(((long long)n * js) / p.nsplit);
    const int jend = (int)(((long long)n * (js + 1)) / p.nsplit);
    const int ntl = (jend - jbeg + J - 1) / J;

    // the first j-tile's loads are in flight while the i-bodies are read
    float4 bh[LPT], bl[LPT], bu[LPT];
    if (ntl > 0) vjp_stage_load<T, J>(bh, bl, bu, Ph, Pl, Pu, jbeg, jend);

    // i-bodies: k-th body of the thread is i0 + tid + k*T; pair q = (2q, 2q+1)
    float2 nx[NP], ny[NP], nz[NP], skx[NP], sky[NP], skz[NP];
    float3 c;
    bool gen;
    {
        float4 h[I], l[I], u[I];
        float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        bool bad = false;
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = i0 + threadIdx.x + k * T;
            const bool ok = i < n;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            h[k] = ok ? __ldg(Ph + i) : z;
            l[k] = ok ? __ldg(Pl + i) : z;
            u[k] = ok ? __ldg(Pu + i) : z;
            if (ok) {
                mn[0] = fminf(mn[0], h[k].x); mx[0] = fmaxf(mx[0], h[k].x);
                mn[1] = fminf(mn[1], h[k].y); mx[1] = fmaxf(mx[1], h[k].y);
                mn[2] = fminf(mn[2], h[k].z); mx[2] = fmaxf(mx[2], h[k].z);
                const float m = h[k].w;
                bad |= !(m > 0.f && isfinite(u[k].x / m) && isfinite(u[k].y / m) &&
                         isfinite(u[k].z / m));
            }
        }
        gen = __syncthreads_or(bad) != 0;
        c = block_center<T>(mn, mx, red);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int a = 2 * q, b = 2 * q + 1;
            nx[q] = make_float2(-rel(h[a].x, l[a].x, c.x), -rel(h[b].x, l[b].x, c.x));
            ny[q] = make_float2(-rel(h[a].y, l[a].y, c.y), -rel(h[b].y, l[b].y, c.y));
            nz[q] = make_float2(-rel(h[a].z, l[a].z, c.z), -rel(h[b].z, l[b].z, c.z));
            if (gen) {
                skx[q] = make_float2(-u[a].x, -u[b].x);
                sky[q] = make_float2(-u[a].y, -u[b].y);
                skz[q] = make_float2(-u[a].z, -u[b].z);
            } else {  // padding bodies (zero mass and cotangent) take sk = 0
                const float ma = h[a].w > 0.f ? h[a].w : 1.f, mb = h[b].w > 0.f ? h[b].w : 1.f;
                skx[q] = make_float2(-(u[a].x / ma), -(u[b].x / mb));
                sky[q] = make_float2(-(u[a].y / ma), -(u[b].y / mb));
                skz[q] = make_float2(-(u[a].z / ma), -(u[b].z / mb));
            }
        }
    }
    const float2 e2 = make_float2(p.eps2f, p.eps2f);
    VjpAcc<NP> acc;
    VjpTotals<T, I, TSM> tot;
    tot.sh = tsh;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < I; ++k) tot.at(q, k) = 0.0;

    if (ntl > 0) vjp_stage_store<T, J>(tile[0], bh, bl, bu, c);
    __syncthreads();
    for (int t = 0; t < ntl; ++t) {
        const int bsel = t & 1;
        if (t + 1 < ntl) vjp_stage_load<T, J>(bh, bl, bu, Ph, Pl, Pu, jbeg + (t + 1) * J, jend);
        acc.zero();
        const float4 *s = tile[bsel];
        const int jb = jbeg + t * J;
        // zero-padded bodies add nothing; the tile loop takes U bodies at a time
        constexpr int U = I == 2 ? 8 : 4;
        const int jn = min(J, (jend - jb + U - 1) & ~(U - 1));
        const bool self_tile = jb < i0 + TILE_I && i0 < jb + J;
        if (!gen && self_tile) {
#pragma unroll 2
            for (int jj = 0; jj < jn; ++jj) {
                const float4 q0 = s[4 * jj], q1 = s[4 * jj + 1], q2 = s[4 * jj + 2],
                             q3 = s[4 * jj + 3];
                const int jg = jb + jj;
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    const int ia = i0 + threadIdx.x + 2 * q * T;
                    vjp_pair<ZEPS, true, false>(
                        make_float2(q0.x, q0.y), make_float2(q0.z, q0.w),
                        make_float2(q1.x, q1.y), make_float2(q1.z, q1.w),
                        make_float2(q2.x, q2.y), make_float2(q2.z, q2.w),
                        make_float2(q3.x, q3.y), e2, nx[q], ny[q], nz[q], e2, skx[q], sky[q],
                        skz[q], jg == ia, jg == ia + T, acc.gx[q], acc.gy[q], acc.gz[q],
                        acc.gm[q]);
                }
            }
        } else if (!gen) {
            for (int j4 = 0; j4 < jn; j4 += U) {
#pragma unroll
                for (int jj = j4; jj < j4 + U; ++jj) {
                    const float4 q0 = s[4 * jj], q1 = s[4 * jj + 1], q2 = s[4 * jj + 2],
                                 q3 = s[4 * jj + 3];
#pragma unroll
                    for (int q = 0; q < NP; ++q)
                        vjp_pair<ZEPS, false, false>(
                            make_float2(q0.x, q0.y), make_float2(q0.z, q0.w),
                            make_float2(q1.x, q1.y), make_float2(q1.z, q1.w),
                            make_float2(q2.x, q2.y), make_float2(q2.z, q2.w),
                            make_float2(q3.x, q3.y), e2, nx[q], ny[q], nz[q], e2, skx[q],
                            sky[q], skz[q], false, false, acc.gx[q], acc.gy[q], acc.gz[q],
                            acc.gm[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            if (!gen && acc.finite(q)) {
                const float2 *v[4] = {&acc.gx[q], &acc.gy[q], &acc.gz[q], &acc.gm[q]};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    tot.at(r, 2 * q) += (double)v[r]->x;
                    tot.at(r, 2 * q + 1) += (double)v[r]->y;
                }
                continue;
            }
            // the direct form for this lane and tile
            const int ia = i0 + threadIdx.x + 2 * q * T, ib = ia + T;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 ua = ia < n ? __ldg(Pu + ia) : z, ub = ib < n ? __ldg(Pu + ib) : z;
            const float ma = ia < n ? __ldg(Ph + ia).w : 0.f, mb = ib < n ? __ldg(Ph + ib).w : 0.f;
            const float2 mk = make_float2(ma, mb);
            const float2 ukx = make_float2(-ua.x, -ub.x), uky = make_float2(-ua.y, -ub.y),
                         ukz = make_float2(-ua.z, -ub.z);
            float2 g0 = make_float2(0.f, 0.f), g1 = g0, g2 = g0, g3 = g0;
            for (int jj = 0; jj < jn; ++jj) {
                const float4 q0 = s[4 * jj], q1 = s[4 * jj + 1], q2 = s[4 * jj + 2],
                             q3 = s[4 * jj + 3];
                const int jg = jb + jj;
                vjp_pair<ZEPS, true, true>(make_float2(q0.x, q0.y), make_float2(q0.z, q0.w),
                                           make_float2(q1.x, q1.y), make_float2(q1.z, q1.w),
                                           make_float2(q2.x, q2.y), make_float2(q2.z, q2.w),
                                           make_float2(q3.x, q3.y), e2, nx[q], ny[q], nz[q], mk,
                                           ukx, uky, ukz, jg == ia, jg == ib, g0, g1, g2, g3);
            }
            // units of the CTA's totals: m_k (scaled form) or absolute
            const double sa = gen || !(ma > 0.f) ? 1.0 : 1.0 / (double)ma;
            const double sb = gen || !(mb > 0.f) ? 1.0 : 1.0 / (double)mb;
            tot.at(0, 2 * q) += (double)g0.x * sa;
            tot.at(1, 2 * q) += (double)g1.x * sa;
            tot.at(2, 2 * q) += (double)g2.x * sa;
            tot.at(3, 2 * q) += (double)g3.x;
            tot.at(0, 2 * q + 1) += (double)g0.y * sb;
            tot.at(1, 2 * q + 1) += (double)g1.y * sb;
            tot.at(2, 2 * q + 1) += (double)g2.y * sb;
            tot.at(3, 2 * q + 1) += (double)g3.y;
        }
        if (t + 1 < ntl) vjp_stage_store<T, J>(tile[bsel ^ 1], bh, bl, bu, c);
        __syncthreads();
    }

    // gx = G m_k sum b/s^3 (G sum b/s^3 in the direct form), gm = -G M
    auto emit = [&](int i, const double *sums) {
        const double f = gen ? p.G : p.G * (double)__ldg(Ph + i).w;
        const double x = f * sums[0], y = f * sums[1], z = f * sums[2];
        const double g = -p.G * sums[3];
        double *o = p.gx + 3 * (size_t)i;
        if (p.accumulate) {
            o[0] += x; o[1] += y; o[2] += z;
            p.gm[i] += g;
        } else {
            o[0] = x; o[1] = y; o[2] = z;
            p.gm[i] = g;
        }
        if (!(finite3(x, y, z) && isfinite(g))) atomicOr(p.err, ERR_NONFINITE);
    };
    if (p.nsplit == 1) {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = i0 + threadIdx.x + k * T;
            if (i < n) {
                double sums[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) sums[r] = tot.at(r, k);
                emit(i, sums);
            }
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        if (i < n) {
            double2 *q = reinterpret_cast<double2 *>(p.partial + ((size_t)js * n + i) * 4);
            q[0] = make_double2(tot.at(0, k), tot.at(1, k));
            q[1] = make_double2(tot.at(2, k), tot.at(3, k));
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(p.counters + it, 1u) == (unsigned)(p.nsplit - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // The splits' sums in split order; the loads of several splits and both
    // bodies are in flight together (this runs at the end of the launch).
    double sums[I][4];
#pragma unroll
    for (int k = 0; k < I; ++k) sums[k][0] = sums[k][1] = sums[k][2] = sums[k][3] = 0.0;
#pragma unroll 4
    for (int q = 0; q < p.nsplit; ++q) {
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = min(i0 + threadIdx.x + k * T, n - 1);  // rows past n: not emitted
            const double2 *r =
                reinterpret_cast<const double2 *>(p.partial + ((size_t)q * n + i) * 4);
            const double2 a = __ldcg(r), b = __ldcg(r + 1);
            sums[k][0] += a.x; sums[k][1] += a.y; sums[k][2] += b.x; sums[k][3] += b.y;
        }
    }
#pragma unroll
    for (int k = 0; k < I; ++k) {
        const int i = i0 + threadIdx.x + k * T;
        if (i < n) emit(i, sums[k]);
    }
    if (threadIdx.x == 0) p.counters[it] = 0u;
}

#define NB_VJP_ENTRY(R, T, I, J)                                       \
    {{T, I, J, (const void *)vjp_kernel<R, T, I, J, false>},           \
     {T, I, J, (const void *)vjp_kernel<R, T, I, J, true>}}

typedef KernelEntry Pair[2];
#define NB_VJP32_ENTRY_X(T, I, J, S, M)                                   \
    {{T, I, J, (const void *)vjp_f32_kernel<T, I, J, false, S, M>},       \
     {T, I, J, (const void *)vjp_f32_kernel<T, I, J, true, S, M>}}
#define NB_VJP32_ENTRY(T, I, J) NB_VJP32_ENTRY_X(T, I, J, false, 0)

const Pair kVjp32[] = {
    NB_VJP32_ENTRY(128, 2, 128),
    NB_VJP32_ENTRY(128, 4, 128),
    NB_VJP32_ENTRY(256, 2, 256),
    NB_VJP32_ENTRY(64, 4, 128),
    NB_VJP32_ENTRY(128, 4, 256),
    // float64 totals in shared memory, registers capped for 5-6 CTAs/SM (5..8)
    NB_VJP32_ENTRY_X(128, 2, 128, true, 5),
    NB_VJP32_ENTRY_X(128, 2, 128, true, 6),
    NB_VJP32_ENTRY_X(64, 2, 64, true, 12),
    NB_VJP32_ENTRY_X(64, 2, 128, true, 10),
    // shorter j-tiles and smaller CTAs with totals in registers (9..10)
    NB_VJP32_ENTRY(64, 2, 64),
    NB_VJP32_ENTRY(64, 2, 128),
    // float64 totals in shared memory, 7 or 8 CTAs/SM (11..12); four bodies
    // per thread at 4 CTAs/SM (13)
    NB_VJP32_ENTRY_X(128, 2, 128, true, 7),
    NB_VJP32_ENTRY_X(128, 2, 128, true, 8),
    NB_VJP32_ENTRY_X(128, 4, 128, true, 4),
};
const Pair kVjp64[] = {
    NB_VJP_ENTRY(double, 128, 1, 128),
    NB_VJP_ENTRY(double, 128, 2, 128),
};

}  // namespace

int f32_vjp_variants() { return (int)(sizeof(kVjp32) / sizeof(kVjp32[0])); }
const KernelEntry &f32_vjp_kernel(int v, bool zeps) { return kVjp32[v][zeps]; }
int f64_vjp_variants() { return (int)(sizeof(kVjp64) / sizeof(kVjp64[0])); }
const KernelEntry &f64_vjp_kernel(int v, bool zeps) { return kVjp64[v][zeps]; }

}  // namespace nb
