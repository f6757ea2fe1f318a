/*
 * FP64 CPU oracle for the softened direct-sum n-body force path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and
 * the benchmark's CPU-baseline leg may load this file's library.  It shares
 * no code, header or constant with the CUDA library and must never be used
 * as a fallback for it.
 *
 * What it computes (the paper's n-body step, Sec. IV and the hybrid
 * pseudo-code of Sec. IV-B):
 *   - the force calculation, which the paper says takes upwards of 90% of the
 *     cycles (Sec. IV-B), done here as the exact all-pairs sum that the
 *     paper's tree code approximates (Sec. IV-A);
 *   - "Move_bodies": the position/velocity update of Sec. IV-A, read as a
 *     kick-drift-kick leapfrog with cached forces;
 *   - energy and momentum diagnostics, and the adjoint (vector-Jacobian
 *     product) of the force and of the leapfrog, which the paper does not
 *     have; they follow from differentiating the same formulas.
 *
 * Readings where the paper is silent (Sec. IV names only "mutual gravitation
 * field"): Plummer-softened Newtonian gravity with constant G and softening
 * eps,   a_i = G sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^{3/2},
 * self pair excluded; potential energy -G sum_{i<j} m_i m_j / sqrt(r^2+eps^2).
 *
 * The loops follow the plain definition: i outer, j ascending inner, no
 * blocking.  The i loop is shared among OpenMP threads with a dynamic
 * schedule, the intra-node scheme the paper uses for its force loop
 * (Sec. IV-B pseudo-code, Sec. V-C / Table VI).  Each i is independent, so
 * the result does not depend on the thread count.
 *
 * Arrays: positions/velocities/accelerations are row-major (n,3) doubles,
 * masses (n) doubles; all caller-owned host memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_CHUNK 32

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Acceleration of body i (softened direct sum, self pair skipped). */
static void accel_one(int64_t n, const double *x, const double *m, double G,
                      double eps, int64_t i, double out[3])
{
    double ax = 0.0, ay = 0.0, az = 0.0;
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx = x[3 * j] - xi;
        double dy = x[3 * j + 1] - yi;
        double dz = x[3 * j + 2] - zi;
        double s2 = dx * dx + dy * dy + dz * dz + eps * eps;
        double inv_s3 = 1.0 / (s2 * sqrt(s2));
        ax += m[j] * dx * inv_s3;
        ay += m[j] * dy * inv_s3;
        az += m[j] * dz * inv_s3;
    }
    out[0] = G * ax;
    out[1] = G * ay;
    out[2] = G * az;
}

/* a_i for every body. */
void oracle_accel(int64_t n, const double *x, const double *m, double G,
                  double eps, double *acc)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, ORACLE_CHUNK)
    for (i = 0; i < n; ++i) accel_one(n, x, m, G, eps, i, acc + 3 * i);
}

/* a_i for the listed bodies only: acc is (nrows,3), row r is body rows[r]. */
void oracle_accel_rows(int64_t n, const double *x, const double *m, double G,
                       double eps, int64_t nrows, const int64_t *rows,
                       double *acc)
{
    int64_t r;
#pragma omp parallel for schedule(dynamic, ORACLE_CHUNK)
    for (r = 0; r < nrows; ++r) accel_one(n, x, m, G, eps, rows[r], acc + 3 * r);
}

/*
 * Diagnostics: out = {E_kin, E_pot, E_tot, P_x, P_y, P_z, F_x, F_y, F_z}
 * with E_kin = 1/2 sum m|v|^2, E_pot = -G sum_{i<j} m_i m_j / s_ij,
 * P = sum m v and F = sum m a (zero by Newton's third law).
 */
void oracle_energy(int64_t n, const double *x, const double *v,
                   const double *m, double G, double eps, double *out)
{
    double *phi = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *acc = (double *)calloc((size_t)(n > 0 ? 3 * n : 1), sizeof(double));
    int64_t i;
#pragma omp parallel for schedule(dynamic, ORACLE_CHUNK)
    for (i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = x[3 * j] - x[3 * i];
            double dy = x[3 * j + 1] - x[3 * i + 1];
            double dz = x[3 * j + 2] - x[3 * i + 2];
            s += m[j] / sqrt(dx * dx + dy * dy + dz * dz + eps * eps);
        }
        phi[i] = s;
    }
    oracle_accel(n, x, m, G, eps, acc);
    double ek = 0.0, ep = 0.0, p[3] = {0, 0, 0}, f[3] = {0, 0, 0};
    for (i = 0; i < n; ++i) {
        ek += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                            v[3 * i + 2] * v[3 * i + 2]);
        ep += -G * m[i] * phi[i];
        for (int c = 0; c < 3; ++c) {
            p[c] += m[i] * v[3 * i + c];
            f[c] += m[i] * acc[3 * i + c];
        }
    }
    out[0] = ek;
    out[1] = ep;
    out[2] = ek + ep;
    for (int c = 0; c < 3; ++c) {
        out[3 + c] = p[c];
        out[6 + c] = f[c];
    }
    free(phi);
    free(acc);
}

/*
 * Kick-drift-kick leapfrog, nsteps steps of dt, in place on x and v.
 * The force at the initial positions is computed here, then each step is
 *   v += dt/2 a;  x += dt v;  a = F(x);  v += dt/2 a,
 * so nsteps steps take nsteps + 1 force evaluations.  On return acc holds
 * F at the final positions.
 */
void oracle_kdk(int64_t n, double *x, double *v, const double *m, double G,
                double eps, double dt, int64_t nsteps, double *acc)
{
    oracle_accel(n, x, m, G, eps, acc);
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int64_t k = 0; k < 3 * n; ++k) v[k] += 0.5 * dt * acc[k];
        for (int64_t k = 0; k < 3 * n; ++k) x[k] += dt * v[k];
        oracle_accel(n, x, m, G, eps, acc);
        for (int64_t k = 0; k < 3 * n; ++k) v[k] += 0.5 * dt * acc[k];
    }
}

/*
 * Vector-Jacobian product of the force map a = F(x, m) with cotangent
 * lam = dL/da (n,3).  With d_kj = x_j - x_k, s = sqrt(|d|^2 + eps^2) and the
 * symmetric tensor K(d) = I/s^3 - 3 d d^T / s^5 (the derivative of d/s^3):
 *   gx_k = G sum_{j != k} K(d_kj) (m_k lam_j - m_j lam_k)
 *   gm_k = G sum_{i != k} lam_i . (x_k - x_i) / s_ik^3
 * gx and gm are overwritten.
 */
void oracle_force_vjp(int64_t n, const double *x, const double *m, double G,
                      double eps, const double *lam, double *gx, double *gm)
{
    int64_t k;
#pragma omp parallel for schedule(dynamic, ORACLE_CHUNK)
    for (k = 0; k < n; ++k) {
        double g[3] = {0, 0, 0}, gmk = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == k) continue;
            double d[3], w[3];
            for (int c = 0; c < 3; ++c) {
                d[c] = x[3 * j + c] - x[3 * k + c];
                w[c] = m[k] * lam[3 * j + c] - m[j] * lam[3 * k + c];
            }
            double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps * eps;
            double s = sqrt(s2);
            double inv_s3 = 1.0 / (s2 * s);
            double inv_s5 = inv_s3 / s2;
            double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
            for (int c = 0; c < 3; ++c)
                g[c] += w[c] * inv_s3 - 3.0 * d[c] * dw * inv_s5;
            /* x_k - x_j = -d */
            double ld = lam[3 * j] * d[0] + lam[3 * j + 1] * d[1] +
                        lam[3 * j + 2] * d[2];
            gmk += -ld * inv_s3;
        }
        for (int c = 0; c < 3; ++c) gx[3 * k + c] = G * g[c];
        gm[k] = G * gmk;
    }
}

/*
 * Gradient of a loss L(x_K, v_K) through nsteps leapfrog steps, from the
 * cotangents gxT = dL/dx_K and gvT = dL/dv_K.  The forward run stores every
 * position; the reverse sweep undoes each step in the opposite order:
 *   second half-kick  v_K = v_h + dt/2 F(x_K):  lx += VJP_F(x_K, dt/2 lv)
 *   drift             x_K = x + dt v_h:         lv += dt lx
 *   first half-kick   v_h = v + dt/2 F(x):      lx += VJP_F(x, dt/2 lv)
 * with the mass cotangent accumulated from every VJP.  Outputs
 * gx0 = dL/dx_0, gv0 = dL/dv_0, gm = dL/dm (overwritten).
 */
int oracle_kdk_grad(int64_t n, const double *x0, const double *v0,
                    const double *m, double G, double eps, double dt,
                    int64_t nsteps, const double *gxT, const double *gvT,
                    double *gx0, double *gv0, double *gm)
{
    size_t per = (size_t)(3 * n);
    double *traj = (double *)malloc(sizeof(double) * per * (size_t)(nsteps + 1) + 8);
    double *v = (double *)malloc(sizeof(double) * per + 8);
    double *acc = (double *)malloc(sizeof(double) * per + 8);
    double *mu = (double *)malloc(sizeof(double) * per + 8);
    double *dgx = (double *)malloc(sizeof(double) * per + 8);
    double *dgm = (double *)malloc(sizeof(double) * (size_t)n + 8);
    if (!traj || !v || !acc || !mu || !dgx || !dgm) {
        free(traj); free(v); free(acc); free(mu); free(dgx); free(dgm);
        return -1;
    }
    memcpy(traj, x0, sizeof(double) * per);
    memcpy(v, v0, sizeof(double) * per);
    oracle_accel(n, traj, m, G, eps, acc);
    for (int64_t s = 0; s < nsteps; ++s) {
        double *xs = traj + per * (size_t)s, *xn = traj + per * (size_t)(s + 1);
        for (size_t k = 0; k < per; ++k) v[k] += 0.5 * dt * acc[k];
        for (size_t k = 0; k < per; ++k) xn[k] = xs[k] + dt * v[k];
        oracle_accel(n, xn, m, G, eps, acc);
        for (size_t k = 0; k < per; ++k) v[k] += 0.5 * dt * acc[k];
    }
    double *lx = gx0, *lv = gv0;
    memcpy(lx, gxT, sizeof(double) * per);
    memcpy(lv, gvT, sizeof(double) * per);
    for (int64_t k = 0; k < n; ++k) gm[k] = 0.0;
    for (int64_t s = nsteps - 1; s >= 0; --s) {
        double *xs = traj + per * (size_t)s, *xn = traj + per * (size_t)(s + 1);
        for (size_t k = 0; k < per; ++k) mu[k] = 0.5 * dt * lv[k];
        oracle_force_vjp(n, xn, m, G, eps, mu, dgx, dgm);
        for (size_t k = 0; k < per; ++k) lx[k] += dgx[k];
        for (int64_t k = 0; k < n; ++k) gm[k] += dgm[k];
        for (size_t k = 0; k < per; ++k) lv[k] += dt * lx[k];
        for (size_t k = 0; k < per; ++k) mu[k] = 0.5 * dt * lv[k];
        oracle_force_vjp(n, xs, m, G, eps, mu, dgx, dgm);
        for (size_t k = 0; k < per; ++k) lx[k] += dgx[k];
        for (int64_t k = 0; k < n; ++k) gm[k] += dgm[k];
    }
    free(traj); free(v); free(acc); free(mu); free(dgx); free(dgm);
    return 0;
}

/* ------------------------------------------------------------------ */
/*
 * Barnes-Hut tree code (paper Sec. IV-A): the bodies are distributed in an
 * octree by recursively dividing space into 8 subspaces until a subspace
 * holds few enough bodies; the force on a body is evaluated by traversing
 * the tree from the root, adding a cell to the interaction list when it is
 * distant enough and otherwise continuing with its children; the list is
 * then looped through to compute the force.
 *
 * Readings where the paper is silent (no opening criterion, threshold or
 * grouping is given):
 *  - space: the cube at the bodies' bounding-box minimum with edge equal to
 *    the longest box side; a body's cell at level L is given by the top 3L
 *    bits of its 30-bit Morton key, q_c = floor((x_c - lo_c) * (1024 / ext))
 *    clamped to [0, 1023];
 *  - a cell is a leaf when it holds at most `leaf_cap` bodies or is at
 *    level 10;
 *  - cells interact as their total mass at their centre of mass (monopole),
 *    softened like a body;
 *  - "distant enough": the distance from the body to the cell's cube is at
 *    least (cell edge) / theta, evaluated in float32 from float32 inputs;
 *  - bodies are taken in groups of `group` consecutive bodies in key order,
 *    and a group walks the tree together: a cell goes on the group's list
 *    only when it is distant enough from every body of the group.  group = 1
 *    is the per-body traversal the paper describes.
 * stats (optional) receives {nodes, leaves, cell interactions, body
 * interactions}; cnt (optional, [n][2]) receives per body the number of
 * cells and bodies on its list (the self pair included).
 */
typedef struct {
    int64_t start, end;
    int level;
    uint32_t prefix;
    int64_t child[8];
    double M, com[3];
    float lo[3], hi[3];
} bh_node;

typedef struct {
    bh_node *nodes;
    int64_t nnodes, cap;
    const uint32_t *key;
    int leaf_cap;
} bh_tree;

static uint32_t spread10(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

static const uint32_t *g_sort_key;
static int cmp_key_index(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    if (g_sort_key[i] != g_sort_key[j]) return g_sort_key[i] < g_sort_key[j] ? -1 : 1;
    return i < j ? -1 : (i > j);
}

static int64_t bh_build(bh_tree *t, int level, uint32_t prefix, int64_t start, int64_t end)
{
    if (t->nnodes == t->cap) {
        t->cap *= 2;
        t->nodes = (bh_node *)realloc(t->nodes, sizeof(bh_node) * (size_t)t->cap);
    }
    int64_t id = t->nnodes++;
    bh_node *nd = &t->nodes[id];
    nd->start = start;
    nd->end = end;
    nd->level = level;
    nd->prefix = prefix;
    for (int o = 0; o < 8; ++o) nd->child[o] = -1;
    if (end - start <= t->leaf_cap || level == 10) return id;
    int shift = 3 * (10 - (level + 1));
    int64_t s = start;
    for (int o = 0; o < 8; ++o) {
        uint32_t cp = prefix * 8u + (uint32_t)o;
        int64_t e = s;
        while (e < end && (t->key[e] >> shift) == cp) ++e;
        if (e > s) {
            int64_t c = bh_build(t, level + 1, cp, s, e);
            t->nodes[id].child[o] = c;
        }
        s = e;
    }
    return id;
}

/* The tree of readings above, with everything the walks need. */
typedef struct {
    bh_tree t;
    int64_t *perm;
    uint32_t *key0, *key;
    float crit2[11];
    int64_t leaves;
    double box_lo[3], ext;  /* the root cube: corner and edge */
} bh_prep;

static void bh_prepare(bh_prep *P, int64_t n, const double *x, const double *m, double theta,
                       int leaf_cap)
{
    double lo[3], hi[3];
    for (int c = 0; c < 3; ++c) lo[c] = hi[c] = x[c];
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            if (x[3 * i + c] < lo[c]) lo[c] = x[3 * i + c];
            if (x[3 * i + c] > hi[c]) hi[c] = x[3 * i + c];
        }
    double ext = hi[0] - lo[0];
    if (hi[1] - lo[1] > ext) ext = hi[1] - lo[1];
    if (hi[2] - lo[2] > ext) ext = hi[2] - lo[2];
    if (!(ext > 0.0)) ext = 1.0;
    const double scale = 1024.0 / ext;

    uint32_t *key0 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int c = 0; c < 3; ++c) {
            double tq = (x[3 * i + c] - lo[c]) * scale;
            q[c] = tq >= 1023.0 ? 1023u : (tq <= 0.0 ? 0u : (uint32_t)tq);
        }
        key0[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
        perm[i] = i;
    }
    g_sort_key = key0;
    qsort(perm, (size_t)n, sizeof(int64_t), cmp_key_index);
    for (int64_t k = 0; k < n; ++k) key[k] = key0[perm[k]];

    bh_tree t;
    t.cap = 1024;
    t.nnodes = 0;
    t.nodes = (bh_node *)malloc(sizeof(bh_node) * (size_t)t.cap);
    t.key = key;
    t.leaf_cap = leaf_cap;
    bh_build(&t, 0, 0u, 0, n);

    /* monopole moments and float32 cell cubes */
    int64_t leaves = 0;
    for (int64_t id = 0; id < t.nnodes; ++id) {
        bh_node *nd = &t.nodes[id];
        double M = 0.0, s[3] = {0, 0, 0};
        for (int64_t k = nd->start; k < nd->end; ++k) {
            int64_t j = perm[k];
            M += m[j];
            for (int c = 0; c < 3; ++c) s[c] += m[j] * x[3 * j + c];
        }
        nd->M = M;
        for (int c = 0; c < 3; ++c) nd->com[c] = M > 0.0 ? s[c] / M : 0.0;
        uint32_t ic[3] = {0, 0, 0};
        for (int b = 0; b < nd->level; ++b) {  /* de-interleave the prefix */
            uint32_t trip = (nd->prefix >> (3 * b)) & 7u;
            for (int c = 0; c < 3; ++c) ic[c] |= ((trip >> c) & 1u) << b;
        }
        double cell = ext / (double)(1u << nd->level);
        for (int c = 0; c < 3; ++c) {
            nd->lo[c] = (float)(lo[c] + cell * (double)ic[c]);
            nd->hi[c] = (float)(lo[c] + cell * (double)(ic[c] + 1u));
        }
        int leaf = 1;
        for (int o = 0; o < 8; ++o) if (nd->child[o] >= 0) leaf = 0;
        leaves += leaf;
    }
    /* squared opening distance per level, in float32 */
    const float th = (float)theta;
    for (int L = 0; L <= 10; ++L) {
        float edge = (float)(ext / (double)(1u << L));
        float d = edge / th;
        P->crit2[L] = d * d;
    }
    P->t = t;
    for (int c = 0; c < 3; ++c) P->box_lo[c] = lo[c];
    P->ext = ext;
    P->perm = perm;
    P->key0 = key0;
    P->key = key;
    P->leaves = leaves;
}

static void bh_release(bh_prep *P)
{
    free(P->key0); free(P->perm); free(P->key); free(P->t.nodes);
}

/* Walk of the group holding sorted bodies [g0, g1): its list, then each of
 * its bodies' sums.  Writes acc and cnt at the original body indices; adds
 * to the interaction totals. */
typedef struct {
    int64_t *stack, *lst, lcap;
    float *xf;
} bh_work;

static void bh_walk_group(const bh_prep *P, bh_work *W, int64_t g0, int64_t g1, const double *x,
                          const double *m, double G, double eps, double *acc, int64_t *cnt,
                          int64_t *ncell, int64_t *nbody)
{
    const bh_tree *t = &P->t;
    const int64_t *perm = P->perm;
    const float *crit2 = P->crit2;
    float *xf = W->xf;
    int64_t *stack = W->stack;
    for (int64_t k = g0; k < g1; ++k)
        for (int c = 0; c < 3; ++c) xf[3 * (k - g0) + c] = (float)x[3 * perm[k] + c];
    /* walk: list entries >= 0 are cells, < 0 encode leaf nodes as ~id */
    int64_t nl = 0, sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        int64_t id = stack[--sp];
        const bh_node *nd = &t->nodes[id];
        int all = 1;
        for (int64_t k = g0; k < g1 && all; ++k) {
            const float *p = xf + 3 * (k - g0);
            float d2 = 0.0f;
            for (int c = 0; c < 3; ++c) {
                float a = nd->lo[c] - p[c];
                float b = p[c] - nd->hi[c];
                float dd = a > b ? a : b;
                dd = dd > 0.0f ? dd : 0.0f;
                float sq = dd * dd;
                d2 = d2 + sq;
            }
            if (!(d2 >= crit2[nd->level])) all = 0;
        }
        int leaf = 1;
        for (int o = 0; o < 8; ++o) if (nd->child[o] >= 0) leaf = 0;
        if (all || leaf) {
            if (nl == W->lcap) {
                W->lcap *= 2;
                W->lst = (int64_t *)realloc(W->lst, sizeof(int64_t) * (size_t)W->lcap);
            }
            W->lst[nl++] = all ? id : ~id;
        } else {
            for (int o = 7; o >= 0; --o)
                if (nd->child[o] >= 0) stack[sp++] = nd->child[o];
        }
    }
    const int64_t *lst = W->lst;
    for (int64_t k = g0; k < g1; ++k) {
        int64_t i = perm[k];
        double a[3] = {0, 0, 0};
        int64_t nc = 0, nb = 0;
        for (int64_t q = 0; q < nl; ++q) {
            if (lst[q] >= 0) {
                const bh_node *nd = &t->nodes[lst[q]];
                double d[3], s2 = eps * eps;
                for (int c = 0; c < 3; ++c) {
                    d[c] = nd->com[c] - x[3 * i + c];
                    s2 += d[c] * d[c];
                }
                double w = nd->M / (s2 * sqrt(s2));
                for (int c = 0; c < 3; ++c) a[c] += w * d[c];
                ++nc;
            } else {
                const bh_node *nd = &t->nodes[~lst[q]];
                for (int64_t kk = nd->start; kk < nd->end; ++kk) {
                    int64_t j = perm[kk];
                    ++nb;
                    if (j == i) continue;
                    double d[3], s2 = eps * eps;
                    for (int c = 0; c < 3; ++c) {
                        d[c] = x[3 * j + c] - x[3 * i + c];
                        s2 += d[c] * d[c];
                    }
                    double w = m[j] / (s2 * sqrt(s2));
                    for (int c = 0; c < 3; ++c) a[c] += w * d[c];
                }
            }
        }
        for (int c = 0; c < 3; ++c) acc[3 * i + c] = G * a[c];
        if (cnt) {
            cnt[2 * i] = nc;
            cnt[2 * i + 1] = nb;
        }
        *ncell += nc;
        *nbody += nb;
    }
}

static void bh_work_init(bh_work *W, int group)
{
    W->stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(8 * 11 + 8));
    W->lcap = 1024;
    W->lst = (int64_t *)malloc(sizeof(int64_t) * (size_t)W->lcap);
    W->xf = (float *)malloc(sizeof(float) * 3 * (size_t)group);
}

static void bh_work_free(bh_work *W)
{
    free(W->stack); free(W->lst); free(W->xf);
}

int oracle_bh_forces(int64_t n, const double *x, const double *m, double G, double eps,
                     double theta, int leaf_cap, int group, double *acc, int64_t *stats,
                     int64_t *cnt)
{
    if (n <= 0) return 0;
    if (leaf_cap < 1 || group < 1) return -1;
    bh_prep P;
    bh_prepare(&P, n, x, m, theta, leaf_cap);
    bh_work W;
    bh_work_init(&W, group);
    int64_t ncell = 0, nbody = 0;
    for (int64_t g0 = 0; g0 < n; g0 += group) {
        int64_t g1 = g0 + group < n ? g0 + group : n;
        bh_walk_group(&P, &W, g0, g1, x, m, G, eps, acc, cnt, &ncell, &nbody);
    }
    if (stats) {
        stats[0] = P.t.nnodes;
        stats[1] = P.leaves;
        stats[2] = ncell;
        stats[3] = nbody;
    }
    bh_work_free(&W);
    bh_release(&P);
    return 0;
}

/*
 * The same tree code for a subset of the groups: the tree is built over all
 * n bodies and only the groups sel[0..nsel) (indices in key order) walk it.
 * acc (n,3) and cnt (n,2) are written for the bodies of those groups only;
 * idx[q * group + r] receives the body index of the r-th body of group
 * sel[q] (-1 past the last body).  Returns -1 for bad arguments or a group
 * index out of range.
 */
int oracle_bh_groups(int64_t n, const double *x, const double *m, double G, double eps,
                     double theta, int leaf_cap, int group, int64_t nsel, const int64_t *sel,
                     int64_t *idx, double *acc, int64_t *cnt)
{
    if (n <= 0 || nsel <= 0) return 0;
    if (leaf_cap < 1 || group < 1) return -1;
    const int64_t ngroups = (n + group - 1) / group;
    for (int64_t q = 0; q < nsel; ++q)
        if (sel[q] < 0 || sel[q] >= ngroups) return -1;
    bh_prep P;
    bh_prepare(&P, n, x, m, theta, leaf_cap);
    bh_work W;
    bh_work_init(&W, group);
    int64_t ncell = 0, nbody = 0;
    for (int64_t q = 0; q < nsel; ++q) {
        int64_t g0 = sel[q] * group;
        int64_t g1 = g0 + group < n ? g0 + group : n;
        for (int64_t r = 0; r < group; ++r) idx[q * group + r] = g0 + r < n ? P.perm[g0 + r] : -1;
        bh_walk_group(&P, &W, g0, g1, x, m, G, eps, acc, cnt, &ncell, &nbody);
    }
    bh_work_free(&W);
    bh_release(&P);
    return 0;
}

/*
 * Parallel tree code (paper Sec. IV-B).  The paper divides space by
 * orthogonal recursive bisection (ORB) into as many non-overlapping
 * subspaces as processors, each holding about the same number of bodies;
 * each processor builds a tree over its own bodies and extends it into a
 * locally essential tree (LET) with the nodes of the other processors' trees
 * that its bodies need -- a node matters to the bodies in its "influence
 * ring", those that open its parent yet use the node itself -- and then
 * computes forces as in the sequential code.  Readings (the paper gives no
 * splitting rule, ring construction or summation order):
 *  - ORB: the bodies of a part that p processors share are cut across the
 *    longest side of their float64 bounding box (the lowest axis on ties);
 *    the lower part takes floor(p/2) processors and the
 *    k = floor(count * floor(p/2) / p) bodies first in (coordinate, body
 *    index) order, the upper part the rest; parts are cut again until each
 *    holds one processor's bodies;
 *  - each processor's tree is the tree code's tree (readings above) over its
 *    own bodies taken in increasing body index, with their own bounding
 *    cube; bodies walk in groups of consecutive bodies of their own tree's
 *    key order;
 *  - a body's acceleration is the sum over every processor's tree of that
 *    tree's group walk (its own tree first, then the others in processor
 *    order); a processor's LET holds, of each other tree, what those walks
 *    meet;
 *  - the LET of tree s for processor d applies the influence-ring test from
 *    the destination's side: the root is sent; a sent node that is distant
 *    enough (the walk's float32 test) from the float32 bounding box of d's
 *    bodies is accepted by every body of d and is sent alone; otherwise a
 *    sent leaf is sent with its bodies and a sent cell with all its
 *    children.  No body inside a box is nearer a cube than the box is (the
 *    float32 operations are monotonic), so no body of d opens a node sent
 *    alone, and every node a body of d opens is sent with what is inside.
 */
static const double *g_orb_x;
static int g_orb_axis;
static int cmp_orb(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    double xi = g_orb_x[3 * i + g_orb_axis], xj = g_orb_x[3 * j + g_orb_axis];
    if (xi != xj) return xi < xj ? -1 : 1;
    return i < j ? -1 : (i > j);
}

static void orb_part(const double *x, int64_t *idx, int64_t cnt, int rank0, int p, int32_t *rank)
{
    if (cnt == 0) return;
    if (p == 1) {
        for (int64_t k = 0; k < cnt; ++k) rank[idx[k]] = rank0;
        return;
    }
    double lo[3], hi[3];
    for (int c = 0; c < 3; ++c) lo[c] = hi[c] = x[3 * idx[0] + c];
    for (int64_t k = 1; k < cnt; ++k)
        for (int c = 0; c < 3; ++c) {
            double v = x[3 * idx[k] + c];
            if (v < lo[c]) lo[c] = v;
            if (v > hi[c]) hi[c] = v;
        }
    int axis = 0;
    for (int c = 1; c < 3; ++c)
        if (hi[c] - lo[c] > hi[axis] - lo[axis]) axis = c;
    g_orb_x = x;
    g_orb_axis = axis;
    qsort(idx, (size_t)cnt, sizeof(int64_t), cmp_orb);
    int p_lo = p / 2;
    int64_t k = cnt * (int64_t)p_lo / p;
    orb_part(x, idx, k, rank0, p_lo, rank);
    orb_part(x, idx + k, cnt - k, rank0 + p_lo, p - p_lo, rank);
}

/* rank[i] in [0, P): the processor whose ORB domain holds body i. */
int oracle_orb(int64_t n, const double *x, int P, int32_t *rank)
{
    if (P < 1) return -1;
    if (n <= 0) return 0;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    orb_part(x, idx, n, 0, P, rank);
    free(idx);
    return 0;
}

/* One group of targets (nt bodies: float32 positions xf for the opening
 * test, float64 positions xt, body indices tid) walks the tree S of the
 * source bodies xs, ms (body indices sid): each target's sum (without G) is
 * ADDED to a[3k..] and its list sizes to c[3k..] = {cells, bodies met
 * directly, bodies inside the cells and met directly}. */
static void bh_walk_sources(const bh_prep *S, bh_work *W, const double *xs, const double *ms,
                            const int64_t *sid, int64_t nt, const float *xf, const double *xt,
                            const int64_t *tid, double eps, double *a, int64_t *c)
{
    const bh_tree *t = &S->t;
    const int64_t *perm = S->perm;
    int64_t nl = 0, sp = 0;
    int64_t *stack = W->stack;
    stack[sp++] = 0;
    while (sp > 0) {
        int64_t id = stack[--sp];
        const bh_node *nd = &t->nodes[id];
        int all = 1;
        for (int64_t k = 0; k < nt && all; ++k) {
            const float *p = xf + 3 * k;
            float d2 = 0.0f;
            for (int cc = 0; cc < 3; ++cc) {
                float aa = nd->lo[cc] - p[cc];
                float bb = p[cc] - nd->hi[cc];
                float dd = aa > bb ? aa : bb;
                dd = dd > 0.0f ? dd : 0.0f;
                float sq = dd * dd;
                d2 = d2 + sq;
            }
            if (!(d2 >= S->crit2[nd->level])) all = 0;
        }
        int leaf = 1;
        for (int o = 0; o < 8; ++o) if (nd->child[o] >= 0) leaf = 0;
        if (all || leaf) {
            if (nl == W->lcap) {
                W->lcap *= 2;
                W->lst = (int64_t *)realloc(W->lst, sizeof(int64_t) * (size_t)W->lcap);
            }
            W->lst[nl++] = all ? id : ~id;
        } else {
            for (int o = 7; o >= 0; --o)
                if (nd->child[o] >= 0) stack[sp++] = nd->child[o];
        }
    }
    const int64_t *lst = W->lst;
    for (int64_t k = 0; k < nt; ++k) {
        const double *xi = xt + 3 * k;
        double s[3] = {0, 0, 0};
        int64_t nc = 0, nb = 0, cov = 0;
        for (int64_t q = 0; q < nl; ++q) {
            if (lst[q] >= 0) {
                const bh_node *nd = &t->nodes[lst[q]];
                double d[3], s2 = eps * eps;
                for (int cc = 0; cc < 3; ++cc) {
                    d[cc] = nd->com[cc] - xi[cc];
                    s2 += d[cc] * d[cc];
                }
                double wc = nd->M / (s2 * sqrt(s2));
                for (int cc = 0; cc < 3; ++cc) s[cc] += wc * d[cc];
                ++nc;
                cov += nd->end - nd->start;
            } else {
                const bh_node *nd = &t->nodes[~lst[q]];
                for (int64_t kk = nd->start; kk < nd->end; ++kk) {
                    int64_t j = perm[kk];
                    ++nb;
                    ++cov;
                    if (sid[j] == tid[k]) continue;
                    double d[3], s2 = eps * eps;
                    for (int cc = 0; cc < 3; ++cc) {
                        d[cc] = xs[3 * j + cc] - xi[cc];
                        s2 += d[cc] * d[cc];
                    }
                    double w = ms[j] / (s2 * sqrt(s2));
                    for (int cc = 0; cc < 3; ++cc) s[cc] += w * d[cc];
                }
            }
        }
        for (int cc = 0; cc < 3; ++cc) a[3 * k + cc] += s[cc];
        c[3 * k] += nc;
        c[3 * k + 1] += nb;
        c[3 * k + 2] += cov;
    }
}

/* The bodies of processor s (rank[i] == s), in increasing body index. */
static int64_t shard_gather(int64_t n, const double *x, const double *m, const int32_t *rank,
                            int s, double *xs, double *ms, int64_t *sid)
{
    int64_t ns = 0;
    for (int64_t i = 0; i < n; ++i)
        if (rank[i] == s) {
            for (int c = 0; c < 3; ++c) xs[3 * ns + c] = x[3 * i + c];
            ms[ns] = m[i];
            sid[ns] = i;
            ++ns;
        }
    return ns;
}

/*
 * Accelerations of the parallel tree code over P processors whose bodies
 * rank[] assigns (e.g. from oracle_orb): every processor's tree built over
 * its own bodies, every group of every processor walking every tree.
 * cnt (optional, [n][3]) receives per body the cells met, the bodies met
 * directly (the self pair included) and the bodies covered (inside the
 * cells met, or met directly: each body of the system exactly once).
 * stats = {nodes of all trees, their leaves, cell interactions, body
 * interactions}.  Returns -1 for bad arguments.
 */
int oracle_bh_sharded(int64_t n, const double *x, const double *m, double G, double eps,
                      double theta, int leaf_cap, int group, int P, const int32_t *rank,
                      double *acc, int64_t *stats, int64_t *cnt)
{
    if (leaf_cap < 1 || group < 1 || P < 1) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (rank[i] < 0 || rank[i] >= P) return -1;
    if (n <= 0) return 0;
    double **xs = (double **)calloc((size_t)P, sizeof(double *));
    double **ms = (double **)calloc((size_t)P, sizeof(double *));
    int64_t **sid = (int64_t **)calloc((size_t)P, sizeof(int64_t *));
    int64_t *ns = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    bh_prep *S = (bh_prep *)calloc((size_t)P, sizeof(bh_prep));
    int64_t st[4] = {0, 0, 0, 0};
    for (int s = 0; s < P; ++s) {
        xs[s] = (double *)malloc(sizeof(double) * 3 * (size_t)n);
        ms[s] = (double *)malloc(sizeof(double) * (size_t)n);
        sid[s] = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        ns[s] = shard_gather(n, x, m, rank, s, xs[s], ms[s], sid[s]);
        if (ns[s] > 0) {
            bh_prepare(&S[s], ns[s], xs[s], ms[s], theta, leaf_cap);
            st[0] += S[s].t.nnodes;
            st[1] += S[s].leaves;
        }
    }
    bh_work W;
    bh_work_init(&W, group);
    float *xf = (float *)malloc(sizeof(float) * 3 * (size_t)group);
    double *xt = (double *)malloc(sizeof(double) * 3 * (size_t)group);
    int64_t *tid = (int64_t *)malloc(sizeof(int64_t) * (size_t)group);
    double *a = (double *)malloc(sizeof(double) * 3 * (size_t)group);
    int64_t *c = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)group);
    for (int r = 0; r < P; ++r) {
        for (int64_t g0 = 0; g0 < ns[r]; g0 += group) {
            int64_t g1 = g0 + group < ns[r] ? g0 + group : ns[r];
            int64_t nt = g1 - g0;
            for (int64_t k = 0; k < nt; ++k) {
                int64_t j = S[r].perm[g0 + k];
                tid[k] = sid[r][j];
                for (int cc = 0; cc < 3; ++cc) {
                    xt[3 * k + cc] = xs[r][3 * j + cc];
                    xf[3 * k + cc] = (float)xs[r][3 * j + cc];
                    a[3 * k + cc] = 0.0;
                    c[3 * k + cc] = 0;
                }
            }
            for (int q = 0; q < P; ++q) {
                int s = q == 0 ? r : (q <= r ? q - 1 : q);  /* own tree, then the others in order */
                if (ns[s] == 0) continue;
                bh_walk_sources(&S[s], &W, xs[s], ms[s], sid[s], nt, xf, xt, tid, eps, a, c);
            }
            for (int64_t k = 0; k < nt; ++k) {
                for (int cc = 0; cc < 3; ++cc) acc[3 * tid[k] + cc] = G * a[3 * k + cc];
                if (cnt)
                    for (int cc = 0; cc < 3; ++cc) cnt[3 * tid[k] + cc] = c[3 * k + cc];
                st[2] += c[3 * k];
                st[3] += c[3 * k + 1];
            }
        }
    }
    if (stats)
        for (int q = 0; q < 4; ++q) stats[q] = st[q];
    free(xf); free(xt); free(tid); free(a); free(c);
    bh_work_free(&W);
    for (int s = 0; s < P; ++s) {
        if (ns[s] > 0) bh_release(&S[s]);
        free(xs[s]); free(ms[s]); free(sid[s]);
    }
    free(xs); free(ms); free(sid); free(ns); free(S);
    return 0;
}

/*
 * The tree over the source bodies (xs, ms) with, per node, its kind in the
 * LET for a destination whose bodies lie in the float32 box [blo, bhi]
 * (readings above): 0 not sent, 1 sent alone (accepted by every body in the
 * box), 2 sent with all its children, 3 a leaf sent with its bodies.  The
 * nodes are in build order (a parent before its children); *nnodes receives
 * their number, and when cap >= *nnodes the arrays are filled: kind, level,
 * prefix (the key bits of the node's cell), child[8] (-1 = none), range[2]
 * (the node's bodies, positions in key order), lo/hi[3] (float32 cube
 * corners), and perm[ns] (key order -> source body).  Returns -1 for bad
 * arguments.
 */
int oracle_bh_let(int64_t ns, const double *xs, const double *ms, double theta, int leaf_cap,
                  const float *blo, const float *bhi, int64_t cap, int64_t *nnodes,
                  int32_t *kind, int32_t *level, int64_t *prefix, int64_t *child, int64_t *range,
                  float *lo, float *hi, int64_t *perm)
{
    if (leaf_cap < 1 || ns <= 0) return -1;
    bh_prep S;
    bh_prepare(&S, ns, xs, ms, theta, leaf_cap);
    const int64_t nn = S.t.nnodes;
    *nnodes = nn;
    if (cap >= nn) {
        for (int64_t id = 0; id < nn; ++id) kind[id] = 0;
        kind[0] = -1;  /* sent; classified below (parents come before children) */
        for (int64_t id = 0; id < nn; ++id) {
            const bh_node *nd = &S.t.nodes[id];
            level[id] = nd->level;
            prefix[id] = nd->prefix;
            for (int o = 0; o < 8; ++o) child[8 * id + o] = nd->child[o];
            range[2 * id] = nd->start;
            range[2 * id + 1] = nd->end;
            for (int c = 0; c < 3; ++c) {
                lo[3 * id + c] = nd->lo[c];
                hi[3 * id + c] = nd->hi[c];
            }
            if (kind[id] != -1) continue;
            float d2 = 0.0f;
            for (int c = 0; c < 3; ++c) {
                float aa = nd->lo[c] - bhi[c];
                float bb = blo[c] - nd->hi[c];
                float dd = aa > bb ? aa : bb;
                dd = dd > 0.0f ? dd : 0.0f;
                float sq = dd * dd;
                d2 = d2 + sq;
            }
            int leaf = 1;
            for (int o = 0; o < 8; ++o) if (nd->child[o] >= 0) leaf = 0;
            if (d2 >= S.crit2[nd->level]) {
                kind[id] = 1;
            } else if (leaf) {
                kind[id] = 3;
            } else {
                kind[id] = 2;
                for (int o = 0; o < 8; ++o)
                    if (nd->child[o] >= 0) kind[nd->child[o]] = -1;
            }
        }
        for (int64_t k = 0; k < ns; ++k) perm[k] = S.perm[k];
    }
    bh_release(&S);
    return 0;
}

/*
 * Fast multipole method: the O(N) method the paper names as the successor
 * of its tree code (Sec. VI, after Greengard and Rokhlin, ref. [20]).  The
 * paper gives no formulation; the readings here are:
 *  - the tree is the Barnes-Hut tree above (same cube, keys and leaf rule);
 *  - every cell carries a Cartesian Taylor expansion about its cube's centre
 *    z, with multi-indices n = (a, b, c), x^n = x^a y^b z^c, n! = a! b! c!
 *    and order p: the multipole moments
 *        Mh_n = sum_{j in cell} m_j (-(x_j - z))^n / n!,      |n| <= p;
 *  - the kernel is the softened one, g(r) = (|r|^2 + eps^2)^{-1/2}: the
 *    acceleration is G times the gradient of sum_j m_j g(x - x_j).  Its
 *    derivatives T_n = d^n g follow from g = f(|r|^2 / 2), whose m-th
 *    derivative is D_m = (-1)^m (2m-1)!! (|r|^2 + eps^2)^{-(2m+1)/2}, by
 *        d^n f_m = r_c d^{n-e_c} f_{m+1} + (n_c - 1) d^{n-2e_c} f_{m+1}
 *    (Leibniz's rule on d^n f_m = d^{n-e_c} (r_c f_{m+1}), c any axis with
 *    n_c >= 1; the first such axis here);
 *  - a source cell B acts on a target cell A through the local expansion
 *        L_k = sum_{|n| <= p - |k|} Mh_n T_{n+k}(z_A - z_B),    |k| <= p,
 *    the Taylor polynomial sum_k L_k u^k / k! (u = x - z_A) of B's potential
 *    in A; a body's far-field acceleration is G times the gradient of the
 *    polynomials of its leaf and of every ancestor of its leaf:
 *        a_c = G sum_{A'} sum_{|k| <= p-1} L^{A'}_{k+e_c} u^k / k!;
 *  - A and B are well separated when |z_A - z_B| >= (r_A + r_B) / theta,
 *    r the cube's circumradius (sqrt(3)/2 of its edge).  In units of
 *    h = ext / 2048 a level-L centre is an odd multiple of 2^(10-L) and its
 *    edge is 2^(11-L), so the test is exact: the integer
 *    D2 = |c_A - c_B|^2 against 0.75 (e_A + e_B)^2 / theta^2 in double;
 *  - which pairs interact: the dual-tree traversal from (root, root).
 *    Each target cell takes the candidates its parent handed down (the root
 *    takes the root).  For target A and candidate B: well separated -> B's
 *    expansion acts on A; else if A and B are leaves -> their bodies
 *    interact directly (self pair excluded); else if A is a leaf -> B's
 *    children are candidates of A; else if B is a leaf or smaller than A ->
 *    B goes down to A's children; else (B as large as A) B's children go
 *    down to A's children.
 * Every body so meets every other body exactly once: directly, or inside a
 * source cell acting on its leaf or on an ancestor of its leaf.
 *
 * The oracle takes the definitions as written: moments summed over each
 * cell's own bodies, every local polynomial evaluated at the body.  It does
 * not translate expansions between cells (the moment and local translations
 * of an FMM are exact rewritings of these sums).
 */
#define FMM_MAX_ORDER 12

typedef struct {
    int p, nt;        /* order; multi-indices of order <= p */
    int (*mi)[3];     /* multi-index of each slot, graded (order by order) */
    double *inv_fact; /* 1 / n! per slot */
} fmm_basis;

/* Slot of (a, b, c): orders below k first, then a descending, b descending. */
static int fmm_slot(int a, int b, int c)
{
    int k = a + b + c, s = b + c;
    return k * (k + 1) * (k + 2) / 6 + s * (s + 1) / 2 + c;
}

static void fmm_basis_init(fmm_basis *B, int p)
{
    B->p = p;
    B->nt = (p + 1) * (p + 2) * (p + 3) / 6;
    B->mi = (int(*)[3])malloc(sizeof(int[3]) * (size_t)B->nt);
    B->inv_fact = (double *)malloc(sizeof(double) * (size_t)B->nt);
    double f[FMM_MAX_ORDER + 1];
    f[0] = 1.0;
    for (int e = 1; e <= FMM_MAX_ORDER; ++e) f[e] = f[e - 1] * (double)e;
    for (int k = 0; k <= p; ++k)
        for (int a = k; a >= 0; --a)
            for (int b = k - a; b >= 0; --b) {
                int c = k - a - b, q = fmm_slot(a, b, c);
                B->mi[q][0] = a;
                B->mi[q][1] = b;
                B->mi[q][2] = c;
                B->inv_fact[q] = 1.0 / (f[a] * f[b] * f[c]);
            }
}

static void fmm_basis_free(fmm_basis *B)
{
    free(B->mi);
    free(B->inv_fact);
}

/* T_n(r) = d^n g(r) for every slot; work holds (p + 1) * nt doubles. */
static void fmm_deriv(const fmm_basis *B, const double r[3], double eps, double *out, double *work)
{
    const int p = B->p, nt = B->nt;
    double s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps * eps;
    double *T = work; /* T[m * nt + q] = d^n f_m */
    T[0] = 1.0 / sqrt(s2);
    for (int m = 1; m <= p; ++m) T[m * nt] = -(double)(2 * m - 1) * T[(m - 1) * nt] / s2;
    for (int q = 1; q < nt; ++q) {
        const int *n = B->mi[q];
        int k = n[0] + n[1] + n[2];
        int c = n[0] > 0 ? 0 : (n[1] > 0 ? 1 : 2);
        int d[3] = {n[0], n[1], n[2]};
        d[c] -= 1;
        int q1 = fmm_slot(d[0], d[1], d[2]), q2 = -1;
        if (n[c] >= 2) {
            d[c] -= 1;
            q2 = fmm_slot(d[0], d[1], d[2]);
        }
        for (int m = 0; m + k <= p; ++m) {
            double v = r[c] * T[(m + 1) * nt + q1];
            if (q2 >= 0) v += (double)(n[c] - 1) * T[(m + 1) * nt + q2];
            T[m * nt + q] = v;
        }
    }
    memcpy(out, T, sizeof(double) * (size_t)nt);
}

/* Public form of fmm_deriv for the pins: out receives (p+1)(p+2)(p+3)/6
 * values in slot order.  Returns -1 for p outside [0, FMM_MAX_ORDER]. */
int oracle_fmm_deriv(int p, const double *r, double eps, double *out)
{
    if (p < 0 || p > FMM_MAX_ORDER) return -1;
    fmm_basis B;
    fmm_basis_init(&B, p);
    double *work = (double *)malloc(sizeof(double) * (size_t)((p + 1) * B.nt));
    fmm_deriv(&B, r, eps, out, work);
    free(work);
    fmm_basis_free(&B);
    return 0;
}

/* Mh += the moments about z of a body of mass mj at xj. */
static void fmm_moments_add(const fmm_basis *B, const double *xj, double mj, const double *z,
                            double *Mh)
{
    double pw[3][FMM_MAX_ORDER + 1];
    for (int c = 0; c < 3; ++c) {
        double y = -(xj[c] - z[c]);
        pw[c][0] = 1.0;
        for (int e = 1; e <= B->p; ++e) pw[c][e] = pw[c][e - 1] * y;
    }
    for (int q = 0; q < B->nt; ++q)
        Mh[q] += mj * pw[0][B->mi[q][0]] * pw[1][B->mi[q][1]] * pw[2][B->mi[q][2]] * B->inv_fact[q];
}

/* L += the local expansion, about z_A, of the moments Mh about z_B;
 * r = z_A - z_B.  Tn holds nt doubles, work (p + 1) nt. */
static void fmm_local_add(const fmm_basis *B, const double *Mh, const double *r, double eps,
                          double *L, double *Tn, double *work)
{
    const int p = B->p;
    fmm_deriv(B, r, eps, Tn, work);
    for (int kq = 0; kq < B->nt; ++kq) {
        const int *k = B->mi[kq];
        int kk = k[0] + k[1] + k[2];
        double s = 0.0;
        for (int nq = 0; nq < B->nt; ++nq) {
            const int *n = B->mi[nq];
            if (n[0] + n[1] + n[2] > p - kk) break; /* slots are graded */
            s += Mh[nq] * Tn[fmm_slot(n[0] + k[0], n[1] + k[1], n[2] + k[2])];
        }
        L[kq] += s;
    }
}

/* a += the gradient of sum_k L_k u^k / k! at u. */
static void fmm_grad_add(const fmm_basis *B, const double *L, const double *u, double *a)
{
    double pw[3][FMM_MAX_ORDER + 1];
    for (int c = 0; c < 3; ++c) {
        pw[c][0] = 1.0;
        for (int e = 1; e <= B->p; ++e) pw[c][e] = pw[c][e - 1] * u[c];
    }
    for (int kq = 0; kq < B->nt; ++kq) {
        const int *k = B->mi[kq];
        if (k[0] + k[1] + k[2] > B->p - 1) break;
        double w = pw[0][k[0]] * pw[1][k[1]] * pw[2][k[2]] * B->inv_fact[kq];
        a[0] += L[fmm_slot(k[0] + 1, k[1], k[2])] * w;
        a[1] += L[fmm_slot(k[0], k[1] + 1, k[2])] * w;
        a[2] += L[fmm_slot(k[0], k[1], k[2] + 1)] * w;
    }
}

/* The expansion chain alone, for the pins: sources (xs, ms) expanded about
 * zB act, through the local expansion about zA, on the targets xt; acc
 * [nt][3] receives the accelerations with G = 1.  Returns -1 for p outside
 * [1, FMM_MAX_ORDER]. */
int oracle_fmm_pair(int p, const double *zA, const double *zB, double eps, int64_t ns,
                    const double *xs, const double *ms, int64_t ntg, const double *xt,
                    double *acc)
{
    if (p < 1 || p > FMM_MAX_ORDER) return -1;
    fmm_basis B;
    fmm_basis_init(&B, p);
    double *Mh = (double *)calloc((size_t)B.nt, sizeof(double));
    double *L = (double *)calloc((size_t)B.nt, sizeof(double));
    double *Tn = (double *)malloc(sizeof(double) * (size_t)B.nt);
    double *work = (double *)malloc(sizeof(double) * (size_t)((p + 1) * B.nt));
    for (int64_t j = 0; j < ns; ++j) fmm_moments_add(&B, xs + 3 * j, ms[j], zB, Mh);
    double r[3] = {zA[0] - zB[0], zA[1] - zB[1], zA[2] - zB[2]};
    fmm_local_add(&B, Mh, r, eps, L, Tn, work);
    for (int64_t i = 0; i < ntg; ++i) {
        double u[3] = {xt[3 * i] - zA[0], xt[3 * i + 1] - zA[1], xt[3 * i + 2] - zA[2]};
        acc[3 * i] = acc[3 * i + 1] = acc[3 * i + 2] = 0.0;
        fmm_grad_add(&B, L, u, acc + 3 * i);
    }
    free(Mh); free(L); free(Tn); free(work);
    fmm_basis_free(&B);
    return 0;
}

typedef struct {
    int32_t *v;
    int64_t n, cap;
} fmm_list;

static void fmm_push(fmm_list *l, int32_t x)
{
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 16;
        l->v = (int32_t *)realloc(l->v, sizeof(int32_t) * (size_t)l->cap);
    }
    l->v[l->n++] = x;
}

typedef struct {
    const bh_prep *P;
    int64_t nn;
    int *leaf, (*ci)[3];
    double crit[11][11];
    fmm_list *m2l, *p2p; /* per node: source cells of its expansion; source leaves */
    int err;
} fmm_trav;

static int fmm_separated(const fmm_trav *T, int64_t a, int64_t b)
{
    int64_t d2 = 0;
    for (int c = 0; c < 3; ++c) {
        int64_t d = (int64_t)T->ci[a][c] - (int64_t)T->ci[b][c];
        d2 += d * d;
    }
    return (double)d2 >= T->crit[T->P->t.nodes[a].level][T->P->t.nodes[b].level];
}

/* Candidate b of the leaf a: b's subtree is walked. */
static void fmm_leaf_visit(fmm_trav *T, int64_t a, int64_t b)
{
    if (fmm_separated(T, a, b)) {
        fmm_push(&T->m2l[a], (int32_t)b);
    } else if (T->leaf[b]) {
        fmm_push(&T->p2p[a], (int32_t)b);
    } else {
        const bh_node *nb = &T->P->t.nodes[b];
        for (int o = 0; o < 8; ++o)
            if (nb->child[o] >= 0) fmm_leaf_visit(T, a, nb->child[o]);
    }
}

/* Target a with the candidates handed down to it. */
static void fmm_down(fmm_trav *T, int64_t a, const int32_t *cand, int64_t ncand)
{
    if (T->leaf[a]) {
        for (int64_t q = 0; q < ncand; ++q) fmm_leaf_visit(T, a, cand[q]);
        return;
    }
    const bh_node *na = &T->P->t.nodes[a];
    fmm_list down = {0, 0, 0};
    for (int64_t q = 0; q < ncand; ++q) {
        int64_t b = cand[q];
        const bh_node *nb = &T->P->t.nodes[b];
        if (fmm_separated(T, a, b)) {
            fmm_push(&T->m2l[a], (int32_t)b);
        } else if (T->leaf[b] || nb->level > na->level) {
            fmm_push(&down, (int32_t)b);
        } else if (nb->level == na->level) {
            for (int o = 0; o < 8; ++o)
                if (nb->child[o] >= 0) fmm_push(&down, (int32_t)nb->child[o]);
        } else {
            T->err = 1; /* a larger non-leaf candidate never reaches a non-leaf */
        }
    }
    for (int o = 0; o < 8; ++o)
        if (na->child[o] >= 0) fmm_down(T, na->child[o], down.v, down.n);
    free(down.v);
}

/*
 * Accelerations by the FMM of the readings above, order p (1..12), opening
 * parameter theta >= 0 (theta = 0: nothing is well separated, every pair
 * interacts directly).  stats (optional) receives {nodes, leaves,
 * cell-cell expansions, body-body pairs (self pairs included)}; cnt
 * (optional, [n][3]) receives per body the number of source cells acting on
 * its leaf and the leaf's ancestors, the bodies those cells hold, and the
 * bodies it meets directly (itself included): the last two sum to n.
 * Returns -1 for bad arguments.
 */
int oracle_fmm_forces(int64_t n, const double *x, const double *m, double G, double eps,
                      double theta, int p, int leaf_cap, double *acc, int64_t *stats,
                      int64_t *cnt)
{
    if (leaf_cap < 1 || p < 1 || p > FMM_MAX_ORDER || !(theta >= 0.0)) return -1;
    if (n <= 0) return 0;
    bh_prep P;
    bh_prepare(&P, n, x, m, theta, leaf_cap);
    const bh_tree *t = &P.t;
    const int64_t nn = t->nnodes;
    fmm_basis B;
    fmm_basis_init(&B, p);
    const int nt = B.nt;

    fmm_trav T;
    T.P = &P;
    T.nn = nn;
    T.err = 0;
    T.leaf = (int *)malloc(sizeof(int) * (size_t)nn);
    T.ci = (int(*)[3])malloc(sizeof(int[3]) * (size_t)nn);
    T.m2l = (fmm_list *)calloc((size_t)nn, sizeof(fmm_list));
    T.p2p = (fmm_list *)calloc((size_t)nn, sizeof(fmm_list));
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)nn);
    double(*z)[3] = (double(*)[3])malloc(sizeof(double[3]) * (size_t)nn);
    parent[0] = -1;
    for (int64_t id = 0; id < nn; ++id) {
        const bh_node *nd = &t->nodes[id];
        int leaf = 1;
        for (int o = 0; o < 8; ++o)
            if (nd->child[o] >= 0) {
                leaf = 0;
                parent[nd->child[o]] = id;
            }
        T.leaf[id] = leaf;
        uint32_t ic[3] = {0, 0, 0};
        for (int b = 0; b < nd->level; ++b) {
            uint32_t trip = (nd->prefix >> (3 * b)) & 7u;
            for (int c = 0; c < 3; ++c) ic[c] |= ((trip >> c) & 1u) << b;
        }
        double cell = P.ext / (double)(1u << nd->level);
        for (int c = 0; c < 3; ++c) {
            T.ci[id][c] = (int)((2u * ic[c] + 1u) << (10 - nd->level));
            z[id][c] = P.box_lo[c] + cell * ((double)ic[c] + 0.5);
        }
    }
    for (int la = 0; la <= 10; ++la)
        for (int lb = 0; lb <= 10; ++lb) {
            double s = (double)((1 << (11 - la)) + (1 << (11 - lb)));
            T.crit[la][lb] = 0.75 * s * s / (theta * theta);
        }
    int32_t root = 0;
    fmm_down(&T, 0, &root, 1);

    /* moments of every cell, from its own bodies */
    double *Mh = (double *)calloc((size_t)(nn * nt), sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t id = 0; id < nn; ++id) {
        const bh_node *nd = &t->nodes[id];
        for (int64_t k = nd->start; k < nd->end; ++k) {
            int64_t j = P.perm[k];
            fmm_moments_add(&B, x + 3 * j, m[j], z[id], Mh + id * nt);
        }
    }
    /* local expansion of every cell from its own source cells */
    double *L = (double *)calloc((size_t)(nn * nt), sizeof(double));
#pragma omp parallel
    {
        double *Tn = (double *)malloc(sizeof(double) * (size_t)nt);
        double *work = (double *)malloc(sizeof(double) * (size_t)((p + 1) * nt));
#pragma omp for schedule(dynamic, 4)
        for (int64_t a = 0; a < nn; ++a) {
            for (int64_t q = 0; q < T.m2l[a].n; ++q) {
                int64_t b = T.m2l[a].v[q];
                double r[3];
                for (int c = 0; c < 3; ++c) r[c] = z[a][c] - z[b][c];
                fmm_local_add(&B, Mh + b * nt, r, eps, L + a * nt, Tn, work);
            }
        }
        free(Tn);
        free(work);
    }
    /* every body: the far field of its leaf and the leaf's ancestors, and
     * its direct partners */
    int64_t npairs = 0, nexp = 0, nleaves = 0;
    for (int64_t a = 0; a < nn; ++a) {
        nexp += T.m2l[a].n;
        nleaves += T.leaf[a];
    }
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : npairs)
    for (int64_t a = 0; a < nn; ++a) {
        if (!T.leaf[a]) continue;
        const bh_node *na = &t->nodes[a];
        int64_t ncells = 0, nfar = 0, nnear = 0;
        for (int64_t q = 0; q < T.p2p[a].n; ++q) {
            const bh_node *nb = &t->nodes[T.p2p[a].v[q]];
            nnear += nb->end - nb->start;
        }
        for (int64_t an = a; an >= 0; an = parent[an])
            for (int64_t q = 0; q < T.m2l[an].n; ++q) {
                const bh_node *nb = &t->nodes[T.m2l[an].v[q]];
                ++ncells;
                nfar += nb->end - nb->start;
            }
        npairs += nnear * (na->end - na->start);
        for (int64_t k = na->start; k < na->end; ++k) {
            int64_t i = P.perm[k];
            double ai[3] = {0, 0, 0};
            for (int64_t an = a; an >= 0; an = parent[an]) {
                double u[3];
                for (int c = 0; c < 3; ++c) u[c] = x[3 * i + c] - z[an][c];
                fmm_grad_add(&B, L + an * nt, u, ai);
            }
            for (int64_t q = 0; q < T.p2p[a].n; ++q) {
                const bh_node *nb = &t->nodes[T.p2p[a].v[q]];
                for (int64_t kk = nb->start; kk < nb->end; ++kk) {
                    int64_t j = P.perm[kk];
                    if (j == i) continue;
                    double d[3], s2 = eps * eps;
                    for (int c = 0; c < 3; ++c) {
                        d[c] = x[3 * j + c] - x[3 * i + c];
                        s2 += d[c] * d[c];
                    }
                    double w = m[j] / (s2 * sqrt(s2));
                    for (int c = 0; c < 3; ++c) ai[c] += w * d[c];
                }
            }
            for (int c = 0; c < 3; ++c) acc[3 * i + c] = G * ai[c];
            if (cnt) {
                cnt[3 * i] = ncells;
                cnt[3 * i + 1] = nfar;
                cnt[3 * i + 2] = nnear;
            }
        }
    }
    if (stats) {
        stats[0] = nn;
        stats[1] = nleaves;
        stats[2] = nexp;
        stats[3] = npairs;
    }
    int err = T.err;
    for (int64_t a = 0; a < nn; ++a) {
        free(T.m2l[a].v);
        free(T.p2p[a].v);
    }
    free(T.m2l); free(T.p2p); free(T.leaf); free(T.ci);
    free(parent); free(z); free(Mh); free(L);
    fmm_basis_free(&B);
    bh_release(&P);
    return err ? -2 : 0;
}
