// C ABI of libnbody.so (declared in include/nbody.h): argument checking,
// scratch ownership, kernel selection and split scheduling, the leapfrog
// loop, graph capture and the batched work queue.  Host code only; the
// arithmetic lives in the .cu files.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <tuple>
#include <vector>

#include "nb_internal.h"

using nb::BatchItem;
using nb::KernelEntry;

namespace {

thread_local std::string g_create_error;

nb_status failf(nb_ctx *c, nb_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->last_error = buf;
    else
        g_create_error = buf;
    return s;
}

#define NB_CUDA(ctx, call)                                                                     \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return failf(ctx, NB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

#define NB_TRY(expr)                       \
    do {                                   \
        nb_status s_ = (expr);             \
        if (s_ != NB_OK) return s_;        \
    } while (0)

// Makes ctx->device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

// ----------------------------------------------------------- pointer checks
typedef CUresult (*PfnGetAddressRange)(CUdeviceptr *, size_t *, CUdeviceptr);

PfnGetAddressRange address_range_fn()
{
    static PfnGetAddressRange fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 3020, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (PfnGetAddressRange)p;
    }();
    return fn;
}

// A device array of `bytes` bytes: non-null, 8-byte aligned, device (or
// managed) memory of the context's device, lying inside one allocation.
nb_status check_dev(nb_ctx *c, const void *p, size_t bytes, const char *name)
{
    if (bytes == 0) return NB_OK;
    if (!p) return failf(c, NB_EINVAL, "%s is NULL", name);
    if ((uintptr_t)p % 8) return failf(c, NB_EINVAL, "%s is not 8-byte aligned", name);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return failf(c, NB_EINVAL, "%s is not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return failf(c, NB_EINVAL, "%s is not device memory", name);
    if (a.type == cudaMemoryTypeDevice && a.device != c->device)
        return failf(c, NB_EINVAL, "%s is on device %d, context on %d", name, a.device, c->device);
    if (PfnGetAddressRange f = address_range_fn()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (f(&base, &size, (CUdeviceptr)(uintptr_t)p) == CUDA_SUCCESS) {
            if ((uintptr_t)p + bytes > (uintptr_t)base + size)
                return failf(c, NB_EINVAL, "%s: %zu bytes do not fit in its allocation", name,
                             bytes);
        }
    }
    return NB_OK;
}

nb_status check_scalars(nb_ctx *c, double G, double eps)
{
    if (!std::isfinite(G)) return failf(c, NB_EINVAL, "G is not finite");
    if (!std::isfinite(eps) || eps < 0) return failf(c, NB_EINVAL, "eps must be finite and >= 0");
    return NB_OK;
}

nb_status check_n(nb_ctx *c, int64_t n)
{
    if (n < 0 || n > c->n_max)
        return failf(c, NB_EINVAL, "n = %lld outside [0, n_max = %lld]", (long long)n,
                     (long long)c->n_max);
    return NB_OK;
}

// ----------------------------------------------------------- kernel choice
// Float64 state in the packed bodies (double4), float64 adjoint: NB_FP64 and
// the double-float NB_DF64.
bool f64_like(nb_precision p) { return p == NB_FP64 || p == NB_DF64; }
bool is_f64(const nb_ctx *c) { return f64_like(c->prec); }

int variant_count(int kind, nb_precision p)
{
    switch (kind) {
    case nb::KIND_FORCE:
        return p == NB_FP64   ? nb::f64_force_variants()
               : p == NB_DF64 ? nb::df_force_variants()
                              : nb::f32_force_variants();
    case nb::KIND_BATCHED: return f64_like(p) ? 0 : nb::f32_batched_variants();
    case nb::KIND_VJP: return f64_like(p) ? nb::f64_vjp_variants() : nb::f32_vjp_variants();
    default: return 0;
    }
}

const KernelEntry &kernel_for(int kind, nb_precision p, int v, bool zeps)
{
    const bool comp = p == NB_FP32_COMP;
    switch (kind) {
    case nb::KIND_FORCE:
        return p == NB_FP64   ? nb::f64_force_kernel(v, zeps)
               : p == NB_DF64 ? nb::df_force_kernel(v, zeps)
                              : nb::f32_force_kernel(v, comp, zeps);
    case nb::KIND_BATCHED: return nb::f32_batched_kernel(v, comp, zeps);
    default: return f64_like(p) ? nb::f64_vjp_kernel(v, zeps) : nb::f32_vjp_kernel(v, zeps);
    }
}

// Untuned defaults.
int default_variant(int kind, nb_precision p, int64_t n)
{
    // double-float: 128-body tiles (more CTAs, more compact tiles) below 4096 bodies
    if (kind == nb::KIND_FORCE && p == NB_DF64) return n < 4096 ? 2 : 0;
    return 0;
}

void pick(nb_ctx *c, int kind, int64_t n, int &variant, int &split)
{
    variant = default_variant(kind, c->prec, n);
    split = 0;
    for (const auto &e : c->tune[kind])
        if (n >= e.lo && n < e.hi) {
            variant = e.variant;
            split = e.split;
        }
}

int occupancy(nb_ctx *c, const KernelEntry &k)
{
    auto it = c->occ.find(k.fn);
    if (it != c->occ.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.fn, k.T, 0) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    nb = nb < 1 ? 1 : nb;
    c->occ[k.fn] = nb;
    return nb;
}

cudaEvent_t pooled_event(nb_ctx *c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Launch a pair kernel; `kind` tags its event timing (nb_profile).
nb_status launch(nb_ctx *c, const KernelEntry &k, int64_t grid, void *params, cudaStream_t s,
                 int kind)
{
    if (grid <= 0) return NB_OK;
    if (grid > 0x7fffffffLL) return failf(c, NB_EINVAL, "grid of %lld CTAs too large", (long long)grid);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    const bool timed = c->prof_on && cs == cudaStreamCaptureStatusNone;
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (timed) {
        ea = pooled_event(c);
        eb = pooled_event(c);
        if (ea && eb) NB_CUDA(c, cudaEventRecord(ea, s));
    }
    void *args[] = {params};
    NB_CUDA(c, cudaLaunchKernel(k.fn, dim3((unsigned)grid), dim3(k.T), args, 0, s));
    c->launches++;
    if (timed && ea && eb) {
        NB_CUDA(c, cudaEventRecord(eb, s));
        c->prof.push_back({kind, ea, eb});
    }
    return NB_OK;
}

#define NB_LAUNCHED(ctx, expr)     \
    do {                           \
        NB_CUDA(ctx, (expr));      \
        (ctx)->launches++;         \
    } while (0)

// Number of j-splits for a pair kernel over n bodies (see nb_choose_split).
int splits_for(nb_ctx *c, const KernelEntry &k, int64_t n, int forced, int64_t per_split_doubles)
{
    const int64_t tile = (int64_t)k.T * k.I;
    const int64_t n_itiles = (n + tile - 1) / tile;
    const int64_t n_jtiles = (n + k.J - 1) / k.J;
    const int64_t cap = c->partial_bodies * 4 / per_split_doubles;  // body-splits that fit
    int s;
    if (forced > 0)
        s = (int)std::min<int64_t>(forced, n_jtiles);
    else
        s = nb::choose_split(n_itiles, n_jtiles, (int64_t)c->num_sms * occupancy(c, k), cap, tile);
    while (s > 1 && (int64_t)s * n > cap) --s;
    if (s > 1 && n_itiles > c->n_counters) s = 1;
    return s < 1 ? 1 : s;
}

// float4 slots between the arrays of the float32 pack (hi, lo, cotangent).
size_t pack_stride(const nb_ctx *c) { return (size_t)std::max<int64_t>(c->n_max, 1); }

// Second array of the float32 pack buffer: the lo parts of the hi/lo pairs.
float4 *lo_half(nb_ctx *c) { return (float4 *)c->pack + pack_stride(c); }

// ------------------------------------------------------------- force paths
// Force on the already packed bodies; optional fused half-kick of vel.
nb_status force_packed(nb_ctx *c, cudaStream_t s, int64_t n, double G, double eps, double *acc,
                       double *vel, double half_dt)
{
    if (n == 0) return NB_OK;
    const bool zeps = eps == 0.0;
    int v, forced;
    pick(c, nb::KIND_FORCE, n, v, forced);
    const KernelEntry &k = kernel_for(nb::KIND_FORCE, c->prec, v, zeps);
    const int S = splits_for(c, k, n, forced, 3);
    nb::ForceParams p;
    p.P = c->pack;
    p.Plo = is_f64(c) ? nullptr : lo_half(c);
    p.perm = c->perm_active ? c->perm : nullptr;
    p.n = (int)n;
    p.nsplit = S;
    p.eps2f = (float)(eps * eps);
    p.eps2 = eps * eps;
    p.G = G;
    p.acc = acc;
    p.vel = vel;
    p.half_dt = half_dt;
    p.partial = c->partial;
    p.counters = c->counters;
    p.err = c->err;
    const int64_t tile = (int64_t)k.T * k.I;
    return launch(c, k, (n + tile - 1) / tile * S, &p, s, 0);
}

// Whether force calls with n bodies process them in Morton order: float32
// modes from order_min_n bodies on; the double-float mode always (unless
// mode 0), as its accuracy on close pairs rests on compact tiles.
bool use_order(const nb_ctx *c, int64_t n)
{
    if (c->prec == NB_FP64 || !c->perm) return false;
    if (c->prec == NB_DF64) return c->order_mode != 0;
    return c->order_mode == 1 || (c->order_mode == 2 && n >= c->order_min_n);
}

// Pack bodies for a force call: float64 (x,y,z,m) in FP64 mode; float32
// hi/lo pairs otherwise, in Morton order when use_order() holds (never for
// the batched kernel, allow_order = false).
nb_status pack(nb_ctx *c, cudaStream_t s, int64_t n, const double *pos, const double *mass,
               bool allow_order = true)
{
    if (n == 0) return NB_OK;
    c->perm_active = allow_order && use_order(c, n);
    if (is_f64(c)) {
        if (c->perm_active) {
            int k = 0;
            NB_CUDA(c, nb::launch_morton_sort(s, (int)n, pos, c->order, c->perm, k));
            c->launches += k;
        }
        NB_LAUNCHED(c, nb::launch_pack_f64(s, (int)n, pos, mass, (double4 *)c->pack,
                                           c->perm_active ? c->perm : nullptr));
        return NB_OK;
    }
    if (c->perm_active) {
        int k = 0;
        NB_CUDA(c, nb::launch_morton_sort(s, (int)n, pos, c->order, c->perm, k));
        c->launches += k;
    }
    NB_LAUNCHED(c, nb::launch_pack_hilo(s, (int)n, pos, mass, c->perm_active ? c->perm : nullptr,
                                        (float4 *)c->pack, lo_half(c)));
    return NB_OK;
}

// Forward leapfrog loop (shared by nb_step, nb_rollout and the graph body).
nb_status rollout_enqueue(nb_ctx *c, cudaStream_t s, int64_t n, double *pos, double *vel,
                          const double *mass, double G, double eps, double dt, int64_t nsteps,
                          double *acc, unsigned flags, int64_t every, double *rec_pos,
                          double *rec_vel)
{
    if (n == 0) return NB_OK;
    if (!(flags & NB_ACC_VALID)) {
        NB_TRY(pack(c, s, n, pos, mass));
        NB_TRY(force_packed(c, s, n, G, eps, acc, nullptr, 0.0));
    }
    const size_t rec = (size_t)n * 3;
    const bool order = use_order(c, n);
    for (int64_t st = 0; st < nsteps; ++st) {
        double *rp = nullptr, *rv = nullptr;
        if (every > 0 && st % every == 0) {
            rp = rec_pos + rec * (size_t)(st / every);
            rv = rec_vel ? rec_vel + rec * (size_t)(st / every) : nullptr;
        }
        // kick + drift; it also repacks unless the bodies are re-ordered first
        NB_LAUNCHED(c, nb::launch_kdp(s, is_f64(c), (int)n, pos, vel, acc, mass, 0.5 * dt, dt,
                                      order ? nullptr : c->pack, lo_half(c), rp, rv));
        if (order) {
            NB_TRY(pack(c, s, n, pos, mass));
        } else {
            c->perm_active = false;
        }
        NB_TRY(force_packed(c, s, n, G, eps, acc, vel, 0.5 * dt));
    }
    if (every > 0 && nsteps % every == 0) {
        const size_t r = (size_t)(nsteps / every);
        NB_CUDA(c, cudaMemcpyAsync(rec_pos + rec * r, pos, rec * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
        if (rec_vel)
            NB_CUDA(c, cudaMemcpyAsync(rec_vel + rec * r, vel, rec * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
    }
    return NB_OK;
}

// ------------------------------------------------------------------ adjoint
nb_status vjp_packed(nb_ctx *c, cudaStream_t s, int64_t n, double G, double eps, double *gx,
                     double *gm, int accumulate)
{
    if (n == 0) return NB_OK;
    const bool zeps = eps == 0.0;
    int v, forced;
    pick(c, nb::KIND_VJP, n, v, forced);
    const KernelEntry &k = kernel_for(nb::KIND_VJP, c->prec, v, zeps);
    const int S = splits_for(c, k, n, forced, 4);
    nb::VjpParams p;
    p.PV = c->pack;
    p.Plo = is_f64(c) ? nullptr : lo_half(c);
    p.Plam = is_f64(c) ? nullptr : lo_half(c) + std::max<int64_t>(c->n_max, 1);
    p.n = (int)n;
    p.nsplit = S;
    p.eps2f = (float)(eps * eps);
    p.eps2 = eps * eps;
    p.G = G;
    p.gx = gx;
    p.gm = gm;
    p.accumulate = accumulate;
    p.partial = c->partial;
    p.counters = c->counters;
    p.err = c->err;
    const int64_t tile = (int64_t)k.T * k.I;
    return launch(c, k, (n + tile - 1) / tile * S, &p, s, 2);
}

// ------------------------------------------------------------------ batched
nb_status batched_force(nb_ctx *c, cudaStream_t s, double G, double eps, double *acc, double *vel,
                        double half_dt)
{
    if (c->n_items == 0) return NB_OK;
    const KernelEntry &k = kernel_for(nb::KIND_BATCHED, c->prec, c->batch_variant, eps == 0.0);
    const int64_t slots = (int64_t)c->num_sms * occupancy(c, k);
    nb::BatchParams p;
    p.P = (const float4 *)c->pack;
    p.Plo = lo_half(c);
    p.items = c->items;
    p.n_items = (int)c->n_items;
    p.queue = c->queue;
    p.partial = c->partial;
    p.counters = c->counters;
    p.eps2f = (float)(eps * eps);
    p.G = G;
    p.acc = acc;
    p.vel = vel;
    p.half_dt = half_dt;
    p.err = c->err;
    return launch(c, k, std::min<int64_t>(slots, c->n_items), &p, s, 1);
}

nb_status batched_enqueue(nb_ctx *c, cudaStream_t s, double *pos, double *vel, const double *mass,
                          double G, double eps, double dt, int64_t nsteps, double *acc,
                          unsigned flags)
{
    const int64_t n = c->batch_n;
    if (n == 0) return NB_OK;
    if (!(flags & NB_ACC_VALID)) {
        NB_TRY(pack(c, s, n, pos, mass, false));
        NB_TRY(batched_force(c, s, G, eps, acc, nullptr, 0.0));
    }
    for (int64_t st = 0; st < nsteps; ++st) {
        NB_LAUNCHED(c, nb::launch_kdp(s, false, (int)n, pos, vel, acc, mass, 0.5 * dt, dt, c->pack,
                                      lo_half(c), nullptr, nullptr));
        NB_TRY(batched_force(c, s, G, eps, acc, vel, 0.5 * dt));
    }
    return NB_OK;
}

// ------------------------------------------------------------ graph capture
// Runs `body` captured once as a CUDA graph on the library's capture stream,
// ordered after prior work on the caller's stream (events both ways).
nb_status run_graph(nb_ctx *c, const nb_ctx::GraphKey &key,
                    const std::function<nb_status(cudaStream_t)> &body)
{
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        const int64_t saved = c->launches;
        NB_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        nb_status st = body(c->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        const int64_t kernels = c->launches - saved;
        c->launches = saved;
        if (st != NB_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess)
            return failf(c, NB_ECUDA, "cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess)
            return failf(c, NB_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
        it = c->graphs.emplace(key, nb_ctx::GraphVal{ex, kernels}).first;
    }
    NB_CUDA(c, cudaEventRecord(c->ev_in, c->stream));
    NB_CUDA(c, cudaStreamWaitEvent(c->cap_stream, c->ev_in, 0));
    NB_CUDA(c, cudaGraphLaunch(it->second.exec, c->cap_stream));
    NB_CUDA(c, cudaEventRecord(c->ev_out, c->cap_stream));
    NB_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_out, 0));
    c->launches += it->second.kernels;
    return NB_OK;
}

void drop_graphs(nb_ctx *c)
{
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
}

template <typename T>
T *dev_alloc(nb_ctx *c, size_t count, nb_status &st)
{
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        st = failf(c, NB_ENOMEM, "cudaMalloc of %zu bytes failed", count * sizeof(T));
        return nullptr;
    }
    return (T *)p;
}

void free_tree_nodes(nb_ctx *c)
{
    nb::TreeView &t = c->tree;
    void *arrays[] = {t.start, t.end,   t.level,  t.nchild, t.first, t.offs, t.parent,
                      t.arrive, t.prefix, t.M,  t.com,    t.box_lo, t.box_hi, t.chi, t.clo};
    for (void *a : arrays) cudaFree(a);
    t.start = t.end = t.level = t.nchild = t.first = t.offs = t.parent = t.arrive = nullptr;
    t.prefix = nullptr;
    t.M = t.com = nullptr;
    t.box_lo = t.box_hi = t.chi = t.clo = nullptr;
    t.cap = 0;
}

void free_fmm(nb_ctx *c)
{
    nb::FmmView &f = c->fmm;
    void *arrays[] = {f.ci,       f.nd,       f.M,      f.L,        f.down,     f.cum,
                      f.leaves,   f.nearc,    f.item_off, f.part_off,
                      f.part,     f.pool,     f.chunk_head, f.chunk_src, f.chunk_next,
                      f.rhead,    f.rchunk,   f.rnext};
    for (void *a : arrays) cudaFree(a);
    f.ci = f.nd = nullptr;
    f.M = f.L = nullptr;
    f.down = f.cum = nullptr;
    f.leaves = f.nearc = f.item_off = f.part_off = f.pool = nullptr;
    f.chunk_head = f.chunk_src = f.chunk_next = nullptr;
    f.rhead = f.rnext = nullptr;
    f.rchunk = nullptr;
    f.part = nullptr;
    f.pool_cap = f.part_cap = f.chunk_cap = f.rchunk_cap = 0;
    c->fmm_cap = c->fmm_np = 0;
}

void free_ctx(nb_ctx *c)
{
    drop_graphs(c);
    for (auto &r : c->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    cudaFree(c->pack);
    cudaFree(c->partial);
    cudaFree(c->counters);
    cudaFree(c->red);
    cudaFree(c->dev_out);
    cudaFree(c->err);
    cudaFree(c->queue);
    cudaFree(c->items);
    cudaFree(c->perm);
    cudaFree(c->order.box);
    cudaFree(c->order.keys[0]);
    cudaFree(c->order.keys[1]);
    cudaFree(c->order.vals[0]);
    cudaFree(c->order.vals[1]);
    cudaFree(c->order.hist);
    free_tree_nodes(c);
    free_fmm(c);
    cudaFree(c->fmm.meta);
    cudaFree(c->fmm.stats);
    cudaFree(c->fmm.crit);
    cudaFree(c->tree.meta);
    cudaFree(c->tree.stats);
    cudaFree(c->tree_P);
    cudaFree(c->tree_Plo);
    cudaFree(c->tree_perm);
    cudaFree(c->tree_box);
    cudaFree(c->orb_buf);
    cudaFree(c->orb_perm);
    cudaFree(c->let.kind);
    cudaFree(c->let.nidx);
    cudaFree(c->let.boff);
    cudaFree(c->let.totals);
    cudaFree(c->let_box);
    cudaFree(c->let_queue);
    cudaFree(c->let_src);
    cudaFree(c->let_tpart);
    cudaFree(c->let_tcnt);
    cudaFree(c->let_tctr);
    if (c->host_out) cudaFreeHost(c->host_out);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    delete c;
}

// ---------------------------------------------------------------- tree code
// Morton-sort scratch (float64 contexts allocate it on first tree call).
nb_status ensure_order(nb_ctx *c)
{
    if (c->order.hist) return NB_OK;
    nb_status st = NB_OK;
    const size_t nc = (size_t)std::max<int64_t>(c->n_max, 1);
    if (!c->order.box) c->order.box = dev_alloc<double>(c, 1024 * 6, st);
    for (int q = 0; q < 2 && st == NB_OK; ++q) {
        if (!c->order.keys[q]) c->order.keys[q] = dev_alloc<unsigned>(c, nc, st);
        if (st == NB_OK && !c->order.vals[q]) c->order.vals[q] = dev_alloc<int>(c, nc, st);
    }
    if (st == NB_OK)
        c->order.hist = dev_alloc<unsigned>(c, nb::sort_hist_entries((int)nc), st);
    return st;
}

// Tree scratch for leaves of up to leaf_cap bodies: body arrays for n_max
// bodies and node arrays for tree_node_bound(n_max, leaf_cap) nodes.  Growing
// the node arrays frees the old ones (cudaFree synchronises the device) and
// drops captured graphs, which hold the old addresses.
nb_status ensure_tree(nb_ctx *c, int leaf_cap)
{
    NB_TRY(ensure_order(c));
    nb_status st = NB_OK;
    const size_t nc = (size_t)std::max<int64_t>(c->n_max, 1);
    if (!c->tree_box) {
        c->tree_P = dev_alloc<float4>(c, nc, st);
        if (st == NB_OK) c->tree_Plo = dev_alloc<float4>(c, nc, st);
        if (st == NB_OK) c->tree_perm = dev_alloc<int>(c, nc, st);
        if (st == NB_OK) c->tree.meta = dev_alloc<int>(c, (size_t)nb::tree_meta_ints(), st);
        if (st == NB_OK) c->tree.stats = dev_alloc<unsigned long long>(c, 4, st);
        if (st == NB_OK) c->tree_box = dev_alloc<double>(c, 4, st);
        if (st != NB_OK) return st;
    }
    const int64_t need = nb::tree_node_bound((int64_t)nc, leaf_cap);
    if (need <= c->tree.cap) return NB_OK;
    if (need > 0x7fffffffLL)
        return failf(c, NB_ENOMEM, "tree of %lld nodes too large", (long long)need);
    drop_graphs(c);
    free_tree_nodes(c);
    nb::TreeView &t = c->tree;
    const size_t m = (size_t)need;
    int **ints[] = {&t.start, &t.end, &t.level, &t.nchild, &t.first, &t.offs, &t.parent, &t.arrive};
    for (int **a : ints)
        if (st == NB_OK) *a = dev_alloc<int>(c, m, st);
    if (st == NB_OK) t.prefix = dev_alloc<unsigned>(c, m, st);
    if (st == NB_OK) t.M = dev_alloc<double>(c, m, st);
    if (st == NB_OK) t.com = dev_alloc<double>(c, 3 * m, st);
    float4 **f4[] = {&t.box_lo, &t.box_hi, &t.chi, &t.clo};
    for (float4 **a : f4)
        if (st == NB_OK) *a = dev_alloc<float4>(c, m, st);
    if (st != NB_OK) {
        free_tree_nodes(c);
        return st;
    }
    t.cap = (int)need;
    return NB_OK;
}

nb_status check_tree_args(nb_ctx *c, double theta, int leaf_cap, int group)
{
    if (group != 32 && group != 64) return failf(c, NB_EINVAL, "group = %d is not 32 or 64", group);
    if (!std::isfinite(theta) || theta < 0)
        return failf(c, NB_EINVAL, "theta must be finite and >= 0");
    if (leaf_cap < 1 || leaf_cap > NB_TREE_MAX_LEAF)
        return failf(c, NB_EINVAL, "leaf_cap = %d outside [1, %d]", leaf_cap, NB_TREE_MAX_LEAF);
    return NB_OK;
}

// Chunked list store (chunks of FMM_CHUNK entries and their links) of at
// least `need` chunks.
template <class T>
nb_status ensure_chunks(nb_ctx *c, long long need, T *&store, int *&next, long long &cap,
                        const char *what)
{
    if (need <= cap) return NB_OK;
    if (need > 0x7fffffffLL / nb::FMM_CHUNK)
        return failf(c, NB_ENOMEM, "FMM %s of %lld chunks too large", what, need);
    cudaFree(store);
    cudaFree(next);
    store = nullptr;
    next = nullptr;
    cap = 0;
    nb_status st = NB_OK;
    store = dev_alloc<T>(c, (size_t)need * nb::FMM_CHUNK, st);
    if (st == NB_OK) next = dev_alloc<int>(c, (size_t)need, st);
    if (st != NB_OK) {
        cudaFree(store);
        store = nullptr;
        return st;
    }
    cap = need;
    return NB_OK;
}

// Expansion, list and candidate-pool scratch of the fast multipole method
// for the tree's node capacity and `order`; the pool holds at least
// pool_need entries, the expansion lists at least chunk_need chunks and the
// leaves' direct-range lists at least rchunk_need.  Growing frees the old
// arrays (cudaFree synchronises).
nb_status ensure_fmm(nb_ctx *c, int order, long long pool_need, long long chunk_need,
                     long long rchunk_need)
{
    nb_status st = NB_OK;
    nb::FmmView &f = c->fmm;
    if (!f.meta) f.meta = dev_alloc<int>(c, nb::FMM_META_INTS, st);
    if (st == NB_OK && !f.stats) f.stats = dev_alloc<unsigned long long>(c, 4, st);
    if (st == NB_OK && !f.crit) f.crit = dev_alloc<int>(c, nb::FMM_CRIT_INTS, st);
    if (st != NB_OK) return st;
    const int np = nb::fmm_floats(order);
    const int cap = c->tree.cap;
    if (cap > c->fmm_cap || np > c->fmm_np) {
        const long long keep_pool = f.pool_cap, keep_chunks = f.chunk_cap,
                        keep_rchunks = f.rchunk_cap;
        free_fmm(c);
        const size_t m = (size_t)cap;
        f.ci = dev_alloc<int4>(c, m, st);
        if (st == NB_OK) f.nd = dev_alloc<int4>(c, m, st);
        if (st == NB_OK) f.M = dev_alloc<float>(c, m * (size_t)np, st);
        if (st == NB_OK) f.L = dev_alloc<float>(c, m * (size_t)np, st);
        if (st == NB_OK) f.down = dev_alloc<int2>(c, m, st);
        if (st == NB_OK) f.cum = dev_alloc<int2>(c, m, st);
        if (st == NB_OK) f.leaves = dev_alloc<int>(c, m, st);
        if (st == NB_OK) f.nearc = dev_alloc<int>(c, m, st);
        if (st == NB_OK) f.item_off = dev_alloc<int>(c, m + 1, st);
        if (st == NB_OK) f.part_off = dev_alloc<int>(c, m + 1, st);
        if (st == NB_OK) f.chunk_head = dev_alloc<int>(c, m, st);
        if (st == NB_OK) f.rhead = dev_alloc<int>(c, m, st);
        if (st != NB_OK) {
            free_fmm(c);
            return st;
        }
        c->fmm_cap = cap;
        c->fmm_np = np;
        pool_need = std::max(pool_need, keep_pool);
        chunk_need = std::max(chunk_need, keep_chunks);
        rchunk_need = std::max(rchunk_need, keep_rchunks);
    }
    NB_TRY(ensure_chunks(c, chunk_need, f.chunk_src, f.chunk_next, f.chunk_cap, "expansion lists"));
    NB_TRY(ensure_chunks(c, rchunk_need, f.rchunk, f.rnext, f.rchunk_cap, "direct-range lists"));
    if (pool_need > f.pool_cap) {
        if (pool_need > 0x7fffffffLL)
            return failf(c, NB_ENOMEM, "FMM candidate lists of %lld entries too large", pool_need);
        cudaFree(f.pool);
        f.pool = dev_alloc<int>(c, (size_t)pool_need, st);
        if (st != NB_OK) {
            f.pool_cap = 0;
            return st;
        }
        f.pool_cap = pool_need;
    }
    return NB_OK;
}

nb_status check_fmm_args(nb_ctx *c, double theta, int order, int leaf_cap)
{
    if (!std::isfinite(theta) || theta < 0)
        return failf(c, NB_EINVAL, "theta must be finite and >= 0");
    if (order < nb::FMM_MIN_ORDER || order > nb::FMM_MAX_ORDER)
        return failf(c, NB_EINVAL, "order = %d outside [%d, %d]", order, nb::FMM_MIN_ORDER,
                     nb::FMM_MAX_ORDER);
    if (leaf_cap < 1 || leaf_cap > nb::FMM_MAX_LEAF)
        return failf(c, NB_EINVAL, "leaf_cap = %d outside [1, %d]", leaf_cap, nb::FMM_MAX_LEAF);
    return NB_OK;
}

// Events around a tree-code launch sequence (nb_profile), outside captures.
struct TreeTimer {
    nb_ctx *c;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    TreeTimer(nb_ctx *c_, int kind_, cudaStream_t s_) : c(c_), kind(kind_), s(s_)
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &cs);
        if (!c->prof_on || cs != cudaStreamCaptureStatusNone) return;
        a = pooled_event(c);
        b = pooled_event(c);
        if (a && b) cudaEventRecord(a, s);
    }
    void done()
    {
        if (a && b && cudaEventRecord(b, s) == cudaSuccess) {
            c->prof.push_back({kind, a, b});
            a = b = nullptr;
        }
    }
    ~TreeTimer()
    {
        if (a) c->ev_pool.push_back(a);
        if (b) c->ev_pool.push_back(b);
    }
};

// Sort, pack and build the tree over n bodies (kept in the context).
nb_status tree_build_enqueue(nb_ctx *c, cudaStream_t s, int64_t n, const double *pos,
                             const double *mass, int leaf_cap)
{
    int k = 0;
    TreeTimer tm(c, nb::PROF_TREE_BUILD, s);
    NB_CUDA(c, nb::launch_tree_sort(s, (int)n, pos, c->order, c->tree_perm, c->tree_box, k));
    c->launches += k;
    NB_LAUNCHED(c, nb::launch_pack_hilo(s, (int)n, pos, mass, c->tree_perm, c->tree_P,
                                        c->tree_Plo));
    NB_CUDA(c, nb::launch_tree_build(s, c->tree, (int)n, c->order.keys[0], c->tree_box, pos, mass,
                                     c->tree_perm, leaf_cap, c->err, k));
    c->launches += k;
    tm.done();
    return NB_OK;
}

// Sort, pack, build and walk: acc = G * (tree sum); vel += half_dt * acc when vel.
nb_status tree_forces_enqueue(nb_ctx *c, cudaStream_t s, int64_t n, const double *pos,
                              const double *mass, double G, double eps, double theta,
                              int leaf_cap, int group, double *acc, double *vel, double half_dt,
                              int *counts)
{
    if (n == 0) return NB_OK;
    int k = 0;
    c->let_n = 0;  // the local tree of nb_let_build is replaced
    NB_TRY(tree_build_enqueue(c, s, n, pos, mass, leaf_cap));
    nb::TreeWalkParams p;
    p.tree = c->tree;
    p.P = c->tree_P;
    p.Plo = c->tree_Plo;
    p.perm = c->tree_perm;
    p.sP = c->tree_P;
    p.sPlo = c->tree_Plo;
    p.box = c->tree_box;
    p.queue = c->tree.meta + nb::TREE_META_QUEUE;
    p.n = (int)n;
    p.group = group;
    p.sched = c->tree_sched;
    p.chunk = c->tree_chunk;
    p.num_sms = c->num_sms;
    p.accumulate = 0;
    p.theta = (float)theta;
    p.eps2f = (float)(eps * eps);
    p.G = G;
    p.acc = acc;
    p.vel = vel;
    p.half_dt = half_dt;
    p.counts = counts;
    p.err = c->err;
    p.more = nullptr;
    p.nmore = 0;
    p.tspan = 1;
    p.tpart = nullptr;
    p.tcnt = nullptr;
    p.tctr = nullptr;
    TreeTimer tm(c, nb::PROF_TREE_WALK, s);
    NB_CUDA(c, nb::launch_tree_walk(s, p, p.eps2f == 0.0f, k));
    c->launches += k;
    tm.done();
    return NB_OK;
}

// Partial-sum slots for the near field's split leaves.
nb_status ensure_fmm_part(nb_ctx *c, long long slots)
{
    nb::FmmView &f = c->fmm;
    if (slots <= f.part_cap) return NB_OK;
    nb_status st = NB_OK;
    cudaFree(f.part);
    const long long want = std::max(slots, f.part_cap * 3 / 2);
    f.part = dev_alloc<double>(c, 3 * (size_t)want, st);
    f.part_cap = st == NB_OK ? want : 0;
    return st;
}

// Sort, pack and build the tree, then the FMM passes; synchronises after the
// downward passes to see whether the candidate pool sufficed (if not, the
// pool grows and those passes run again) and how many partial sums the near
// field needs.
nb_status fmm_forces_run(nb_ctx *c, int64_t n, const double *pos, const double *mass, double G,
                         double eps, double theta, int order, int leaf_cap, double *acc,
                         int *counts, double *vel = nullptr, double half_dt = 0.0)
{
    cudaStream_t s = c->stream;
    int k = 0;
    c->let_n = 0;  // the local tree of nb_let_build is replaced
    {
        TreeTimer tm(c, nb::PROF_TREE_BUILD, s);
        NB_CUDA(c, nb::launch_tree_sort(s, (int)n, pos, c->order, c->tree_perm, c->tree_box, k));
        c->launches += k;
        NB_LAUNCHED(c, nb::launch_pack_hilo(s, (int)n, pos, mass, c->tree_perm, c->tree_P,
                                            c->tree_Plo));
        NB_CUDA(c, nb::launch_tree_build(s, c->tree, (int)n, c->order.keys[0], c->tree_box, pos,
                                         mass, c->tree_perm, leaf_cap, c->err, k));
        c->launches += k;
        tm.done();
    }
    for (int attempt = 0;; ++attempt) {
        nb::FmmParams p;
        p.tree = c->tree;
        p.f = c->fmm;
        p.f.order = order;
        p.f.np = nb::fmm_floats(order);
        p.P = c->tree_P;
        p.Plo = c->tree_Plo;
        p.perm = c->tree_perm;
        p.pos = pos;
        p.mass = mass;
        p.box = c->tree_box;
        p.n = (int)n;
        p.theta = theta;
        p.eps2 = eps * eps;
        p.eps2f = (float)(eps * eps);
        p.G = G;
        p.acc = acc;
        p.vel = vel;
        p.half_dt = half_dt;
        p.counts = counts;
        p.err = c->err;
        p.num_sms = c->num_sms;
        TreeTimer tm(c, nb::PROF_FMM_FAR, s);
        NB_CUDA(c, nb::launch_fmm(s, p, false, k));
        c->launches += k;
        tm.done();
        int meta[nb::FMM_META_INTS];
        NB_CUDA(c, cudaMemcpyAsync(meta, c->fmm.meta, sizeof(meta), cudaMemcpyDeviceToHost, s));
        NB_CUDA(c, cudaStreamSynchronize(s));
        if (!meta[nb::FMM_META_OVERFLOW]) {
            NB_TRY(ensure_fmm_part(c, std::max(1, meta[nb::FMM_META_PSLOTS])));
            p.f = c->fmm;
            p.f.order = order;
            p.f.np = nb::fmm_floats(order);
            TreeTimer tn(c, nb::PROF_FMM_NEAR, s);
            NB_CUDA(c, nb::launch_fmm(s, p, true, k));
            c->launches += k;
            tn.done();
            return NB_OK;
        }
        if (attempt == 8) return failf(c, NB_ENOMEM, "FMM candidate lists keep overflowing");
        // the counters hold what was asked for (past the end too); what the
        // cut-short passes did not reach, the next attempt asks for
        long long need = c->fmm.pool_cap, chunks = c->fmm.chunk_cap, rchunks = c->fmm.rchunk_cap;
        const int over = meta[nb::FMM_META_OVERFLOW];
        if (over & 1) need = std::max<long long>((unsigned)meta[nb::FMM_META_POOL], need) * 2;
        if (over & 2) chunks = std::max<long long>((unsigned)meta[nb::FMM_META_CHUNKS], chunks) * 2;
        if (over & 4) rchunks = std::max<long long>((unsigned)meta[nb::FMM_META_RCHUNKS], rchunks) * 2;
        NB_TRY(ensure_fmm(c, order, need, chunks, rchunks));
    }
}

nb_status tree_step_enqueue(nb_ctx *c, cudaStream_t s, int64_t n, double *pos, double *vel,
                            const double *mass, double G, double eps, double theta, int leaf_cap,
                            int group, double dt, int64_t nsteps, double *acc, unsigned flags)
{
    if (n == 0) return NB_OK;
    if (!(flags & NB_ACC_VALID))
        NB_TRY(tree_forces_enqueue(c, s, n, pos, mass, G, eps, theta, leaf_cap, group, acc,
                                   nullptr, 0.0, nullptr));
    for (int64_t st = 0; st < nsteps; ++st) {
        NB_LAUNCHED(c, nb::launch_kdp(s, is_f64(c), (int)n, pos, vel, acc, mass, 0.5 * dt, dt,
                                      nullptr, nullptr, nullptr, nullptr));
        NB_TRY(tree_forces_enqueue(c, s, n, pos, mass, G, eps, theta, leaf_cap, group, acc, vel,
                                   0.5 * dt, nullptr));
    }
    return NB_OK;
}

int min_tile_bodies()
{
    int m = 1 << 30;
    const nb_precision ps[] = {NB_FP64, NB_FP32, NB_FP32_COMP, NB_DF64};
    for (nb_precision p : ps)
        for (int kind = 0; kind < nb::KIND_COUNT; ++kind)
            for (int v = 0; v < variant_count(kind, p); ++v) {
                const KernelEntry &k = kernel_for(kind, p, v, false);
                m = std::min(m, k.T * k.I);
            }
    return std::max(m, 1);
}

}  // namespace

bool nb_ctx::GraphKey::operator<(const GraphKey &o) const
{
    return std::tie(kind, pos, vel, mass, acc, rec_pos, rec_vel, G, eps, dt, n, nsteps, every,
                    flags, plan_gen, theta, leaf_cap) <
           std::tie(o.kind, o.pos, o.vel, o.mass, o.acc, o.rec_pos, o.rec_vel, o.G, o.eps, o.dt,
                    o.n, o.nsteps, o.every, o.flags, o.plan_gen, o.theta, o.leaf_cap);
}

namespace nb {

int choose_split(int64_t n_itiles, int64_t n_jtiles, int64_t slots, int64_t max_split_bodies,
                 int64_t tile_bodies)
{
    if (n_itiles <= 0 || n_jtiles <= 0 || slots <= 0) return 1;
    auto score = [&](int64_t s) {
        const double items = (double)(n_itiles * s);
        const double waves = items / (double)slots;
        const double q = waves / std::ceil(waves);
        const double per_item = (double)n_jtiles / (double)s;  // j-tiles per item
        return q * per_item / (per_item + 1.0);
    };
    int64_t best_s = 1;
    double best = score(1);
    const int64_t smax = std::min<int64_t>(n_jtiles, 256);
    for (int64_t s = 2; s <= smax; ++s) {
        if (s * n_itiles * tile_bodies > max_split_bodies) break;
        const double sc = score(s);
        if (sc > best * 1.002) {
            best = sc;
            best_s = s;
        }
    }
    return (int)best_s;
}

}  // namespace nb

// ====================================================================== ABI
extern "C" {

int nb_choose_split(int64_t n_itiles, int64_t n_jtiles, int64_t slots, int64_t max_split_bodies,
                    int64_t tile_bodies)
{
    return nb::choose_split(n_itiles, n_jtiles, slots, max_split_bodies, tile_bodies);
}

int64_t nb_plan_batch_host(int64_t nsys, const int64_t *off, int T, int I, int J,
                           int64_t max_item_pairs, int32_t *items_out, int64_t max_items)
{
    if (nsys < 0 || !off || T <= 0 || I <= 0 || J <= 0 || (T & (T - 1))) return -1;
    if (off[0] != 0) return -1;
    for (int64_t k = 0; k < nsys; ++k)
        if (off[k + 1] < off[k] || off[k + 1] > 0x7fffffffLL) return -1;
    static_assert(sizeof(BatchItem) == nb::BATCH_ITEM_INTS * sizeof(int32_t), "item layout");
    const int64_t TI = (int64_t)T * I;
    int lmax = 1;  // lanes: a power of two, at most 32 (one warp), T and J
    while (lmax * 2 <= 32 && lmax * 2 <= T && lmax * 2 <= J) lmax *= 2;
    struct Cand { BatchItem it; int64_t cost; };
    std::vector<Cand> v;
    int ctr = 0, pbase = 0;
    // One piece: bodies [i0, i0 + cnt) of system k with `lanes` lanes, its j
    // range split into chunks while a piece would exceed max_item_pairs (a
    // shorter tail when the queue runs dry; the chunks' partial sums are
    // added in order, so results do not depend on which CTA ran which).
    auto piece = [&](int64_t k, int64_t i0, int64_t cnt, int lanes) {
        const int64_t nj = off[k + 1] - off[k];
        const int64_t ntiles = (nj + J - 1) / J;
        int64_t S = 1;
        if (max_item_pairs > 0) {
            const int64_t pairs = TI / lanes * nj;
            S = std::min<int64_t>((pairs + max_item_pairs - 1) / max_item_pairs, ntiles);
            S = std::max<int64_t>(S, 1);
        }
        for (int64_t c = 0; c < S; ++c) {
            const int64_t t0 = ntiles * c / S, t1 = ntiles * (c + 1) / S;
            BatchItem b;
            b.i0 = (int)i0;
            b.i_end = (int)(i0 + cnt);
            b.j0 = (int)(off[k] + t0 * J);
            b.j1 = (int)std::min(off[k] + t1 * J, off[k + 1]);
            b.lanes = lanes;
            b.sys = (int)k;
            b.ctr = S > 1 ? ctr : -1;
            b.pbase = S > 1 ? pbase : 0;
            b.chunk = (int)c;
            b.nchunks = (int)S;
            b.pad0 = b.pad1 = 0;
            v.push_back({b, (t1 - t0) * J / lanes});  // j-pairs per thread
        }
        if (S > 1) {
            ++ctr;
            pbase += (int)S;
        }
    };
    for (int64_t k = 0; k < nsys; ++k) {
        int64_t i = off[k];
        const int64_t e = off[k + 1];
        // full tiles, one lane per body
        for (; e - i >= TI; i += TI) piece(k, i, TI, 1);
        // the remainder r < TI in pieces of TI/lanes bodies (lanes = 2, 4,
        // ...): the smallest piece that covers r when it wastes at most an
        // eighth of its slots (or lanes are exhausted), else the largest
        // piece within r and continue with the rest
        while (i < e) {
            const int64_t r = e - i;
            int lanes = 1;
            while (lanes < lmax && TI / (lanes * 2) >= r) lanes *= 2;
            const int64_t cover = TI / lanes;  // smallest piece >= r
            if (lanes == lmax || (cover - r) * 8 <= cover) {
                piece(k, i, r, lanes);
                break;
            }
            piece(k, i, cover / 2, lanes * 2);
            i += cover / 2;
        }
    }
    std::stable_sort(v.begin(), v.end(), [](const Cand &a, const Cand &b) { return a.cost > b.cost; });
    const int64_t cnt = (int64_t)v.size();
    if (items_out) {
        if (cnt > max_items) return -1;
        for (int64_t q = 0; q < cnt; ++q)
            std::memcpy(items_out + nb::BATCH_ITEM_INTS * q, &v[q].it, sizeof(BatchItem));
    }
    return cnt;
}

const char *nb_last_error(const nb_ctx *ctx)
{
    return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

int nb_variant_count(int kind, nb_precision p)
{
    if (kind < 0 || kind >= nb::KIND_COUNT || p < NB_FP64 || p > NB_DF64) return 0;
    return variant_count(kind, p);
}

nb_status nb_variant_info(int kind, nb_precision p, int variant, int *T, int *I, int *J)
{
    if (variant < 0 || variant >= nb_variant_count(kind, p)) return NB_EINVAL;
    const KernelEntry &k = kernel_for(kind, p, variant, false);
    if (T) *T = k.T;
    if (I) *I = k.I;
    if (J) *J = k.J;
    return NB_OK;
}

nb_status nb_create(nb_ctx **out, int64_t n_max, nb_precision p, int device, void *stream)
{
    if (!out) return failf(nullptr, NB_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_max < 0 || n_max > (int64_t)0x7fffffff / 4)
        return failf(nullptr, NB_EINVAL, "n_max = %lld out of range", (long long)n_max);
    if (p < NB_FP64 || p > NB_DF64) return failf(nullptr, NB_EINVAL, "bad precision %d", (int)p);
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return failf(nullptr, NB_ECUDA, "cudaGetDeviceCount failed: %s", cudaGetErrorString(e));
    }
    if (device < 0 || device >= count)
        return failf(nullptr, NB_EINVAL, "device %d not in [0, %d)", device, count);
    DeviceGuard guard(device);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != device)
        return failf(nullptr, NB_ECUDA, "cannot make device %d current", device);

    nb_ctx *c = new nb_ctx();
    c->device = device;
    c->prec = p;
    c->n_max = n_max;
    c->stream = (cudaStream_t)stream;
    nb_status st = NB_OK;
    auto bail = [&](nb_status s) {
        g_create_error = c->last_error;
        free_ctx(c);
        return s;
    };
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return bail(failf(c, NB_ECUDA, "cannot read the SM count"));
    const int64_t ncap = std::max<int64_t>(n_max, 1);
    c->pack_bytes = (size_t)ncap * 64;
    c->pack = dev_alloc<char>(c, c->pack_bytes, st);
    c->partial_bodies = std::max<int64_t>(4 * ncap, (int64_t)1 << 22);
    if (st == NB_OK) c->partial = dev_alloc<double>(c, (size_t)c->partial_bodies * 4, st);
    c->n_counters = ncap / min_tile_bodies() + 2;
    if (st == NB_OK) c->counters = dev_alloc<unsigned>(c, (size_t)c->n_counters, st);
    c->n_red = c->partial_bodies / 64 + 4096;
    if (st == NB_OK) c->red = dev_alloc<double>(c, (size_t)c->n_red * 8, st);
    if (st == NB_OK) c->dev_out = dev_alloc<double>(c, 16, st);
    if (st == NB_OK) c->err = dev_alloc<int>(c, 4, st);
    if (st == NB_OK) c->queue = dev_alloc<unsigned>(c, 4, st);
    if (p != NB_FP64) {  // Morton-order scratch for the float32 kernels
        const size_t nc = (size_t)ncap;
        if (st == NB_OK) c->perm = dev_alloc<int>(c, nc, st);
        if (st == NB_OK) c->order.box = dev_alloc<double>(c, 1024 * 6, st);
        for (int q = 0; q < 2 && st == NB_OK; ++q) {
            c->order.keys[q] = dev_alloc<unsigned>(c, nc, st);
            if (st == NB_OK) c->order.vals[q] = dev_alloc<int>(c, nc, st);
        }
        if (st == NB_OK)
            c->order.hist = dev_alloc<unsigned>(c, nb::sort_hist_entries((int)ncap), st);
    }
    if (st != NB_OK) return bail(st);
    if (cudaMallocHost(&c->host_out, 16 * sizeof(double)) != cudaSuccess)
        return bail(failf(c, NB_ENOMEM, "cudaMallocHost failed"));
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return bail(failf(c, NB_ECUDA, "stream/event creation failed"));
    if (cudaMemset(c->counters, 0, (size_t)c->n_counters * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(c->err, 0, 4 * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->queue, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
        return bail(failf(c, NB_ECUDA, "scratch initialisation failed"));
    *out = c;
    return NB_OK;
}

nb_status nb_destroy(nb_ctx *c)
{
    if (!c) return NB_OK;
    DeviceGuard guard(c->device);
    cudaStreamSynchronize(c->stream);
    cudaStreamSynchronize(c->cap_stream);
    free_ctx(c);
    return NB_OK;
}

nb_status nb_set_stream(nb_ctx *c, void *stream)
{
    if (!c) return NB_EINVAL;
    c->stream = (cudaStream_t)stream;
    return NB_OK;
}

nb_status nb_sync(nb_ctx *c)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    int h = 0;
    NB_CUDA(c, cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h) {
        NB_CUDA(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
        NB_CUDA(c, cudaStreamSynchronize(c->stream));
        if (h & nb::ERR_TREE)
            return failf(c, NB_ENOMEM, "a tree outgrew its node arrays (it stopped a level early)");
        return failf(c, NB_ENONFINITE, "a kernel produced a non-finite result");
    }
    return NB_OK;
}

nb_status nb_forces(nb_ctx *c, int64_t n, const double *pos, const double *mass, double G,
                    double eps, double *acc)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    NB_TRY(check_scalars(c, G, eps));
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, acc, v3, "acc"));
    if (n == 0) return NB_OK;
    NB_TRY(pack(c, c->stream, n, pos, mass));
    return force_packed(c, c->stream, n, G, eps, acc, nullptr, 0.0);
}

nb_status nb_rollout(nb_ctx *c, int64_t n, double *pos, double *vel, const double *mass, double G,
                     double eps, double dt, int64_t nsteps, double *acc, unsigned flags,
                     int64_t every, double *rec_pos, double *rec_vel)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    NB_TRY(check_scalars(c, G, eps));
    if (!std::isfinite(dt)) return failf(c, NB_EINVAL, "dt is not finite");
    if (nsteps < 0) return failf(c, NB_EINVAL, "nsteps < 0");
    if (flags & ~(NB_ACC_VALID | NB_USE_GRAPH)) return failf(c, NB_EINVAL, "unknown flags");
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, vel, v3, "vel"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, acc, v3, "acc"));
    if (every > 0) {
        const size_t nrec = (size_t)(nsteps / every) + 1;
        NB_TRY(check_dev(c, rec_pos, v3 * nrec, "rec_pos"));
        if (rec_vel) NB_TRY(check_dev(c, rec_vel, v3 * nrec, "rec_vel"));
    } else {
        every = 0;
    }
    if (n == 0) return NB_OK;
    if (flags & NB_USE_GRAPH) {
        nb_ctx::GraphKey key{0,  pos,   vel, mass, acc,    rec_pos, rec_vel, G,
                             eps, dt,   n,   nsteps, every, flags,  0};
        return run_graph(c, key, [&](cudaStream_t s) {
            return rollout_enqueue(c, s, n, pos, vel, mass, G, eps, dt, nsteps, acc, flags, every,
                                   rec_pos, rec_vel);
        });
    }
    return rollout_enqueue(c, c->stream, n, pos, vel, mass, G, eps, dt, nsteps, acc, flags, every,
                           rec_pos, rec_vel);
}

nb_status nb_step(nb_ctx *c, int64_t n, double *pos, double *vel, const double *mass, double G,
                  double eps, double dt, int64_t nsteps, double *acc, unsigned flags)
{
    return nb_rollout(c, n, pos, vel, mass, G, eps, dt, nsteps, acc, flags, 0, nullptr, nullptr);
}

nb_status nb_energy(nb_ctx *c, int64_t n, const double *pos, const double *vel, const double *mass,
                    double G, double eps, double *out)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    NB_TRY(check_scalars(c, G, eps));
    if (!out) return failf(c, NB_EINVAL, "out_host is NULL");
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, vel, v3, "vel"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    if (n == 0) {
        for (int q = 0; q < 9; ++q) out[q] = 0.0;
        return NB_OK;
    }
    cudaStream_t s = c->stream;
    NB_LAUNCHED(c, nb::launch_pack_f64(s, (int)n, pos, mass, (double4 *)c->pack));
    const KernelEntry &k = nb::f64_energy_kernel(eps == 0.0);
    int S = splits_for(c, k, n, 0, 3);
    const int64_t tile = (int64_t)k.T * k.I;
    const int64_t n_itiles = (n + tile - 1) / tile;
    while (S > 1 && n_itiles * S > c->n_red) --S;
    if (n_itiles * S > c->n_red) return failf(c, NB_ENOMEM, "energy reduction scratch too small");
    nb::EnergyParams p;
    p.P = (const double4 *)c->pack;
    p.vel = vel;
    p.n = (int)n;
    p.nsplit = S;
    p.eps2 = eps * eps;
    p.red = c->red;
    p.err = c->err;
    NB_TRY(launch(c, k, n_itiles * S, &p, s, 3));
    NB_LAUNCHED(c, nb::launch_energy_final(s, c->red, (int)(n_itiles * S), G, c->dev_out));
    NB_CUDA(c, cudaMemcpyAsync(c->host_out, c->dev_out, 9 * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
    NB_CUDA(c, cudaStreamSynchronize(s));
    for (int q = 0; q < 9; ++q) out[q] = c->host_out[q];
    for (int q = 0; q < 9; ++q)
        if (!std::isfinite(out[q])) return failf(c, NB_ENONFINITE, "non-finite diagnostic");
    return nb_sync(c);
}

nb_status nb_forces_backward(nb_ctx *c, int64_t n, const double *pos, const double *mass, double G,
                             double eps, const double *grad_acc, double *grad_pos,
                             double *grad_mass)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    NB_TRY(check_scalars(c, G, eps));
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, grad_acc, v3, "grad_acc"));
    NB_TRY(check_dev(c, grad_pos, v3, "grad_pos"));
    NB_TRY(check_dev(c, grad_mass, v1, "grad_mass"));
    if (n == 0) return NB_OK;
    cudaStream_t s = c->stream;
    NB_LAUNCHED(c, nb::launch_pack_vjp(s, is_f64(c), (int)n, pos, mass, grad_acc, nullptr, nullptr,
                                       0.0, 1.0, c->pack, pack_stride(c)));
    return vjp_packed(c, s, n, G, eps, grad_pos, grad_mass, 0);
}

nb_status nb_step_backward(nb_ctx *c, int64_t n, const double *traj, const double *mass, double G,
                           double eps, double dt, int64_t nsteps, double *lam_x, double *lam_v,
                           double *lam_m, unsigned flags)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    NB_TRY(check_scalars(c, G, eps));
    if (!std::isfinite(dt)) return failf(c, NB_EINVAL, "dt is not finite");
    if (nsteps < 0) return failf(c, NB_EINVAL, "nsteps < 0");
    if (flags & ~(NB_BWD_AT_END | NB_BWD_AT_START)) return failf(c, NB_EINVAL, "unknown flags");
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, traj, v3 * (size_t)(nsteps + 1), "traj"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, lam_x, v3, "lam_x"));
    NB_TRY(check_dev(c, lam_v, v3, "lam_v"));
    NB_TRY(check_dev(c, lam_m, v1, "lam_m"));
    if (n == 0 || nsteps == 0) return NB_OK;  // no step: nothing to reverse
    cudaStream_t s = c->stream;
    const size_t per = (size_t)n * 3;
    const bool f64 = is_f64(c);
    if (flags & NB_BWD_AT_END) {
        // closing half-kick of the run's last step: VJP at x_K with dt/2 lam_v
        NB_LAUNCHED(c, nb::launch_pack_vjp(s, f64, (int)n, traj + per * (size_t)nsteps, mass,
                                           nullptr, lam_v, nullptr, 0.0, 0.5 * dt, c->pack,
                                           pack_stride(c)));
        NB_TRY(vjp_packed(c, s, n, G, eps, lam_x, lam_m, 1));
    }
    for (int64_t st = nsteps - 1; st >= 0; --st) {
        const double coef = (st == 0 && (flags & NB_BWD_AT_START)) ? 0.5 * dt : dt;
        NB_LAUNCHED(c, nb::launch_pack_vjp(s, f64, (int)n, traj + per * (size_t)st, mass, nullptr,
                                           lam_v, lam_x, dt, coef, c->pack, pack_stride(c)));
        NB_TRY(vjp_packed(c, s, n, G, eps, lam_x, lam_m, 1));
    }
    return NB_OK;
}

nb_status nb_batch_plan(nb_ctx *c, int64_t nsys, const int64_t *offsets)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    if (is_f64(c)) return failf(c, NB_EINVAL, "the batched kernel needs an FP32 context");
    if (nsys < 0 || !offsets) return failf(c, NB_EINVAL, "bad nsys/offsets");
    if (offsets[0] != 0) return failf(c, NB_EINVAL, "offsets[0] must be 0");
    for (int64_t k = 0; k < nsys; ++k)
        if (offsets[k + 1] < offsets[k]) return failf(c, NB_EINVAL, "offsets must be non-decreasing");
    if (offsets[nsys] > c->n_max) return failf(c, NB_EINVAL, "offsets[nsys] > n_max");
    int v, divisor;
    pick(c, nb::KIND_BATCHED, offsets[nsys], v, divisor);
    if (divisor <= 0) divisor = 4;
    const KernelEntry &k = nb::f32_batched_kernel(v, c->prec == NB_FP32_COMP, false);
    // When the batch has more work than one item per resident CTA, cap an
    // item at 1/divisor of an even share of the pairs per CTA (j-chunks of
    // big pieces) to shorten the tail; the tuning entry's split field holds
    // the divisor (0 = 4).  A plan whose chunks would not fit the context's
    // partial-sum scratch or counters is redone with a doubled cap.
    double pairs = 0.0;
    for (int64_t q = 0; q < nsys; ++q)
        pairs += (double)(offsets[q + 1] - offsets[q]) * (double)(offsets[q + 1] - offsets[q]);
    const int64_t slots = (int64_t)c->num_sms * occupancy(c, k);
    const int64_t TI = (int64_t)k.T * k.I;
    int64_t cap = 0;
    if (nb_plan_batch_host(nsys, offsets, k.T, k.I, k.J, 0, nullptr, 0) >= slots)
        cap = (int64_t)(pairs / ((double)divisor * (double)std::max<int64_t>(slots, 1))) + 1;
    std::vector<int32_t> host;
    int64_t cnt = 0;
    for (int attempt = 0;; ++attempt) {
        cnt = nb_plan_batch_host(nsys, offsets, k.T, k.I, k.J, cap, nullptr, 0);
        if (cnt < 0) return failf(c, NB_EINVAL, "cannot plan these offsets");
        host.assign((size_t)std::max<int64_t>(cnt, 1) * nb::BATCH_ITEM_INTS, 0);
        nb_plan_batch_host(nsys, offsets, k.T, k.I, k.J, cap, host.data(), cnt);
        int64_t ctrs = 0, pslots = 0;
        for (int64_t q = 0; q < cnt; ++q) {
            const BatchItem *it = reinterpret_cast<const BatchItem *>(host.data()) + q;
            if (it->nchunks > 1) {
                ctrs = std::max<int64_t>(ctrs, it->ctr + 1);
                pslots = std::max<int64_t>(pslots, (int64_t)it->pbase + it->nchunks);
            }
        }
        if (cap == 0 || (ctrs <= c->n_counters && pslots * TI * 3 <= c->partial_bodies * 4)) break;
        cap = attempt < 8 ? cap * 2 : 0;
    }
    if (cnt > c->items_cap) {
        cudaFree(c->items);
        c->items = nullptr;
        c->items_cap = 0;
        nb_status st = NB_OK;
        c->items = dev_alloc<BatchItem>(c, (size_t)cnt, st);
        if (st != NB_OK) return st;
        c->items_cap = cnt;
    }
    if (cnt > 0)
        NB_CUDA(c, cudaMemcpyAsync(c->items, host.data(), (size_t)cnt * sizeof(BatchItem),
                                   cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaMemsetAsync(c->queue, 0, 4 * sizeof(unsigned), c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    c->n_items = cnt;
    c->batch_variant = v;
    c->batch_n = offsets[nsys];
    c->batch_nsys = nsys;
    c->plan_gen++;
    drop_graphs(c);
    return NB_OK;
}

nb_status nb_forces_batched(nb_ctx *c, const double *pos, const double *mass, double G, double eps,
                            double *acc)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    if (is_f64(c)) return failf(c, NB_EINVAL, "the batched kernel needs an FP32 context");
    NB_TRY(check_scalars(c, G, eps));
    const int64_t n = c->batch_n;
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, acc, v3, "acc"));
    if (n == 0) return NB_OK;
    NB_TRY(pack(c, c->stream, n, pos, mass, false));
    return batched_force(c, c->stream, G, eps, acc, nullptr, 0.0);
}

nb_status nb_step_batched(nb_ctx *c, double *pos, double *vel, const double *mass, double G,
                          double eps, double dt, int64_t nsteps, double *acc, unsigned flags)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    if (is_f64(c)) return failf(c, NB_EINVAL, "the batched kernel needs an FP32 context");
    NB_TRY(check_scalars(c, G, eps));
    if (!std::isfinite(dt)) return failf(c, NB_EINVAL, "dt is not finite");
    if (nsteps < 0) return failf(c, NB_EINVAL, "nsteps < 0");
    if (flags & ~(NB_ACC_VALID | NB_USE_GRAPH)) return failf(c, NB_EINVAL, "unknown flags");
    const int64_t n = c->batch_n;
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, vel, v3, "vel"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, acc, v3, "acc"));
    if (n == 0) return NB_OK;
    if (flags & NB_USE_GRAPH) {
        nb_ctx::GraphKey key{1,   pos, vel,           mass, acc,   nullptr,     nullptr, G,
                             eps, dt,  c->batch_n,    nsteps, 0,   flags,       c->plan_gen};
        return run_graph(c, key, [&](cudaStream_t s) {
            return batched_enqueue(c, s, pos, vel, mass, G, eps, dt, nsteps, acc, flags);
        });
    }
    return batched_enqueue(c, c->stream, pos, vel, mass, G, eps, dt, nsteps, acc, flags);
}

nb_status nb_tune_set(nb_ctx *c, int kind, int64_t lo, int64_t hi, int variant, int split)
{
    if (!c) return NB_EINVAL;
    if (kind < 0 || kind >= nb::KIND_COUNT) return failf(c, NB_EINVAL, "bad kind %d", kind);
    if (variant < 0) {
        c->tune[kind].clear();
        drop_graphs(c);
        return NB_OK;
    }
    if (variant >= variant_count(kind, c->prec))
        return failf(c, NB_EINVAL, "variant %d out of range for kind %d", variant, kind);
    if (lo < 0 || hi <= lo || split < 0) return failf(c, NB_EINVAL, "bad range or split");
    c->tune[kind].push_back({lo, hi, variant, split});
    drop_graphs(c);
    return NB_OK;
}

nb_status nb_tune_get(nb_ctx *c, int kind, int64_t n, int *variant, int *split)
{
    if (!c || kind < 0 || kind >= nb::KIND_COUNT) return NB_EINVAL;
    int v, s;
    pick(c, kind, n, v, s);
    if (variant) *variant = v;
    if (split) *split = s;
    return NB_OK;
}

int64_t nb_launch_count(const nb_ctx *c) { return c ? c->launches : 0; }

nb_status nb_set_order(nb_ctx *c, int mode, int64_t min_n)
{
    if (!c) return NB_EINVAL;
    if (mode < 0 || mode > 2 || min_n < 0) return failf(c, NB_EINVAL, "bad order mode");
    c->order_mode = mode;
    c->order_min_n = min_n;
    drop_graphs(c);
    return NB_OK;
}

nb_status nb_profile(nb_ctx *c, int enable)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    if (enable) {
        NB_CUDA(c, cudaStreamSynchronize(c->stream));
        for (auto &r : c->prof) {
            c->ev_pool.push_back(r.a);
            c->ev_pool.push_back(r.b);
        }
        c->prof.clear();
    }
    c->prof_on = enable != 0;
    return NB_OK;
}

nb_status nb_profile_read(nb_ctx *c, int kind, int64_t *launches, double *total_ms)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    int64_t cnt = 0;
    double ms = 0.0;
    for (const auto &r : c->prof) {
        if (r.kind != kind) continue;
        float t = 0.f;
        NB_CUDA(c, cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        ++cnt;
    }
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = ms;
    return NB_OK;
}

nb_status nb_tree_forces(nb_ctx *c, int64_t n, const double *pos, const double *mass, double G,
                         double eps, double theta, int leaf_cap, int group, double *acc,
                         int32_t *counts)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    NB_TRY(check_scalars(c, G, eps));
    NB_TRY(check_tree_args(c, theta, leaf_cap, group));
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, acc, v3, "acc"));
    if (counts) NB_TRY(check_dev(c, counts, (size_t)n * 2 * sizeof(int32_t), "counts"));
    if (n == 0) return NB_OK;
    NB_TRY(ensure_tree(c, leaf_cap));
    return tree_forces_enqueue(c, c->stream, n, pos, mass, G, eps, theta, leaf_cap, group, acc,
                               nullptr, 0.0, counts);
}

nb_status nb_tree_step(nb_ctx *c, int64_t n, double *pos, double *vel, const double *mass,
                       double G, double eps, double theta, int leaf_cap, int group, double dt,
                       int64_t nsteps, double *acc, unsigned flags)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    NB_TRY(check_scalars(c, G, eps));
    NB_TRY(check_tree_args(c, theta, leaf_cap, group));
    if (!std::isfinite(dt)) return failf(c, NB_EINVAL, "dt is not finite");
    if (nsteps < 0) return failf(c, NB_EINVAL, "nsteps < 0");
    if (flags & ~(NB_ACC_VALID | NB_USE_GRAPH)) return failf(c, NB_EINVAL, "unknown flags");
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, vel, v3, "vel"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, acc, v3, "acc"));
    if (n == 0) return NB_OK;
    NB_TRY(ensure_tree(c, leaf_cap));
    if (flags & NB_USE_GRAPH) {
        nb_ctx::GraphKey key{2,   pos, vel, mass,   acc, nullptr, nullptr, G,
                             eps, dt,  n,   nsteps, 0,   flags,   0};
        key.theta = theta;
        key.leaf_cap = leaf_cap * 128 + group;
        return run_graph(c, key, [&](cudaStream_t s) {
            return tree_step_enqueue(c, s, n, pos, vel, mass, G, eps, theta, leaf_cap, group, dt,
                                     nsteps, acc, flags);
        });
    }
    return tree_step_enqueue(c, c->stream, n, pos, vel, mass, G, eps, theta, leaf_cap, group, dt,
                             nsteps, acc, flags);
}

nb_status nb_tree_schedule(nb_ctx *c, int sched, int chunk)
{
    if (!c) return NB_EINVAL;
    if (sched < 0 || sched > 2) return failf(c, NB_EINVAL, "schedule %d is not 0, 1 or 2", sched);
    if (chunk < 1 || chunk > (1 << 20)) return failf(c, NB_EINVAL, "chunk %d out of range", chunk);
    c->tree_sched = sched;
    c->tree_chunk = chunk;
    drop_graphs(c);  // captured walks hold the old schedule
    return NB_OK;
}

nb_status nb_fmm_forces(nb_ctx *c, int64_t n, const double *pos, const double *mass, double G,
                        double eps, double theta, int order, int leaf_cap, double *acc,
                        int32_t *counts)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    NB_TRY(check_scalars(c, G, eps));
    NB_TRY(check_fmm_args(c, theta, order, leaf_cap));
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, acc, v3, "acc"));
    if (counts) NB_TRY(check_dev(c, counts, (size_t)n * 3 * sizeof(int32_t), "counts"));
    if (n == 0) return NB_OK;
    NB_TRY(ensure_tree(c, leaf_cap));
    NB_TRY(ensure_fmm(c, order, c->fmm.pool ? 1 : (long long)(1 << 20) + 32LL * c->n_max,
                      c->fmm.chunk_src ? 1 : 4096LL + 2LL * c->n_max,
                      c->fmm.rchunk ? 1 : 4096LL + c->n_max / 4));
    return fmm_forces_run(c, n, pos, mass, G, eps, theta, order, leaf_cap, acc, counts);
}

nb_status nb_fmm_step(nb_ctx *c, int64_t n, double *pos, double *vel, const double *mass,
                      double G, double eps, double theta, int order, int leaf_cap, double dt,
                      int64_t nsteps, double *acc, unsigned flags)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    NB_TRY(check_scalars(c, G, eps));
    NB_TRY(check_fmm_args(c, theta, order, leaf_cap));
    if (!std::isfinite(dt)) return failf(c, NB_EINVAL, "dt is not finite");
    if (nsteps < 0) return failf(c, NB_EINVAL, "nsteps < 0");
    if (flags & ~NB_ACC_VALID)
        return failf(c, NB_EINVAL, "unknown flags (the FMM synchronises: no graph)");
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, vel, v3, "vel"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, acc, v3, "acc"));
    if (n == 0) return NB_OK;
    NB_TRY(ensure_tree(c, leaf_cap));
    NB_TRY(ensure_fmm(c, order, c->fmm.pool ? 1 : (long long)(1 << 20) + 32LL * c->n_max,
                      c->fmm.chunk_src ? 1 : 4096LL + 2LL * c->n_max,
                      c->fmm.rchunk ? 1 : 4096LL + c->n_max / 4));
    if (!(flags & NB_ACC_VALID))
        NB_TRY(fmm_forces_run(c, n, pos, mass, G, eps, theta, order, leaf_cap, acc, nullptr));
    for (int64_t st = 0; st < nsteps; ++st) {
        NB_LAUNCHED(c, nb::launch_kdp(c->stream, is_f64(c), (int)n, pos, vel, acc, mass, 0.5 * dt,
                                      dt, nullptr, nullptr, nullptr, nullptr));
        NB_TRY(fmm_forces_run(c, n, pos, mass, G, eps, theta, order, leaf_cap, acc, nullptr, vel,
                              0.5 * dt));
    }
    return NB_OK;
}

nb_status nb_fmm_reserve(nb_ctx *c, int64_t entries)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    if (entries < 1 || entries > 0x7fffffffLL)
        return failf(c, NB_EINVAL, "pool of %lld entries outside [1, 2^31)", (long long)entries);
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    nb::FmmView &f = c->fmm;
    void *old[] = {f.pool, f.chunk_src, f.chunk_next, f.rchunk, f.rnext};
    for (void *a : old) cudaFree(a);
    f.pool = f.chunk_src = f.chunk_next = f.rnext = nullptr;
    f.rchunk = nullptr;
    f.pool_cap = f.chunk_cap = f.rchunk_cap = 0;
    nb_status st = NB_OK;
    f.pool = dev_alloc<int>(c, (size_t)entries, st);
    if (st != NB_OK) return st;
    f.pool_cap = entries;
    const long long chunks = entries / nb::FMM_CHUNK + 1;
    NB_TRY(ensure_chunks(c, chunks, f.chunk_src, f.chunk_next, f.chunk_cap, "expansion lists"));
    return ensure_chunks(c, chunks, f.rchunk, f.rnext, f.rchunk_cap, "direct-range lists");
}

nb_status nb_fmm_stats(nb_ctx *c, int64_t *out)
{
    if (!c || !out) return failf(c, NB_EINVAL, "ctx or out is NULL");
    DeviceGuard guard(c->device);
    unsigned long long h[4] = {0, 0, 0, 0};
    if (c->fmm.stats)
        NB_CUDA(c, cudaMemcpyAsync(h, c->fmm.stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < 4; ++q) out[q] = (int64_t)h[q];
    return NB_OK;
}

nb_status nb_tree_stats(nb_ctx *c, int64_t *out)
{
    if (!c || !out) return failf(c, NB_EINVAL, "ctx or out is NULL");
    DeviceGuard guard(c->device);
    unsigned long long h[4] = {0, 0, 0, 0};
    if (c->tree.stats)
        NB_CUDA(c, cudaMemcpyAsync(h, c->tree.stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < 4; ++q) out[q] = (int64_t)h[q];
    return NB_OK;
}

nb_status nb_device_info(nb_ctx *c, int64_t n, int *num_sms, int *ctas_per_sm)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    int v, s;
    pick(c, nb::KIND_FORCE, n, v, s);
    if (num_sms) *num_sms = c->num_sms;
    if (ctas_per_sm) *ctas_per_sm = occupancy(c, kernel_for(nb::KIND_FORCE, c->prec, v, false));
    return NB_OK;
}

// ----------------------------------------------- ORB and locally essential trees
namespace {

nb_status ensure_orb(nb_ctx *c)
{
    nb_status st = NB_OK;
    NB_TRY(ensure_order(c));
    if (!c->orb_buf)
        c->orb_buf = dev_alloc<unsigned long long>(
            c, (size_t)nb::ORB_MAX_P * 6 + (size_t)nb::ORB_MAX_P / 2 * 256 + nb::ORB_MAX_P, st);
    if (st == NB_OK && !c->orb_perm)
        c->orb_perm = dev_alloc<int>(c, (size_t)std::max<int64_t>(c->n_max, 1), st);
    return st;
}

nb_status check_orb_tables(nb_ctx *c, int nactive, const int32_t *active, const int32_t *axis,
                           const uint64_t *key, const int32_t *upper, nb::OrbTables &t)
{
    if (nactive < 0 || nactive > nb::ORB_MAX_P / 2)
        return failf(c, NB_EINVAL, "nactive = %d outside [0, %d]", nactive, nb::ORB_MAX_P / 2);
    if (nactive > 0 && (!active || !axis || !key))
        return failf(c, NB_EINVAL, "active, axis or key table is NULL");
    for (int g = 0; g < nb::ORB_MAX_P; ++g) t.slot[g] = -1;
    for (int r = 0; r < nactive; ++r) {
        if (active[r] < 0 || active[r] >= nb::ORB_MAX_P || t.slot[active[r]] >= 0)
            return failf(c, NB_EINVAL, "active[%d] = %d is not a distinct group below %d", r,
                         active[r], nb::ORB_MAX_P);
        if (axis[r] < 0 || axis[r] > 2) return failf(c, NB_EINVAL, "axis[%d] = %d", r, axis[r]);
        if (upper && (upper[r] <= active[r] || upper[r] >= nb::ORB_MAX_P))
            return failf(c, NB_EINVAL, "upper[%d] = %d must lie above %d", r, upper[r], active[r]);
        t.slot[active[r]] = r;
        t.axis[r] = axis[r];
        t.upper[r] = upper ? upper[r] : 0;
        t.key_hi[r] = key[2 * r];
        t.key_lo[r] = (unsigned)key[2 * r + 1];
    }
    return NB_OK;
}

// Scratch of the LET selection for the tree's node capacity.
nb_status ensure_let(nb_ctx *c)
{
    nb_status st = NB_OK;
    if (!c->let_box) c->let_box = dev_alloc<float>(c, 12, st);
    if (st == NB_OK && !c->let_queue) c->let_queue = dev_alloc<int>(c, 1, st);
    if (st == NB_OK && !c->let_src)
        c->let_src = dev_alloc<nb::WalkSource>(c, 1 + nb::WALK_MAX_MORE, st);
    if (st == NB_OK && !c->let.totals) c->let.totals = dev_alloc<int>(c, 2, st);
    if (st != NB_OK) return st;
    if (c->let_cap < c->tree.cap) {
        cudaFree(c->let.kind);
        cudaFree(c->let.nidx);
        cudaFree(c->let.boff);
        c->let.kind = c->let.nidx = c->let.boff = nullptr;
        c->let_cap = 0;
        const size_t m = (size_t)c->tree.cap;
        c->let.kind = dev_alloc<int>(c, m, st);
        if (st == NB_OK) c->let.nidx = dev_alloc<int>(c, m, st);
        if (st == NB_OK) c->let.boff = dev_alloc<int>(c, m, st);
        if (st != NB_OK) return st;
        c->let_cap = c->tree.cap;
    }
    return NB_OK;
}

// Scratch of the split LET walk for ntrees trees over `groups` groups of
// `group` bodies (grown, never shrunk; the arrival counters are zeroed on
// stream s when allocated and every launch leaves them at zero).
nb_status ensure_let_split(nb_ctx *c, cudaStream_t s, int ntrees, int64_t groups, int group)
{
    nb_status st = NB_OK;
    const int64_t part = (int64_t)ntrees * groups * group * 3, cnt = (int64_t)ntrees * groups * 2;
    if (c->let_tpart_cap < part) {
        cudaFree(c->let_tpart);
        c->let_tpart = dev_alloc<double>(c, (size_t)part, st);
        c->let_tpart_cap = st == NB_OK ? part : 0;
        if (st != NB_OK) return st;
    }
    if (c->let_tcnt_cap < cnt) {
        cudaFree(c->let_tcnt);
        c->let_tcnt = dev_alloc<int>(c, (size_t)cnt, st);
        c->let_tcnt_cap = st == NB_OK ? cnt : 0;
        if (st != NB_OK) return st;
    }
    if (c->let_tctr_cap < groups) {
        cudaFree(c->let_tctr);
        c->let_tctr = dev_alloc<unsigned>(c, (size_t)groups, st);
        c->let_tctr_cap = 0;
        if (st != NB_OK) return st;
        NB_CUDA(c, cudaMemsetAsync(c->let_tctr, 0, (size_t)groups * sizeof(unsigned), s));
        c->let_tctr_cap = groups;
    }
    return NB_OK;
}

// One walk launch over tree view t with sources (sP, sPlo) and box, then
// the nmore trees at more (device), onto the context's local bodies; with
// received trees, one task per (group, tree).
nb_status let_walk(nb_ctx *c, cudaStream_t s, const nb::TreeView &t, const float4 *sP,
                   const float4 *sPlo, const double *box, const nb::WalkSource *more,
                   int nmore, double G, double eps, double theta, int group, double *acc,
                   int *counts, int accumulate)
{
    NB_CUDA(c, cudaMemsetAsync(c->let_queue, 0, sizeof(int), s));
    nb::TreeWalkParams p;
    p.tree = t;
    p.P = c->tree_P;
    p.Plo = c->tree_Plo;
    p.perm = c->tree_perm;
    p.sP = sP;
    p.sPlo = sPlo;
    p.box = box;
    p.queue = c->let_queue;
    p.n = (int)c->let_n;
    p.group = group;
    p.sched = c->tree_sched;
    p.chunk = c->tree_chunk;
    p.num_sms = c->num_sms;
    p.accumulate = accumulate;
    p.theta = (float)theta;
    p.eps2f = (float)(eps * eps);
    p.G = G;
    p.acc = acc;
    p.vel = nullptr;
    p.half_dt = 0.0;
    p.counts = counts;
    p.err = c->err;
    p.more = more;
    p.nmore = nmore;
    p.tspan = 1;
    p.tpart = nullptr;
    p.tcnt = nullptr;
    p.tctr = nullptr;
    if (nmore > 0 && p.n > 0) {
        const int64_t groups = (p.n + group - 1) / group;
        NB_TRY(ensure_let_split(c, s, 1 + nmore, groups, group));
        p.tpart = c->let_tpart;
        p.tcnt = c->let_tcnt;
        p.tctr = c->let_tctr;
    }
    int k = 0;
    TreeTimer tm(c, nb::PROF_TREE_WALK, s);
    NB_CUDA(c, nb::launch_tree_walk(s, p, p.eps2f == 0.0f, k));
    c->launches += k;
    tm.done();
    return NB_OK;
}

}  // namespace

nb_status nb_orb_box(nb_ctx *c, int64_t n, const double *pos, const int32_t *group, int ngroups,
                     double *box_out)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    if (ngroups < 1 || ngroups > nb::ORB_MAX_P)
        return failf(c, NB_EINVAL, "ngroups = %d outside [1, %d]", ngroups, nb::ORB_MAX_P);
    if (!box_out) return failf(c, NB_EINVAL, "box_out is NULL");
    NB_TRY(check_dev(c, pos, (size_t)n * 3 * sizeof(double), "pos"));
    NB_TRY(check_dev(c, group, (size_t)n * sizeof(int32_t), "group"));
    NB_TRY(ensure_orb(c));
    cudaStream_t s = c->stream;
    NB_LAUNCHED(c, nb::launch_orb_box(s, (int)n, pos, group, ngroups, c->orb_buf));
    std::vector<unsigned long long> h((size_t)ngroups * 6);
    NB_CUDA(c, cudaMemcpyAsync(h.data(), c->orb_buf, h.size() * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
    NB_CUDA(c, cudaStreamSynchronize(s));
    for (size_t q = 0; q < h.size(); ++q) {
        const unsigned long long k = h[q];
        const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
        double v;
        std::memcpy(&v, &b, sizeof v);
        const bool empty = (q % 6 < 3) ? k == ~0ull : k == 0ull;
        box_out[q] = empty ? ((q % 6 < 3) ? INFINITY : -INFINITY) : v;
    }
    return NB_OK;
}

nb_status nb_orb_hist(nb_ctx *c, int64_t n, const double *pos, const int64_t *id,
                      const int32_t *group, int nactive, const int32_t *active, const int32_t *axis,
                      const uint64_t *prefix, int round, int64_t *hist_out)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    if (round < 0 || round > 11) return failf(c, NB_EINVAL, "round = %d outside [0, 11]", round);
    if (!hist_out && nactive > 0) return failf(c, NB_EINVAL, "hist_out is NULL");
    nb::OrbTables t;
    NB_TRY(check_orb_tables(c, nactive, active, axis, prefix, nullptr, t));
    NB_TRY(check_dev(c, pos, (size_t)n * 3 * sizeof(double), "pos"));
    NB_TRY(check_dev(c, id, (size_t)n * sizeof(int64_t), "id"));
    NB_TRY(check_dev(c, group, (size_t)n * sizeof(int32_t), "group"));
    NB_TRY(ensure_orb(c));
    if (nactive == 0) return NB_OK;
    cudaStream_t s = c->stream;
    unsigned long long *hist = c->orb_buf + (size_t)nb::ORB_MAX_P * 6;
    NB_LAUNCHED(c, nb::launch_orb_hist(s, (int)n, pos, (const long long *)id, group, nactive, t,
                                       round, hist));
    NB_CUDA(c, cudaMemcpyAsync(hist_out, hist, (size_t)nactive * 256 * sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
    NB_CUDA(c, cudaStreamSynchronize(s));
    return NB_OK;
}

nb_status nb_orb_cut(nb_ctx *c, int64_t n, const double *pos, const int64_t *id, int32_t *group,
                     int nactive, const int32_t *active, const int32_t *axis,
                     const uint64_t *split, const int32_t *upper)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    if (nactive > 0 && !upper) return failf(c, NB_EINVAL, "upper is NULL");
    nb::OrbTables t;
    NB_TRY(check_orb_tables(c, nactive, active, axis, split, upper, t));
    NB_TRY(check_dev(c, pos, (size_t)n * 3 * sizeof(double), "pos"));
    NB_TRY(check_dev(c, id, (size_t)n * sizeof(int64_t), "id"));
    NB_TRY(check_dev(c, group, (size_t)n * sizeof(int32_t), "group"));
    if (nactive == 0 || n == 0) return NB_OK;
    NB_LAUNCHED(c, nb::launch_orb_cut(c->stream, (int)n, pos, (const long long *)id, group, t));
    return NB_OK;
}

nb_status nb_orb_pack(nb_ctx *c, int64_t n, const int32_t *rank, int P, const double *pos,
                      const double *vel, const double *mass, const int64_t *id, double *pos_out,
                      double *vel_out, double *mass_out, int64_t *id_out, int64_t *counts_out)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    if (P < 1 || P > nb::ORB_MAX_P) return failf(c, NB_EINVAL, "P = %d outside [1, %d]", P, nb::ORB_MAX_P);
    if (!counts_out) return failf(c, NB_EINVAL, "counts_out is NULL");
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, rank, (size_t)n * sizeof(int32_t), "rank"));
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, vel, v3, "vel"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, id, (size_t)n * sizeof(int64_t), "id"));
    NB_TRY(check_dev(c, pos_out, v3, "pos_out"));
    NB_TRY(check_dev(c, vel_out, v3, "vel_out"));
    NB_TRY(check_dev(c, mass_out, v1, "mass_out"));
    NB_TRY(check_dev(c, id_out, (size_t)n * sizeof(int64_t), "id_out"));
    NB_TRY(ensure_orb(c));
    cudaStream_t s = c->stream;
    unsigned long long *cnt = c->orb_buf + (size_t)nb::ORB_MAX_P * 6 + (size_t)nb::ORB_MAX_P / 2 * 256;
    NB_LAUNCHED(c, nb::launch_rank_counts(s, (int)n, rank, P, cnt));
    if (n > 0) {
        int k = 0;
        NB_CUDA(c, nb::launch_key_sort(s, (int)n, rank, nullptr, 1, c->order, c->orb_perm, k));
        c->launches += k;
        NB_LAUNCHED(c, nb::launch_gather_bodies(s, (int)n, c->orb_perm, pos, vel, mass,
                                                (const long long *)id, pos_out, vel_out, mass_out,
                                                (long long *)id_out));
    }
    NB_CUDA(c, cudaMemcpyAsync(counts_out, cnt, (size_t)P * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    NB_CUDA(c, cudaStreamSynchronize(s));
    int64_t tot = 0;
    for (int r = 0; r < P; ++r) tot += counts_out[r];
    if (tot != n) return failf(c, NB_EINVAL, "rank values outside [0, %d)", P);
    return NB_OK;
}

nb_status nb_orb_order(nb_ctx *c, int64_t n, const double *pos, const double *vel,
                       const double *mass, const int64_t *id, double *pos_out, double *vel_out,
                       double *mass_out, int64_t *id_out)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    const size_t v3 = (size_t)n * 3 * sizeof(double), v1 = (size_t)n * sizeof(double);
    NB_TRY(check_dev(c, pos, v3, "pos"));
    NB_TRY(check_dev(c, vel, v3, "vel"));
    NB_TRY(check_dev(c, mass, v1, "mass"));
    NB_TRY(check_dev(c, id, (size_t)n * sizeof(int64_t), "id"));
    NB_TRY(check_dev(c, pos_out, v3, "pos_out"));
    NB_TRY(check_dev(c, vel_out, v3, "vel_out"));
    NB_TRY(check_dev(c, mass_out, v1, "mass_out"));
    NB_TRY(check_dev(c, id_out, (size_t)n * sizeof(int64_t), "id_out"));
    if (n == 0) return NB_OK;
    NB_TRY(ensure_orb(c));
    cudaStream_t s = c->stream;
    int k = 0;
    NB_CUDA(c, nb::launch_key_sort(s, (int)n, nullptr, (const long long *)id, 4, c->order,
                                   c->orb_perm, k));
    c->launches += k;
    NB_LAUNCHED(c, nb::launch_gather_bodies(s, (int)n, c->orb_perm, pos, vel, mass,
                                            (const long long *)id, pos_out, vel_out, mass_out,
                                            (long long *)id_out));
    return NB_OK;
}

nb_status nb_let_build(nb_ctx *c, int64_t n, const double *pos, const double *mass, int leaf_cap,
                       float *box_out)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_n(c, n));
    if (leaf_cap < 1 || leaf_cap > NB_TREE_MAX_LEAF)
        return failf(c, NB_EINVAL, "leaf_cap = %d outside [1, %d]", leaf_cap, NB_TREE_MAX_LEAF);
    if (!box_out) return failf(c, NB_EINVAL, "box_out is NULL");
    NB_TRY(check_dev(c, pos, (size_t)n * 3 * sizeof(double), "pos"));
    NB_TRY(check_dev(c, mass, (size_t)n * sizeof(double), "mass"));
    c->let_n = 0;
    if (n == 0) {
        for (int q = 0; q < 6; ++q) box_out[q] = q < 3 ? INFINITY : -INFINITY;
        return NB_OK;
    }
    NB_TRY(ensure_tree(c, leaf_cap));
    NB_TRY(ensure_let(c));
    cudaStream_t s = c->stream;
    NB_TRY(tree_build_enqueue(c, s, n, pos, mass, leaf_cap));
    NB_LAUNCHED(c, nb::launch_hi_box(s, (int)n, c->tree_P, c->let_box));
    NB_CUDA(c, cudaMemcpyAsync(box_out, c->let_box, 6 * sizeof(float), cudaMemcpyDeviceToHost, s));
    NB_CUDA(c, cudaStreamSynchronize(s));
    c->let_n = n;
    return NB_OK;
}

nb_status nb_let_export(nb_ctx *c, double theta, const float *box, void *out, int64_t capacity,
                        int64_t *size_out)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    if (!box || !size_out) return failf(c, NB_EINVAL, "box or size_out is NULL");
    if (!std::isfinite(theta) || theta < 0)
        return failf(c, NB_EINVAL, "theta must be finite and >= 0");
    for (int q = 0; q < 6; ++q)
        if (std::isnan(box[q])) return failf(c, NB_EINVAL, "box[%d] is NaN", q);
    if (c->let_n == 0) return failf(c, NB_EINVAL, "no local tree: call nb_let_build first");
    NB_TRY(ensure_let(c));
    cudaStream_t s = c->stream;
    int k = 0;
    NB_CUDA(c, nb::launch_let_select(s, c->tree, c->tree_box, (float)theta,
                                     make_float3(box[0], box[1], box[2]),
                                     make_float3(box[3], box[4], box[5]), c->let, k));
    c->launches += k;
    int tot[2] = {0, 0};
    NB_CUDA(c, cudaMemcpyAsync(tot, c->let.totals, sizeof tot, cudaMemcpyDeviceToHost, s));
    NB_CUDA(c, cudaStreamSynchronize(s));
    const nb::LetLayout lay = nb::let_layout(tot[0], tot[1]);
    *size_out = (int64_t)lay.total;
    if (!out) return NB_OK;  // size query
    if (capacity < (int64_t)lay.total)
        return failf(c, NB_ENOMEM, "LET of %zu bytes exceeds the buffer's %lld", lay.total,
                     (long long)capacity);
    if ((uintptr_t)out % 16) return failf(c, NB_EINVAL, "out is not 16-byte aligned");
    NB_TRY(check_dev(c, out, lay.total, "out"));
    NB_CUDA(c, nb::launch_let_emit(s, c->tree, c->tree_box, c->let, c->tree_P, c->tree_Plo, out, k));
    c->launches += k;
    return NB_OK;
}

nb_status nb_let_forces(nb_ctx *c, double G, double eps, double theta, int group, int64_t nlet,
                        const void *const *lets, double *acc, int32_t *counts)
{
    if (!c) return NB_EINVAL;
    DeviceGuard guard(c->device);
    NB_TRY(check_scalars(c, G, eps));
    if (!std::isfinite(theta) || theta < 0)
        return failf(c, NB_EINVAL, "theta must be finite and >= 0");
    if (group != 32 && group != 64) return failf(c, NB_EINVAL, "group = %d is not 32 or 64", group);
    if (nlet < 0 || (nlet > 0 && !lets)) return failf(c, NB_EINVAL, "bad nlet or lets");
    const int64_t n = c->let_n;
    if (n == 0) return failf(c, NB_EINVAL, "no local tree: call nb_let_build first");
    NB_TRY(check_dev(c, acc, (size_t)n * 3 * sizeof(double), "acc"));
    if (counts) NB_TRY(check_dev(c, counts, (size_t)n * 2 * sizeof(int32_t), "counts"));
    // every received tree's header, checked before anything is launched
    std::vector<nb::LetHeader> hdr((size_t)nlet);
    cudaStream_t s = c->stream;
    for (int64_t q = 0; q < nlet; ++q) {
        if ((uintptr_t)lets[q] % 16) return failf(c, NB_EINVAL, "lets[%lld] is not 16-byte aligned", (long long)q);
        NB_TRY(check_dev(c, lets[q], sizeof(nb::LetHeader), "lets[q]"));
        NB_CUDA(c, cudaMemcpyAsync(&hdr[(size_t)q], lets[q], sizeof(nb::LetHeader),
                                   cudaMemcpyDeviceToHost, s));
    }
    NB_CUDA(c, cudaStreamSynchronize(s));
    for (int64_t q = 0; q < nlet; ++q) {
        const nb::LetHeader &h = hdr[(size_t)q];
        if (h.magic != nb::LET_MAGIC || h.n_nodes < 1 || h.n_bodies < 0 ||
            h.n_nodes > 0x7fffffffLL || h.n_bodies > 0x7fffffffLL)
            return failf(c, NB_EINVAL, "lets[%lld] does not hold a LET", (long long)q);
        NB_TRY(check_dev(c, lets[q], nb::let_layout(h.n_nodes, h.n_bodies).total, "lets[q]"));
    }
    NB_TRY(ensure_let(c));
    NB_CUDA(c, cudaMemsetAsync(c->tree.stats + 2, 0, 2 * sizeof(unsigned long long), s));
    // the local tree first, then the received ones in order: the local tree
    // and up to WALK_MAX_MORE received ones per launch
    std::vector<nb::WalkSource> src((size_t)nlet);
    for (int64_t q = 0; q < nlet; ++q) {
        const nb::LetHeader &h = hdr[(size_t)q];
        const nb::LetLayout lay = nb::let_layout(h.n_nodes, h.n_bodies);
        const unsigned char *b = static_cast<const unsigned char *>(lets[q]);
        src[(size_t)q] = nb::WalkSource{(const float4 *)(b + lay.lo),  (const float4 *)(b + lay.hi),
                                        (const float4 *)(b + lay.chi), (const float4 *)(b + lay.clo),
                                        (const int *)(b + lay.start),  (const int *)(b + lay.end),
                                        (const float4 *)(b + lay.P),   (const float4 *)(b + lay.Plo),
                                        (const double *)(b + offsetof(nb::LetHeader, box))};
    }
    // a multi-tree launch reads every tree it walks, the first included, from
    // let_src: the local tree, then the received ones
    src.insert(src.begin(), nb::WalkSource{c->tree.box_lo, c->tree.box_hi, c->tree.chi,
                                           c->tree.clo, c->tree.start, c->tree.end, c->tree_P,
                                           c->tree_Plo, c->tree_box});
    const int first = (int)std::min<int64_t>(nlet, nb::WALK_MAX_MORE);
    if (first > 0)  // from pageable memory: staged before the call returns
        NB_CUDA(c, cudaMemcpyAsync(c->let_src, src.data(), (1 + first) * sizeof(nb::WalkSource),
                                   cudaMemcpyHostToDevice, s));
    NB_TRY(let_walk(c, s, c->tree, c->tree_P, c->tree_Plo, c->tree_box, c->let_src, first, G, eps,
                    theta, group, acc, counts, 0));
    for (int64_t q0 = first; q0 < nlet; q0 += 1 + nb::WALK_MAX_MORE) {
        // a further launch: tree q0, then up to WALK_MAX_MORE more, added on
        const int more = (int)std::min<int64_t>(nlet - q0 - 1, nb::WALK_MAX_MORE);
        if (more > 0)  // (src[0] is the local tree: received tree q is src[1 + q])
            NB_CUDA(c, cudaMemcpyAsync(c->let_src, src.data() + 1 + q0,
                                       (1 + more) * sizeof(nb::WalkSource),
                                       cudaMemcpyHostToDevice, s));
        const nb::WalkSource &w = src[(size_t)(1 + q0)];
        nb::TreeView t{};
        t.cap = (int)hdr[(size_t)q0].n_nodes;
        t.box_lo = const_cast<float4 *>(w.box_lo);
        t.box_hi = const_cast<float4 *>(w.box_hi);
        t.chi = const_cast<float4 *>(w.chi);
        t.clo = const_cast<float4 *>(w.clo);
        t.start = const_cast<int *>(w.start);
        t.end = const_cast<int *>(w.end);
        t.stats = c->tree.stats;
        NB_TRY(let_walk(c, s, t, w.sP, w.sPlo, w.box, c->let_src, more, G, eps, theta, group, acc,
                        counts, 1));
    }
    return NB_OK;
}

}  // extern "C"
