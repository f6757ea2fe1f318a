// nb_forces_noalloc: the float32 Kahan-compensated force kernel for callers
// that must not allocate device memory.
//
// Who needs it: code whose device memory is owned by someone else -- a
// framework's memory pool that must see every byte, a sandbox or service
// with a fixed device-memory budget -- and latency-critical loops in which a
// cudaMalloc could block or synchronise the device.  nb_create cannot serve
// them, because creating a context allocates its scratch.
//
// How: the scratch the kernel needs (packed hi/lo bodies, j-split partial
// sums, arrival counters, an error word) lives in one file-scope
// __device__ array of fixed size, which every GPU that loads the library
// holds until the process exits.  Host code cannot use the array's name as a
// device address.  The first call made in a CUDA context (with that context
// current) asks the runtime for the array's device address with
// cudaGetSymbolAddress and keeps it, keyed by the context's unique ID: the
// address belongs to the module loaded in that context, so a call made in
// another context of the same device, or after cudaDeviceReset has replaced
// the primary context, does its own set-up instead of reusing a stale
// address.  Bodies are processed in input order (no Morton sort, which would
// need more scratch).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "nb_internal.h"

namespace {

constexpr int64_t kMaxBodies = NB_NOALLOC_MAX_BODIES;
constexpr int64_t kMaxSplitBodies = 4 * kMaxBodies;  // sum over splits of partial rows
constexpr int kMaxCounters = 1024;
constexpr int kVariant = 2;  // (128 threads, 8 bodies/thread, j-tile 128)

// Byte layout of the static scratch.
constexpr size_t kPackBytes = (size_t)kMaxBodies * 2 * sizeof(float4);  // hi + lo
constexpr size_t kPartialOff = kPackBytes;
constexpr size_t kPartialBytes = (size_t)kMaxSplitBodies * 3 * sizeof(double);
constexpr size_t kCountersOff = kPartialOff + kPartialBytes;
constexpr size_t kErrOff = kCountersOff + kMaxCounters * sizeof(unsigned);
constexpr size_t kScratchBytes = kErrOff + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Set-up results, one slot per CUDA context that has called the entry point
// (slots are reused round-robin once all are taken).
constexpr int kSlots = 64;
struct Setup {
    unsigned long long ctx_id;  // cuCtxGetId of the context; 0 = free slot
    unsigned char *addr;        // device address of the scratch in that context
    int sms;
};
std::mutex g_mu;
Setup g_setup[kSlots] = {};
int g_next = 0;

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

void *driver_fn(const char *name, int version)
{
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &f, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return f;
}

// Unique ID (never reused within the process) of the calling thread's
// current CUDA context; 0 if there is none.
unsigned long long current_ctx_id()
{
    static PfnCtxGetCurrent get_cur = (PfnCtxGetCurrent)driver_fn("cuCtxGetCurrent", 4000);
    static PfnCtxGetId get_id = (PfnCtxGetId)driver_fn("cuCtxGetId", 12000);
    if (!get_cur || !get_id) return 0;
    CUcontext cur = nullptr;
    unsigned long long id = 0;
    if (get_cur(&cur) != CUDA_SUCCESS || !cur) return 0;
    if (get_id(cur, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Errors are reported by status code only (there is no context to hold a
// message); the text names the check for readers of this file.
nb_status fail(nb_status s, const char *) { return s; }

typedef CUresult (*PfnRange)(CUdeviceptr *, size_t *, CUdeviceptr);

// `bytes` bytes at p: device (or managed) memory of device `dev`, inside one
// allocation when the driver can tell.
bool is_device_array(const void *p, size_t bytes, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeManaged && !(a.type == cudaMemoryTypeDevice && a.device == dev))
        return false;
    static PfnRange range = (PfnRange)driver_fn("cuMemGetAddressRange", 3020);
    if (range) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (range(&base, &size, (CUdeviceptr)(uintptr_t)p) == CUDA_SUCCESS &&
            (uintptr_t)p + bytes > (uintptr_t)base + size)
            return false;
    }
    return true;
}

}  // namespace

extern "C" nb_status nb_forces_noalloc(int64_t n, const double *pos, const double *mass, double G,
                                       double eps, double *acc, void *cuda_stream)
{
    if (n < 0 || n > kMaxBodies)
        return fail(NB_EINVAL, "n outside [0, NB_NOALLOC_MAX_BODIES]");
    if (!std::isfinite(G)) return fail(NB_EINVAL, "G is not finite");
    if (!std::isfinite(eps) || eps < 0) return fail(NB_EINVAL, "eps must be finite and >= 0");
    if (n == 0) return NB_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return fail(NB_ECUDA, "no current CUDA device");
    }
    const void *arrays[3] = {pos, mass, acc};
    const size_t bytes[3] = {(size_t)n * 3 * sizeof(double), (size_t)n * sizeof(double),
                             (size_t)n * 3 * sizeof(double)};
    for (int q = 0; q < 3; ++q) {
        if (!arrays[q] || (uintptr_t)arrays[q] % 8)
            return fail(NB_EINVAL, "array NULL or not 8-byte aligned");
        if (!is_device_array(arrays[q], bytes[q], dev))
            return fail(NB_EINVAL, "array not n bodies of device memory of the current device");
    }

    // Set-up, once per CUDA context (the argument checks above have run in
    // the current one): the scratch array's device address in that context.
    const unsigned long long ctx_id = current_ctx_id();
    if (!ctx_id) return fail(NB_ECUDA, "no CUDA context is current");
    unsigned char *base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (const Setup &e : g_setup)
            if (e.ctx_id == ctx_id) {
                base = e.addr;
                sms = e.sms;
            }
        if (!base) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return fail(NB_ECUDA, "cudaGetSymbolAddress failed");
            }
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                return fail(NB_ECUDA, "cannot read the SM count");
            }
            base = (unsigned char *)p;
            g_setup[g_next] = Setup{ctx_id, base, sms};
            g_next = (g_next + 1) % kSlots;
        }
    }

    cudaStream_t s = (cudaStream_t)cuda_stream;
    float4 *Phi = (float4 *)base;
    float4 *Plo = Phi + kMaxBodies;
    double *partial = (double *)(base + kPartialOff);
    unsigned *counters = (unsigned *)(base + kCountersOff);
    int *err = (int *)(base + kErrOff);

    const nb::KernelEntry &k = nb::f32_force_kernel(kVariant, true, eps == 0.0);
    const int64_t tile = (int64_t)k.T * k.I;
    const int64_t n_itiles = (n + tile - 1) / tile;
    const int64_t n_jtiles = (n + k.J - 1) / k.J;
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.fn, k.T, 0) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    int S = nb::choose_split(n_itiles, n_jtiles, (int64_t)sms * std::max(occ, 1), kMaxSplitBodies,
                             tile);
    while (S > 1 && (int64_t)S * n > kMaxSplitBodies) --S;
    if (S < 1) S = 1;

    // The counters and the error word must start at zero; clear them here
    // rather than trusting the previous call's contents.
    cudaError_t e = cudaMemsetAsync(counters, 0, (size_t)n_itiles * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = nb::launch_pack_hilo(s, (int)n, pos, mass, nullptr, Phi, Plo);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NB_ECUDA, "memset or pack launch failed");
    }

    nb::ForceParams p;
    p.P = Phi;
    p.Plo = Plo;
    p.perm = nullptr;
    p.n = (int)n;
    p.nsplit = S;
    p.eps2f = (float)(eps * eps);
    p.eps2 = eps * eps;
    p.G = G;
    p.acc = acc;
    p.vel = nullptr;
    p.half_dt = 0.0;
    p.partial = partial;
    p.counters = counters;
    p.err = err;
    void *args[] = {&p};
    e = cudaLaunchKernel(k.fn, dim3((unsigned)(n_itiles * S)), dim3(k.T), args, 0, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NB_ECUDA, "force kernel launch failed");
    }
    return NB_OK;
}

static_assert(kMaxBodies / 256 + 1 <= kMaxCounters, "counter scratch too small");
