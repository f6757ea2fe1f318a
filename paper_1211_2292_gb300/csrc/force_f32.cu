// float32 force kernel variants 0..10 (kernels in force_f32.cuh).  The
// variant table is split over translation units so that nvcc compiles them in
// parallel.
#include "force_f32.cuh"

namespace nb {
namespace {

const Quad kForceA[] = {
    // rsqrt form (variants 0..7)
    NB_F32_ENTRY(128, 4, 128, 0),
    NB_F32_ENTRY(256, 4, 256, 0),
    NB_F32_ENTRY(128, 8, 128, 0),
    NB_F32_ENTRY(256, 2, 256, 0),
    NB_F32_ENTRY(64, 8, 128, 0),
    NB_F32_ENTRY(128, 6, 256, 0),
    NB_F32_ENTRY(256, 8, 256, 0),
    NB_F32_ENTRY(128, 2, 256, 0),
    // log-domain form for every pair (8..9)
    NB_F32_ENTRY(256, 8, 256, 4),
    NB_F32_ENTRY(64, 8, 128, 4),
    // mixed: LP of the I/2 body pairs in the log-domain form (10..15)
    NB_F32_ENTRY(256, 8, 256, 2),
};

}  // namespace

int f32_force_variants_a() { return (int)(sizeof(kForceA) / sizeof(kForceA[0])); }
const KernelEntry &f32_force_kernel_a(int v, bool comp, bool zeps) { return kForceA[v][comp][zeps]; }

}  // namespace nb
