// float32 force kernel variants 11.. (kernels in force_f32.cuh).  The
// variant table is split over translation units so that nvcc compiles them in
// parallel.
#include "force_f32.cuh"

namespace nb {
namespace {

const Quad kForceB[] = {
    NB_F32_ENTRY(256, 8, 256, 3),
    NB_F32_ENTRY(128, 6, 256, 2),
    NB_F32_ENTRY(256, 6, 256, 2),
    NB_F32_ENTRY(64, 8, 128, 2),
    NB_F32_ENTRY(128, 8, 128, 3),
    // Kahan state in shared memory, registers capped at 128 for 4 CTAs of
    // 128 threads per SM (16..17)
    NB_F32_ENTRY_X(128, 8, 128, 0, true, 4),
    NB_F32_ENTRY_X(128, 6, 128, 2, true, 4),
    // mixed, registers capped for 3 CTAs of 128 threads per SM (18..20)
    NB_F32_ENTRY_X(128, 6, 256, 2, false, 3),
    NB_F32_ENTRY_X(128, 6, 256, 2, true, 3),
    NB_F32_ENTRY_X(128, 6, 128, 2, true, 3),
};

}  // namespace

int f32_force_variants_b() { return (int)(sizeof(kForceB) / sizeof(kForceB[0])); }
const KernelEntry &f32_force_kernel_b(int v, bool comp, bool zeps) { return kForceB[v][comp][zeps]; }

}  // namespace nb
