// Batched persistent float32 kernel variants (kernels in force_f32.cuh) and the
// float32 force-table accessors.
#include "force_f32.cuh"

namespace nb {
namespace {

const Quad kBatched[] = {
    NB_F32B_ENTRY(128, 2, 128, 0),
    NB_F32B_ENTRY(128, 4, 128, 0),
    NB_F32B_ENTRY(256, 2, 256, 0),
    NB_F32B_ENTRY(64, 4, 128, 0),
    // wider tiles, mixed rsqrt / log-domain pairs (4..7)
    NB_F32B_ENTRY(128, 6, 256, 2),
    NB_F32B_ENTRY(64, 6, 128, 2),
    NB_F32B_ENTRY(128, 8, 128, 0),
    NB_F32B_ENTRY(128, 4, 128, 1),
    // the solo kernel's mixed shapes on 128-body j-tiles (8..10)
    NB_F32B_ENTRY(128, 6, 128, 2),
    NB_F32B_ENTRY(128, 8, 128, 3),
    NB_F32B_ENTRY(64, 8, 128, 3),
};

}  // namespace

int f32_force_variants() { return f32_force_variants_a() + f32_force_variants_b(); }
const KernelEntry &f32_force_kernel(int v, bool comp, bool zeps)
{
    const int na = f32_force_variants_a();
    return v < na ? f32_force_kernel_a(v, comp, zeps) : f32_force_kernel_b(v - na, comp, zeps);
}
int f32_batched_variants() { return (int)(sizeof(kBatched) / sizeof(kBatched[0])); }
const KernelEntry &f32_batched_kernel(int v, bool comp, bool zeps)
{
    return kBatched[v][comp][zeps];
}

}  // namespace nb
