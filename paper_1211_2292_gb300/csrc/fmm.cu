// Fast multipole method: dispatch over the compiled expansion orders (the
// kernels are in fmm_impl.cuh, one translation unit per order).
#include "fmm_impl.cuh"

namespace nb {
namespace fmm {
extern template cudaError_t launch_fmm_order<2>(cudaStream_t, const FmmParams &, bool, int &);
extern template cudaError_t launch_fmm_order<3>(cudaStream_t, const FmmParams &, bool, int &);
extern template cudaError_t launch_fmm_order<4>(cudaStream_t, const FmmParams &, bool, int &);
extern template cudaError_t launch_fmm_order<5>(cudaStream_t, const FmmParams &, bool, int &);
extern template cudaError_t launch_fmm_order<6>(cudaStream_t, const FmmParams &, bool, int &);
static_assert(FMM_MIN_ORDER == 2 && FMM_MAX_ORDER == 6, "one instantiation per order");
}  // namespace fmm

int fmm_floats(int order) { return fmm::padded(order); }

cudaError_t launch_fmm(cudaStream_t s, const FmmParams &p, bool near, int &kernels)
{
    switch (p.f.order) {
    case 2: return fmm::launch_fmm_order<2>(s, p, near, kernels);
    case 3: return fmm::launch_fmm_order<3>(s, p, near, kernels);
    case 4: return fmm::launch_fmm_order<4>(s, p, near, kernels);
    case 5: return fmm::launch_fmm_order<5>(s, p, near, kernels);
    case 6: return fmm::launch_fmm_order<6>(s, p, near, kernels);
    default: kernels = 0; return cudaErrorInvalidValue;
    }
}

}  // namespace nb
