// Fast multipole method kernels of expansion order 2.
#include "fmm_impl.cuh"

namespace nb {
namespace fmm {
template cudaError_t launch_fmm_order<2>(cudaStream_t, const FmmParams &, bool, int &);
}  // namespace fmm
}  // namespace nb
