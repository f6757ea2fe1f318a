// Fast multipole method kernels of expansion order 4.
#include "fmm_impl.cuh"

namespace nb {
namespace fmm {
template cudaError_t launch_fmm_order<4>(cudaStream_t, const FmmParams &, bool, int &);
}  // namespace fmm
}  // namespace nb
