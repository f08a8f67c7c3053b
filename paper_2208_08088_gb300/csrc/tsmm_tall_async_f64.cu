// FP64 instantiations of the regime (i) bulk-copy kernel (an A that a
// tensor map cannot describe).
#include "tsmm_tall.cuh"

namespace tsmm {
cudaError_t launch_tall_async_f64(int np, const TallArgs &a, cudaStream_t s) {
    return launch_tall_async_dispatch<double>(np, a, s);
}
}  // namespace tsmm
