// FP32 regime (i) bulk-copy kernel of width 48, in its five load forms.
#include "tsmm_tall.cuh"

namespace tsmm {
template cudaError_t launch_tall_async_t<float, 48>(const TallArgs &, cudaStream_t);
}  // namespace tsmm
