// FP32 instantiations of the regime (i) bulk-copy kernel (an A that a tensor
// map cannot describe): widths up to 24 here, 32 / 48 / 64 (five load forms
// each) in tsmm_tall_async_f32_w<width>.cu, compiled in parallel.
#include "tsmm_tall.cuh"

namespace tsmm {
extern template cudaError_t launch_tall_async_t<float, 32>(const TallArgs &, cudaStream_t);
extern template cudaError_t launch_tall_async_t<float, 48>(const TallArgs &, cudaStream_t);
extern template cudaError_t launch_tall_async_t<float, 64>(const TallArgs &, cudaStream_t);

cudaError_t launch_tall_async_f32(int np, const TallArgs &a, cudaStream_t s) {
    return launch_tall_async_dispatch<float>(np, a, s);
}
}  // namespace tsmm
