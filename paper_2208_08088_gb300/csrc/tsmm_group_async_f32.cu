// FP32 instantiations of the grouped regime (i) kernel for an A that a tensor
// map cannot describe, in each load form: widths up to 24 here, 32 / 48 / 64
// in tsmm_group_async_f32_w<width>.cu, compiled in parallel.
#include "tsmm_group.cuh"

namespace tsmm {
extern template cudaError_t launch_grouped_async_np<float, 32>(int, const GroupParams &, cudaStream_t);
extern template cudaError_t launch_grouped_async_np<float, 48>(int, const GroupParams &, cudaStream_t);
extern template cudaError_t launch_grouped_async_np<float, 64>(int, const GroupParams &, cudaStream_t);

cudaError_t launch_grouped_async_f32(int np, int lv, const GroupParams &gp, cudaStream_t s) {
    return launch_grouped_async_dispatch<float>(np, lv, gp, s);
}
}  // namespace tsmm
