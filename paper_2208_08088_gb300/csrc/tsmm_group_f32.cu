// FP32 instantiations of the grouped regime (i) kernel for tensor-map A (an A
// that a tensor map cannot describe: tsmm_group_async_f32.cu).
#include "tsmm_group.cuh"

namespace tsmm {
cudaError_t launch_grouped_f32(int np, bool unaligned, int lv, const GroupParams &gp, cudaStream_t s) {
    return unaligned ? launch_grouped_async_f32(np, lv, gp, s) : launch_grouped_tma_dispatch<float>(np, gp, s);
}
}  // namespace tsmm
