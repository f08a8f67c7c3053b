// FP32 instantiations of the grouped regime (i) kernel.
#include "tsmm_group.cuh"

namespace tsmm {
cudaError_t launch_grouped_f32(int np, bool unaligned, int lv, const GroupParams &gp, cudaStream_t s) {
    return launch_grouped_dispatch<float>(np, unaligned, lv, gp, s);
}
}  // namespace tsmm
