// FP32 instantiations of the grouped regime (i) kernel.
#include "tsmm_group.cuh"

namespace tsmm {
cudaError_t launch_grouped_f32(int np, const GroupParams &gp, int num_sms, bool persistent,
                               cudaStream_t s) {
    return launch_grouped_dispatch<float>(np, gp, num_sms, persistent, s);
}
}  // namespace tsmm
