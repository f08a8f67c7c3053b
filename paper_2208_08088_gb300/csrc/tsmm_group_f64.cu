// FP64 instantiations of the grouped regime (i) kernel.
#include "tsmm_group.cuh"

namespace tsmm {
cudaError_t launch_grouped_f64(int np, const GroupParams &gp, int num_sms, bool persistent,
                               cudaStream_t s) {
    return launch_grouped_dispatch<double>(np, gp, num_sms, persistent, s);
}
}  // namespace tsmm
