// FP64 instantiations of the grouped regime (i) kernel for an A that a tensor
// map cannot describe, in each load form.
#include "tsmm_group.cuh"

namespace tsmm {
cudaError_t launch_grouped_async_f64(int np, int lv, const GroupParams &gp, cudaStream_t s) {
    return launch_grouped_async_dispatch<double>(np, lv, gp, s);
}
}  // namespace tsmm
