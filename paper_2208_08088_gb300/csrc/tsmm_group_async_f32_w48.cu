// FP32 grouped regime (i) kernel of width 48 for an A that a tensor map cannot
// describe, in its five load forms.
#include "tsmm_group.cuh"

namespace tsmm {
template cudaError_t launch_grouped_async_np<float, 48>(int, const GroupParams &, cudaStream_t);
}  // namespace tsmm
