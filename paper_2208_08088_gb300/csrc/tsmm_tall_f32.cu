// FP32 instantiations of the regime (i) kernels.
#include "tsmm_tall.cuh"

namespace tsmm {
cudaError_t launch_tall_f32(bool tma, int np, const CUtensorMap *tmap, const TallArgs &a,
                            cudaStream_t s) {
    return launch_tall_dispatch<float>(tma, np, tmap, a, s);
}
}  // namespace tsmm
