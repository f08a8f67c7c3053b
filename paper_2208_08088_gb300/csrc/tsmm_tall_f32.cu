// FP32 instantiations of the regime (i) TMA kernel (the bulk-copy kernel for
// an A that a tensor map cannot describe: tsmm_tall_async_f32.cu).
#include "tsmm_tall.cuh"

namespace tsmm {
cudaError_t launch_tall_f32(bool tma, int np, const CUtensorMap *tmap, const TallArgs &a,
                            cudaStream_t s) {
    return tma ? launch_tall_tma_dispatch<float>(np, tmap, a, s) : launch_tall_async_f32(np, a, s);
}
}  // namespace tsmm
