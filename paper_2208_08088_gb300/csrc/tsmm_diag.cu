// Diagnostics: the bounded mbarrier wait that every kernel of the library
// uses, run against a barrier that nothing completes, so that the timeout
// path (status word set, kernel returns, context stays usable) can be tested
// on a GPU without a fault or a hang.
#include "tsmm_device.cuh"
#include "tsmm_internal.h"

namespace tsmm {

__global__ void diag_wait_kernel(uint32_t polls, unsigned *status, unsigned long long *cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        // no thread arrives: phase 0 never completes and the wait runs out
        const bool got = mbar_wait_bounded(&bar, 0, polls);
        *cycles = (unsigned long long)(clock64() - t0);
        if (!got) atomicOr(status, kDevErrTimeout);
    }
}

}  // namespace tsmm

using namespace tsmm;

extern "C" tsmm_status tsmm_diag_bounded_wait(uint32_t polls, uint64_t *cycles_out, double *seconds_out) {
    if (polls == 0) return TSMM_ERR_INVALID_ARG;
    void *buf = nullptr;
    if (cudaMalloc(&buf, 16) != cudaSuccess) return TSMM_ERR_CUDA;
    unsigned *status = static_cast<unsigned *>(buf);
    unsigned long long *cycles = reinterpret_cast<unsigned long long *>(static_cast<char *>(buf) + 8);
    tsmm_status st = TSMM_OK;
    unsigned long long host[2] = {0, 0};
    if (cudaMemset(buf, 0, 16) != cudaSuccess) {
        st = TSMM_ERR_CUDA;
    } else {
        diag_wait_kernel<<<1, 32>>>(polls, status, cycles);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(host, buf, 16, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = TSMM_ERR_CUDA;
    }
    cudaFree(buf);
    if (st != TSMM_OK) return st;
    const uint64_t cyc = host[1];
    if (cycles_out) *cycles_out = cyc;
    if (seconds_out) {
        int dev = 0, khz = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        *seconds_out = khz > 0 ? (double)cyc / ((double)khz * 1e3) : 0.0;
    }
    return (host[0] & kDevErrTimeout) ? TSMM_ERR_TIMEOUT : TSMM_OK;
}
