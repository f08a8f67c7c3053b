// PACKB of Algorithm 1 (bit-preserving re-layout of B into column tiles of
// row-major panels), and the alpha == 0 / k == 0 path C = beta * C0.
#include "tsmm_device.cuh"
#include "tsmm_internal.h"

namespace tsmm {

// One thread per packed element.  dst tile t: kp x w row-major at t*kp*w;
// element (p, jj) <- B[p + (t*w + jj)*ldb], or +0 outside the k x n matrix.
// Consecutive threads write consecutive packed elements (coalesced stores);
// the gather from column-major B is served by L1/L2 (B is small and read once).
template <typename T>
__global__ void pack_b_kernel(const T *__restrict__ B, int64_t k, int64_t n, int64_t ldb,
                              T *__restrict__ dst, int64_t kp, int64_t w, int64_t total) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / (kp * w);
        const int64_t rem = e - t * kp * w;
        const int64_t p = rem / w;
        const int64_t j = t * w + (rem - p * w);
        dst[e] = (p < k && j < n) ? B[p + j * ldb] : T(0);
    }
}

// C = beta * C0 (beta != 0) or C = 0 (beta == 0, C0 not read).
template <typename T>
__global__ void scale_kernel(int64_t m, int64_t n, T beta, T *__restrict__ C, int64_t ldc) {
    const int64_t total = m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / m;
        const int64_t i = e - j * m;
        T *c = C + i + j * ldc;
        *c = (beta != T(0)) ? beta * *c : T(0);
    }
}

// dst[i + p*ldd] = src[i + p*lds] for i < m, p < k (blockIdx.y = p): a
// column-major copy into another leading dimension.  Regime (ii) uses it to give
// an A that a tensor map cannot describe an aligned copy that one can.
template <typename T>
__global__ void copy_columns_kernel(const T *__restrict__ src, int64_t lds, int64_t m, T *__restrict__ dst,
                                    int64_t ldd) {
    const T *sc = src + (int64_t)blockIdx.y * lds;
    T *dc = dst + (int64_t)blockIdx.y * ldd;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        dc[i] = sc[i];
}

static unsigned grid_for(int64_t total, int threads) {
    int64_t blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    return (unsigned)blocks;
}

cudaError_t launch_pack_b(tsmm_dtype dt, int64_t k, int64_t n, const void *B, int64_t ldb,
                          void *dst, int64_t kp, int64_t w, int64_t ntiles, cudaStream_t s) {
    const int64_t total = kp * w * ntiles;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    if (dt == TSMM_F32)
        pack_b_kernel<float><<<grid_for(total, threads), threads, 0, s>>>(
            static_cast<const float *>(B), k, n, ldb, static_cast<float *>(dst), kp, w, total);
    else
        pack_b_kernel<double><<<grid_for(total, threads), threads, 0, s>>>(
            static_cast<const double *>(B), k, n, ldb, static_cast<double *>(dst), kp, w, total);
    return cudaGetLastError();
}

cudaError_t launch_copy_columns(tsmm_dtype dt, const void *src, int64_t lds, int64_t m, int64_t k, void *dst,
                                int64_t ldd, cudaStream_t s) {
    if (m == 0 || k == 0) return cudaSuccess;
    if (k > 65535) return cudaErrorInvalidValue;
    const int threads = 256;
    int64_t bx = (m + threads - 1) / threads;
    if (bx > 64) bx = 64;
    const dim3 grid((unsigned)bx, (unsigned)k);
    if (dt == TSMM_F32)
        copy_columns_kernel<float><<<grid, threads, 0, s>>>(static_cast<const float *>(src), lds, m,
                                                            static_cast<float *>(dst), ldd);
    else
        copy_columns_kernel<double><<<grid, threads, 0, s>>>(static_cast<const double *>(src), lds, m,
                                                             static_cast<double *>(dst), ldd);
    return cudaGetLastError();
}

cudaError_t launch_scale(tsmm_dtype dt, int64_t m, int64_t n, double beta, void *C, int64_t ldc,
                         cudaStream_t s) {
    const int64_t total = m * n;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    if (dt == TSMM_F32)
        scale_kernel<float><<<grid_for(total, threads), threads, 0, s>>>(
            m, n, static_cast<float>(beta), static_cast<float *>(C), ldc);
    else
        scale_kernel<double><<<grid_for(total, threads), threads, 0, s>>>(
            m, n, beta, static_cast<double *>(C), ldc);
    return cudaGetLastError();
}

}  // namespace tsmm
