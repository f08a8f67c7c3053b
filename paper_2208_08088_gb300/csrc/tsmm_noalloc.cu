// tsmm_execute_noalloc: the regime (i) split-K path with all of its scratch
// (packed B, partial tiles, arrival counters, error word) in one file-scope
// device array, for callers that cannot allocate device memory.  Nothing here
// calls cudaMalloc, cudaFree or any allocating library routine.
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "tsmm_device.cuh"
#include "tsmm_internal.h"

using namespace tsmm;

namespace {

constexpr size_t kScratchBytes = TSMM_NOALLOC_SCRATCH_BYTES;
constexpr size_t kAlign = 256;

// The scratch itself: every device that loads this library holds it until exit.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host-side device addresses of g_scratch, one per device (the symbol name in
// host code is only a host stand-in and must never be passed to a kernel).
constexpr int kMaxDevices = 128;
std::mutex g_mu;
void *g_scratch_dev[kMaxDevices] = {};

PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;
std::once_flag g_enc_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    std::call_once(g_enc_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_enc;
}

// Set-up, once per device, with that device current: look up the device
// address of g_scratch.
tsmm_status scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return TSMM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return TSMM_ERR_CUDA;
        }
        g_scratch_dev[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_dev[dev]);
    return TSMM_OK;
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

tsmm_status from_cuda(cudaError_t e) { return e == cudaSuccess ? TSMM_OK : TSMM_ERR_CUDA; }

}  // namespace

extern "C" tsmm_status tsmm_execute_noalloc(tsmm_dtype dtype, int64_t m, int64_t n, int64_t k,
                                            double alpha, const void *A_dev, int64_t lda,
                                            const void *B_dev, int64_t ldb, double beta,
                                            void *C_dev, int64_t ldc, tsmm_stream_t stream) {
    // ---- argument checks (no device work yet)
    if ((dtype != TSMM_F32 && dtype != TSMM_F64) || m < 0 || n < 0 || k < 0)
        return TSMM_ERR_INVALID_ARG;
    if (lda < std::max<int64_t>(1, m) || ldc < std::max<int64_t>(1, m) ||
        ldb < std::max<int64_t>(1, k))
        return TSMM_ERR_INVALID_ARG;
    if (n > kTallMaxN) return TSMM_ERR_UNSUPPORTED_SHAPE;
    const size_t es = dtype_size(dtype);
    const int np = tall_np(n);
    const int bm = tall_bm(dtype, np);
    const int64_t kp = round_up(k, kTallBKS);
    const int64_t slabs = (m + bm - 1) / bm;
    // scratch layout: [error word][arrival counters][packed B][split-K partials]
    const size_t off_tickets = kAlign;
    const size_t tickets_bytes = align_up((size_t)slabs * sizeof(unsigned));
    const size_t off_b = off_tickets + tickets_bytes;
    const size_t b_bytes = align_up((size_t)kp * (size_t)np * es);
    const size_t off_ws = off_b + b_bytes;
    if (off_ws > kScratchBytes) return TSMM_ERR_UNSUPPORTED_SHAPE;
    if (m == 0 || n == 0) return TSMM_OK;
    const bool use_ab = (alpha != 0.0) && (k > 0) &&
                        !(dtype == TSMM_F32 && static_cast<float>(alpha) == 0.0f);
    if (!C_dev || (use_ab && (!A_dev || !B_dev))) return TSMM_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(C_dev) % es != 0 ||
        (use_ab && (reinterpret_cast<uintptr_t>(A_dev) % es != 0 ||
                    reinterpret_cast<uintptr_t>(B_dev) % es != 0)))
        return TSMM_ERR_MISALIGNED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!use_ab) return from_cuda(launch_scale(dtype, m, n, beta, C_dev, ldc, s));

    int dev = -1, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSMM_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TSMM_ERR_CUDA;
    unsigned char *scratch = nullptr;
    tsmm_status st = scratch_address(dev, &scratch);
    if (st != TSMM_OK) return st;

    // ---- split-K factor limited by the partial-tile room left in the scratch
    const int64_t kstages = kp / kTallBKS;
    const int64_t per_split = (int64_t)np * slabs * bm * (int64_t)es;
    const int64_t room = (int64_t)(kScratchBytes - off_ws);
    int64_t max_splits = std::min<int64_t>(65535, per_split > 0 ? room / per_split : 1);
    if (max_splits < 2) max_splits = 1;
    const int splits_req =
        choose_splits(slabs, kstages, sms, max_splits, tall_resident_blocks(dtype == TSMM_F64, np));
    const int64_t chunk_stages = (kstages + splits_req - 1) / splits_req;
    const int splits = (int)((kstages + chunk_stages - 1) / chunk_stages);

    unsigned *status = reinterpret_cast<unsigned *>(scratch);
    unsigned *tickets = reinterpret_cast<unsigned *>(scratch + off_tickets);
    void *packed = scratch + off_b;
    void *ws = scratch + off_ws;

    // ---- what must start at zero: the error word and the arrival counters
    cudaError_t e = cudaMemsetAsync(scratch, 0, off_b, s);
    if (e != cudaSuccess) return TSMM_ERR_CUDA;
    e = launch_pack_b(dtype, k, n, B_dev, ldb, packed, kp, np, 1, s);
    if (e != cudaSuccess) return TSMM_ERR_CUDA;

    TallArgs a;
    a.m = m;
    a.n = n;
    a.k = k;
    a.lda = lda;
    a.ldc = ldc;
    a.A = A_dev;
    a.Bp = packed;
    a.C = C_dev;
    a.alpha = alpha;
    a.beta = beta;
    a.ws = splits > 1 ? ws : nullptr;
    a.tickets = tickets;
    a.status = status;
    a.splits = splits;
    a.kchunk = chunk_stages * kTallBKS;
    a.kp = kp;
    a.slabs = slabs;

    CUtensorMap tmap;
    const bool tma = reinterpret_cast<uintptr_t>(A_dev) % 16 == 0 &&
                     (lda * (int64_t)es) % 16 == 0 && m < INT_MAX && k < INT_MAX &&
                     (lda * (int64_t)es) < (1LL << 40) && encoder() != nullptr;
    if (tma) {
        const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)k};
        const cuuint64_t gstride[1] = {(cuuint64_t)(lda * (int64_t)es)};
        const cuuint32_t box[2] = {(cuuint32_t)bm, (cuuint32_t)kTallBKS};
        const cuuint32_t estr[2] = {1, 1};
        if (encoder()(&tmap,
                      dtype == TSMM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                      2, const_cast<void *>(A_dev), gdim, gstride, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return TSMM_ERR_CUDA;
    }
    e = dtype == TSMM_F32 ? launch_tall_f32(tma, np, &tmap, a, s)
                          : launch_tall_f64(tma, np, &tmap, a, s);
    return from_cuda(e);
}
