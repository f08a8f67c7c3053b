// The C ABI (include/tsmm.h): argument checking, the planner, packed-B and
// plan lifetimes, and kernel dispatch.  No entry point throws or aborts.
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <new>

#include "tsmm_device.cuh"
#include "tsmm_internal.h"

using namespace tsmm;

namespace {

constexpr int kVersion = 100;  // 0.1.0

// Resolved once: the driver's tensor-map encoder (no -lcuda link needed).
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode;
}

bool valid_dtype(tsmm_dtype d) { return d == TSMM_F32 || d == TSMM_F64; }

bool aligned(const void *p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

thread_local const char *g_last_cuda_error = "no error";

tsmm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return TSMM_OK;
    g_last_cuda_error = cudaGetErrorString(e);  // static string owned by the runtime
    if (e == cudaErrorMemoryAllocation) return TSMM_ERR_OUT_OF_MEMORY;
    return TSMM_ERR_CUDA;
}

int current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    return dev;
}

// C may be read by TMA: 16-byte aligned base and column stride, sizes in range.
bool c_tma_ok(const void *C_dev, int64_t ldc, int64_t n, size_t es) {
    return aligned(C_dev, 16) && ((ldc * (int64_t)es) % 16 == 0) && n < INT_MAX &&
           (ldc * (int64_t)es) < (1LL << 40) && encoder() != nullptr;
}

// (Re)encode the plan's cached tensor map of C (box 128-or-bm rows x `cols`)
// when C's address or stride changed since the last execute.
tsmm_status encode_tmapc(tsmm_plan_t p, void *C_dev, int64_t m, int64_t n, int64_t ldc, size_t es,
                         int cols) {
    if (p->tmapc_ptr == C_dev && p->tmapc_ldc == ldc) return TSMM_OK;
    const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)n};
    const cuuint64_t gstride[1] = {(cuuint64_t)(ldc * (int64_t)es)};
    const cuuint32_t box[2] = {(cuuint32_t)p->bm, (cuuint32_t)cols};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encoder()(&p->tmapc,
                           p->dtype == TSMM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                           2, C_dev, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        p->tmapc_ptr = nullptr;
        return TSMM_ERR_CUDA;
    }
    p->tmapc_ptr = C_dev;
    p->tmapc_ldc = ldc;
    return TSMM_OK;
}

}  // namespace

namespace tsmm {

// Split-K choice for regime (i): minimise a wave-quantised time model
//   T(S) = ceil(slabs*S / resident) * (ceil(kstages / S) + overhead)
// where `resident` thread blocks run at once (per SM, times the SM count) and
// `overhead` is the per-block fixed cost (pipeline fill, reduction, epilogue)
// in stage units.  Smallest S wins ties, which also keeps the workspace small.
int choose_splits(int64_t slabs, int64_t kstages, int num_sms, int64_t max_splits,
                  int per_sm) {
    const int64_t resident = (int64_t)per_sm * num_sms;
    const int64_t overhead = 4;
    int64_t best_s = 1;
    double best_t = -1.0;
    const int64_t s_max = std::max<int64_t>(1, std::min<int64_t>(kstages, max_splits));
    for (int64_t s = 1; s <= s_max; ++s) {
        const int64_t waves = (slabs * s + resident - 1) / resident;
        const int64_t per = (kstages + s - 1) / s + overhead;
        const double t = (double)waves * (double)per;
        if (best_t < 0 || t < best_t) {
            best_t = t;
            best_s = s;
        }
    }
    return (int)best_s;
}

}  // namespace tsmm

extern "C" {

const char *tsmm_status_string(tsmm_status status) {
    switch (status) {
        case TSMM_OK: return "TSMM_OK";
        case TSMM_ERR_INVALID_ARG: return "TSMM_ERR_INVALID_ARG";
        case TSMM_ERR_UNSUPPORTED_SHAPE: return "TSMM_ERR_UNSUPPORTED_SHAPE";
        case TSMM_ERR_MISMATCH: return "TSMM_ERR_MISMATCH";
        case TSMM_ERR_MISALIGNED: return "TSMM_ERR_MISALIGNED";
        case TSMM_ERR_OUT_OF_MEMORY: return "TSMM_ERR_OUT_OF_MEMORY";
        case TSMM_ERR_CUDA: return "TSMM_ERR_CUDA";
        case TSMM_ERR_TIMEOUT: return "TSMM_ERR_TIMEOUT";
    }
    return "TSMM_ERR_UNKNOWN";
}

int tsmm_version(void) { return kVersion; }

const char *tsmm_last_cuda_error(void) { return g_last_cuda_error; }

tsmm_status tsmm_pack_b(tsmm_dtype dtype, int64_t k, int64_t n, const void *B_dev, int64_t ldb,
                        tsmm_stream_t stream, tsmm_packed_b *out) {
    return tsmm_pack_b_ex(dtype, TSMM_PREC_NATIVE, k, n, B_dev, ldb, stream, out);
}

tsmm_status tsmm_pack_b_ex(tsmm_dtype dtype, tsmm_precision precision, int64_t k, int64_t n,
                           const void *B_dev, int64_t ldb, tsmm_stream_t stream, tsmm_packed_b *out) {
    if (!out || !valid_dtype(dtype) || k < 0 || n < 0) return TSMM_ERR_INVALID_ARG;
    if (precision != TSMM_PREC_NATIVE && precision != TSMM_PREC_BF16X3) return TSMM_ERR_INVALID_ARG;
    if (precision == TSMM_PREC_BF16X3 && dtype != TSMM_F32) return TSMM_ERR_INVALID_ARG;
    if (ldb < std::max<int64_t>(1, k)) return TSMM_ERR_INVALID_ARG;
    if (k > 0 && n > 0 && !B_dev) return TSMM_ERR_INVALID_ARG;
    const size_t es = dtype_size(dtype);
    if (B_dev && !aligned(B_dev, es)) return TSMM_ERR_MISALIGNED;
    const int regime = regime_of(k, n);
    if (regime == 0) return TSMM_ERR_UNSUPPORTED_SHAPE;
    const int dev = current_device();
    if (dev < 0) return TSMM_ERR_CUDA;

    tsmm_packed_b pb = new (std::nothrow) tsmm_packed_b_s();
    if (!pb) return TSMM_ERR_OUT_OF_MEMORY;
    pb->dtype = dtype;
    pb->precision = precision;
    pb->k = k;
    pb->n = n;
    pb->regime = regime;
    pb->device = dev;
    if (precision == TSMM_PREC_BF16X3) {
        pb->kp = round_up(k, kX3KB);
        pb->w = regime == 1 ? x3_np(n) : kX3RankNT;
        pb->ntiles = regime == 1 ? 1 : (n + kX3RankNT - 1) / kX3RankNT;
    } else if (regime == 1) {
        pb->kp = round_up(k, kTallBKS);
        pb->w = tall_np(n);
        pb->ntiles = 1;
    } else {
        pb->kp = round_up(k, kRankKGran);
        pb->w = kRankNT;
        pb->ntiles = (n + kRankNT - 1) / kRankNT;
    }
    // BF16x3: a hi and a lo BF16 copy of every element
    pb->bytes = precision == TSMM_PREC_BF16X3 ? (size_t)(pb->kp * pb->w * pb->ntiles) * 2 * 2
                                              : (size_t)(pb->kp * pb->w * pb->ntiles) * es;
    pb->data = nullptr;
    if (pb->bytes > 0) {
        cudaError_t e = cudaMalloc(&pb->data, pb->bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete pb;
            return cuda_status(e);
        }
        e = precision == TSMM_PREC_BF16X3
                ? launch_pack_b_bf16x3(k, n, B_dev, ldb, pb->data, (int)pb->w, pb->kp / kX3KB,
                                       pb->ntiles, static_cast<cudaStream_t>(stream))
                : launch_pack_b(dtype, k, n, B_dev, ldb, pb->data, pb->kp, pb->w, pb->ntiles,
                                static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) {
            cudaFree(pb->data);
            delete pb;
            return cuda_status(e);
        }
    }
    *out = pb;
    return TSMM_OK;
}

tsmm_status tsmm_packed_b_destroy(tsmm_packed_b pb) {
    if (!pb) return TSMM_OK;
    tsmm_status st = TSMM_OK;
    if (pb->data) st = cuda_status(cudaFree(pb->data));
    delete pb;
    return st;
}

tsmm_status tsmm_packed_b_info(tsmm_packed_b pb, tsmm_dtype *dtype, int64_t *k, int64_t *n,
                               int64_t *kp, int64_t *w, int64_t *ntiles, const void **data_dev,
                               size_t *bytes) {
    if (!pb) return TSMM_ERR_INVALID_ARG;
    if (dtype) *dtype = pb->dtype;
    if (k) *k = pb->k;
    if (n) *n = pb->n;
    if (kp) *kp = pb->kp;
    if (w) *w = pb->w;
    if (ntiles) *ntiles = pb->ntiles;
    if (data_dev) *data_dev = pb->data;
    if (bytes) *bytes = pb->bytes;
    return TSMM_OK;
}

tsmm_status tsmm_packed_b_read(tsmm_packed_b pb, void *host_dst, size_t bytes) {
    if (!pb || bytes < pb->bytes || (pb->bytes > 0 && !host_dst)) return TSMM_ERR_INVALID_ARG;
    if (pb->bytes == 0) return TSMM_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return TSMM_ERR_CUDA;
    return cuda_status(cudaMemcpy(host_dst, pb->data, pb->bytes, cudaMemcpyDeviceToHost));
}

tsmm_status tsmm_plan(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype, tsmm_plan_t *out) {
    return tsmm_plan_ex(m, n, k, dtype, TSMM_PREC_NATIVE, out);
}

tsmm_status tsmm_plan_ex(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype, tsmm_precision precision,
                         tsmm_plan_t *out) {
    if (!out || !valid_dtype(dtype) || m < 0 || n < 0 || k < 0) return TSMM_ERR_INVALID_ARG;
    if (precision != TSMM_PREC_NATIVE && precision != TSMM_PREC_BF16X3) return TSMM_ERR_INVALID_ARG;
    if (precision == TSMM_PREC_BF16X3 && dtype != TSMM_F32) return TSMM_ERR_INVALID_ARG;
    int dev = current_device();
    int sms = 0;
    if (dev >= 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 0;
    // a tuned choice recorded in the plan cache wins over the heuristic (native precision)
    const int cached = precision == TSMM_PREC_NATIVE ? plan_cache_lookup(dtype, m, n, k, sms) : 0;
    return create_plan(m, n, k, dtype, cached, out, precision);
}

}  // extern "C"

namespace tsmm {

tsmm_status create_plan(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype, int forced_splits,
                        tsmm_plan_t *out, int precision) {
    if (!out || !valid_dtype(dtype) || m < 0 || n < 0 || k < 0) return TSMM_ERR_INVALID_ARG;
    const int regime = regime_of(k, n);
    if (regime == 0) return TSMM_ERR_UNSUPPORTED_SHAPE;  // before any device query
    const int dev = current_device();
    if (dev < 0) return TSMM_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TSMM_ERR_CUDA;

    tsmm_plan_t p = new (std::nothrow) tsmm_plan_s();
    if (!p) return TSMM_ERR_OUT_OF_MEMORY;
    size_t ticket_bytes = 0;
    tsmm_status st = plan_layout(m, n, k, dtype, forced_splits, precision, dev, sms, 512LL << 20, p,
                                 &ticket_bytes);
    if (st != TSMM_OK) {
        delete p;
        return st;
    }
    cudaError_t e = cudaSuccess;
    if (p->workspace_bytes) e = cudaMalloc(&p->workspace, p->workspace_bytes);
    if (e == cudaSuccess && ticket_bytes) {
        e = cudaMalloc(reinterpret_cast<void **>(&p->tickets), ticket_bytes);
        if (e == cudaSuccess) e = cudaMemset(p->tickets, 0, ticket_bytes);
    }
    if (e == cudaSuccess) {
        e = cudaMalloc(reinterpret_cast<void **>(&p->status), sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(unsigned));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (p->workspace) cudaFree(p->workspace);
        if (p->tickets) cudaFree(p->tickets);
        if (p->status) cudaFree(p->status);
        delete p;
        return cuda_status(e);
    }
    *out = p;
    return TSMM_OK;
}

tsmm_status plan_layout(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype, int forced_splits,
                        int precision, int dev, int sms, int64_t max_workspace, tsmm_plan_s *p,
                        size_t *ticket_bytes_out) {
    if (!valid_dtype(dtype) || m < 0 || n < 0 || k < 0) return TSMM_ERR_INVALID_ARG;
    const int regime = regime_of(k, n);
    if (regime == 0) return TSMM_ERR_UNSUPPORTED_SHAPE;
    std::memset(static_cast<void *>(p), 0, sizeof(*p));
    p->m = m;
    p->n = n;
    p->k = k;
    p->dtype = dtype;
    p->precision = precision;
    p->regime = regime;
    p->device = dev;
    p->num_sms = sms;
    const size_t es = dtype_size(dtype);
    size_t ticket_bytes = 0;
    if (precision == TSMM_PREC_BF16X3 && regime == 2) {
        // 128 x 128 output tiles, k (<= 128) in one or two 64-column chunks
        p->kp = round_up(k, kX3KB);
        p->bm = 128;
        p->np = kX3RankNT;
        p->splits = 1;
        p->mtiles = (m + p->bm - 1) / p->bm;
        p->ntiles = (n + kX3RankNT - 1) / kX3RankNT;
    } else if (precision == TSMM_PREC_BF16X3) {
        // one 128-row slab per block, k in 64-column chunks, one block per SM
        p->np = x3_np(n);
        p->bm = 128;
        p->kp = round_up(k, kX3KB);
        p->slabs = (m + p->bm - 1) / p->bm;
        const int64_t kstages = p->kp / kX3KB;
        const int64_t per_split = (int64_t)p->np * p->slabs * p->bm * (int64_t)es;
        int64_t max_splits = 65535;
        if (per_split > 0) max_splits = std::min<int64_t>(max_splits, max_workspace / per_split);
        int s = (kstages > 0 && p->slabs > 0)
                    ? choose_splits(p->slabs, kstages, sms, max_splits, 1)
                    : 1;
        if (forced_splits > 0)
            s = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)forced_splits, kstages, max_splits}));
        const int64_t chunk_stages = kstages > 0 ? (kstages + s - 1) / s : 1;
        p->kchunk = chunk_stages * kX3KB;
        p->splits = kstages > 0 ? (int)((kstages + chunk_stages - 1) / chunk_stages) : 1;
        if (p->splits > 1) {
            p->workspace_bytes = (size_t)p->splits * (size_t)per_split;
            ticket_bytes = (size_t)p->slabs * sizeof(unsigned);
        }
    } else if (regime == 1) {
        p->np = tall_np(n);
        p->bm = tall_bm(dtype, p->np);
        p->kp = round_up(k, kTallBKS);
        p->slabs = (m + p->bm - 1) / p->bm;
        const int64_t kstages = p->kp / kTallBKS;
        // keep the workspace within max_workspace and the grid's y extent legal
        const int64_t per_split = (int64_t)p->np * p->slabs * p->bm * (int64_t)es;
        int64_t max_splits = 65535;
        if (per_split > 0) max_splits = std::min<int64_t>(max_splits, max_workspace / per_split);
        const int per_sm = tall_resident_blocks(dtype == TSMM_F64, p->np);
        int s = (kstages > 0 && p->slabs > 0)
                    ? choose_splits(p->slabs, kstages, sms, max_splits, per_sm)
                    : 1;
        if (forced_splits > 0)
            s = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)forced_splits, kstages, max_splits}));
        const int64_t chunk_stages = kstages > 0 ? (kstages + s - 1) / s : 1;
        p->kchunk = chunk_stages * kTallBKS;
        p->splits = kstages > 0 ? (int)((kstages + chunk_stages - 1) / chunk_stages) : 1;
        if (p->splits > 1) {
            p->workspace_bytes = (size_t)p->splits * (size_t)per_split;
            ticket_bytes = (size_t)p->slabs * sizeof(unsigned);
        }
    } else {
        p->kp = round_up(k, kRankKGran);
        p->bm = dtype == TSMM_F64 ? 64 : 128;
        p->np = kRankNT;
        p->splits = 1;
        p->mtiles = (m + p->bm - 1) / p->bm;
        p->ntiles = (n + kRankNT - 1) / kRankNT;
    }
    if (ticket_bytes_out) *ticket_bytes_out = ticket_bytes;
    return TSMM_OK;
}

}  // namespace tsmm

extern "C" {

tsmm_status tsmm_plan_destroy(tsmm_plan_t p) {
    if (!p) return TSMM_OK;
    tsmm_status st = TSMM_OK;
    if (p->workspace && cudaFree(p->workspace) != cudaSuccess) st = TSMM_ERR_CUDA;
    if (p->tickets && cudaFree(p->tickets) != cudaSuccess) st = TSMM_ERR_CUDA;
    if (p->status && cudaFree(p->status) != cudaSuccess) st = TSMM_ERR_CUDA;
    delete p;
    return st;
}

tsmm_status tsmm_plan_info(tsmm_plan_t p, int *regime, int *np, int *bm, int *splits,
                           size_t *workspace_bytes) {
    if (!p) return TSMM_ERR_INVALID_ARG;
    if (regime) *regime = p->regime;
    if (np) *np = p->np;
    if (bm) *bm = p->bm;
    if (splits) *splits = p->splits;
    if (workspace_bytes) *workspace_bytes = p->workspace_bytes;
    return TSMM_OK;
}

int tsmm_plan_launches_per_execute(tsmm_plan_t p) {
    if (!p) return 0;
    return (p->m == 0 || p->n == 0) ? 0 : 1;
}

tsmm_status tsmm_execute(tsmm_plan_t p, double alpha, const void *A_dev, int64_t lda,
                         tsmm_packed_b pb, double beta, void *C_dev, int64_t ldc,
                         tsmm_stream_t stream) {
    if (!p || !pb) return TSMM_ERR_INVALID_ARG;
    if (pb->dtype != p->dtype || pb->k != p->k || pb->n != p->n || pb->device != p->device ||
        pb->precision != p->precision)
        return TSMM_ERR_MISMATCH;
    if (current_device() != p->device) return TSMM_ERR_MISMATCH;
    const int64_t m = p->m, n = p->n, k = p->k;
    if (lda < std::max<int64_t>(1, m) || ldc < std::max<int64_t>(1, m)) return TSMM_ERR_INVALID_ARG;
    if (m == 0 || n == 0) return TSMM_OK;
    const bool use_ab = (alpha != 0.0) && (k > 0);
    if (!C_dev || (use_ab && !A_dev)) return TSMM_ERR_INVALID_ARG;
    const size_t es = dtype_size(p->dtype);
    if (!aligned(C_dev, es) || (use_ab && !aligned(A_dev, es))) return TSMM_ERR_MISALIGNED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->dtype == TSMM_F32 && static_cast<float>(alpha) == 0.0f && alpha != 0.0) {
        // alpha underflows to zero in float: behave as alpha == 0
        return cuda_status(launch_scale(p->dtype, m, n, beta, C_dev, ldc, s));
    }
    if (!use_ab) return cuda_status(launch_scale(p->dtype, m, n, beta, C_dev, ldc, s));

    TallArgs a;
    a.m = m;
    a.n = n;
    a.k = k;
    a.lda = lda;
    a.ldc = ldc;
    a.A = A_dev;
    a.Bp = pb->data;
    a.C = C_dev;
    a.alpha = alpha;
    a.beta = beta;
    a.ws = p->workspace;
    a.tickets = p->tickets;
    a.status = p->status;
    a.splits = p->splits;
    a.kchunk = p->kchunk;
    a.kp = p->kp;
    a.slabs = p->slabs;

    const bool tma = aligned(A_dev, 16) && ((lda * (int64_t)es) % 16 == 0) && m < INT_MAX &&
                     k < INT_MAX && (lda * (int64_t)es) < (1LL << 40) && encoder() != nullptr;
    if (tma && (p->tmap_ptr != A_dev || p->tmap_lda != lda)) {
        // box: bm rows x 32 columns (the regime (i) stage and the regime (ii) k chunk)
        const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)k};
        const cuuint64_t gstride[1] = {(cuuint64_t)(lda * (int64_t)es)};
        const cuuint32_t box[2] = {(cuuint32_t)p->bm,
                                   (cuuint32_t)a_box_k(p->dtype, p->regime, p->precision, p->k)};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encoder()(&p->tmap,
                               p->dtype == TSMM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                               2, const_cast<void *>(A_dev), gdim, gstride, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            p->tmap_ptr = nullptr;
            return TSMM_ERR_CUDA;
        }
        p->tmap_ptr = A_dev;
        p->tmap_lda = lda;
    }
    if (p->precision == TSMM_PREC_BF16X3) {
        if (p->regime == 2) {
            RankArgs ra;
            ra.m = m;
            ra.n = n;
            ra.k = k;
            ra.lda = lda;
            ra.ldc = ldc;
            ra.kp = pb->kp;
            ra.A = A_dev;
            ra.Bp = pb->data;
            ra.C = C_dev;
            ra.alpha = alpha;
            ra.beta = beta;
            ra.num_sms = p->num_sms;
            // C0 loads and C stores go through TMA when C allows it (any beta)
            const bool tmc = c_tma_ok(C_dev, ldc, n, es);
            if (tmc) {
                const tsmm_status st = encode_tmapc(p, C_dev, m, n, ldc, es, kX3RankSub);
                if (st != TSMM_OK) return st;
            }
            // an A that a tensor map cannot describe is moved column by column
            return cuda_status(
                launch_rankk_bf16x3(tma ? &p->tmap : nullptr, tmc ? &p->tmapc : nullptr, ra, p->status, s));
        }
        // regime (i): an A that a tensor map cannot describe is moved column by column
        return cuda_status(launch_tall_bf16x3(p->np, tma ? &p->tmap : nullptr, a, p->num_sms, s));
    }
    if (p->regime == 2) {
        RankArgs ra;
        ra.m = m;
        ra.n = n;
        ra.k = k;
        ra.lda = lda;
        ra.ldc = ldc;
        ra.kp = pb->kp;
        ra.A = A_dev;
        ra.Bp = pb->data;
        ra.C = C_dev;
        ra.alpha = alpha;
        ra.beta = beta;
        ra.num_sms = p->num_sms;
        // An A that a tensor map cannot describe is small here (k <= 128 columns
        // against an m x n output): it is copied into an aligned scratch buffer
        // from the stream's memory pool (released on the stream after the
        // kernel) so that the tensor-copy kernels run; only if that allocation
        // fails does the plain-load kernel read it directly.
        void *scratch = nullptr;
        CUtensorMap tm_scratch;
        bool tma_a = tma;
        if (!tma && encoder() != nullptr && m < INT_MAX && k <= 65535) {
            const int64_t v = 16 / (int64_t)es;
            const int64_t ldd = (m + v - 1) / v * v;
            const size_t bytes = (size_t)ldd * (size_t)k * es;
            if (bytes <= (size_t(1) << 32) && cudaMallocAsync(&scratch, bytes, s) == cudaSuccess) {
                const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)k};
                const cuuint64_t gstride[1] = {(cuuint64_t)(ldd * (int64_t)es)};
                const cuuint32_t box[2] = {(cuuint32_t)p->bm,
                                           (cuuint32_t)a_box_k(p->dtype, p->regime, p->precision, p->k)};
                const cuuint32_t estr[2] = {1, 1};
                const cudaError_t ce = launch_copy_columns(p->dtype, A_dev, lda, m, k, scratch, ldd, s);
                if (ce == cudaSuccess &&
                    encoder()(&tm_scratch,
                              p->dtype == TSMM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                              2, scratch, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
                    tma_a = true;
                    ra.A = scratch;
                    ra.lda = ldd;
                } else {
                    cudaFreeAsync(scratch, s);
                    scratch = nullptr;
                    if (ce != cudaSuccess) return cuda_status(ce);
                }
            } else {
                cudaGetLastError();  // no scratch: the plain-load kernel
                scratch = nullptr;
            }
        }
        // C tiles by TMA (C0 prefetch; C0 and C in the FP32 k > 32 kernel): the
        // same 16-byte rules for C
        const bool tmc = tma_a && c_tma_ok(C_dev, ldc, n, es);
        if (tmc) {
            const tsmm_status st = encode_tmapc(p, C_dev, m, n, ldc, es, kRankNT);
            if (st != TSMM_OK) {
                if (scratch) cudaFreeAsync(scratch, s);
                return st;
            }
        }
        const cudaError_t e = launch_rankk(p->dtype, tma_a ? (scratch ? &tm_scratch : &p->tmap) : nullptr,
                                           tmc ? &p->tmapc : nullptr, ra, p->status, s);
        if (scratch) cudaFreeAsync(scratch, s);  // after the kernel, in stream order
        return cuda_status(e);
    }
    cudaError_t e = p->dtype == TSMM_F32 ? launch_tall_f32(tma, p->np, &p->tmap, a, s)
                                         : launch_tall_f64(tma, p->np, &p->tmap, a, s);
    return cuda_status(e);
}

tsmm_status tsmm_plan_check(tsmm_plan_t p) {
    if (!p) return TSMM_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return TSMM_ERR_CUDA;
    unsigned word = 0;
    if (cudaMemcpy(&word, p->status, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TSMM_ERR_CUDA;
    if (word == 0) return TSMM_OK;
    // clear the record and the split-K arrival counters a failed launch may have left
    cudaMemset(p->status, 0, sizeof(unsigned));
    if (p->tickets) cudaMemset(p->tickets, 0, (size_t)p->slabs * sizeof(unsigned));
    cudaDeviceSynchronize();
    return (word & kDevErrTimeout) ? TSMM_ERR_TIMEOUT : TSMM_ERR_CUDA;
}

}  // extern "C"
