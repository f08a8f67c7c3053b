// tsmm_execute_grouped: many pre-packed TSMMs in as few launches as possible.
// Regime (i) problems are batched, per dtype, padded column count and kind of
// A (one a tensor map can describe, or one whose base or column stride is not
// a multiple of 16 bytes, and then its load form), into launches of the
// grouped kernel (up to
// kGroupMax problems and INT_MAX work items each, one block per item); every
// other problem (regime (ii), alpha = 0, k = 0, the BF16x3 mode) is executed by
// its own tsmm_execute launch on the same stream.
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <map>
#include <memory>
#include <set>
#include <tuple>
#include <utility>
#include <vector>

#include "tsmm_group.cuh"

namespace tsmm {
cudaError_t launch_grouped_f32(int np, bool unaligned, int lv, const GroupParams &gp, cudaStream_t s);
cudaError_t launch_grouped_f64(int np, bool unaligned, int lv, const GroupParams &gp, cudaStream_t s);
}  // namespace tsmm

using namespace tsmm;

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder_grouped() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

bool is_aligned(const void *p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

// Same argument rules as tsmm_execute.
tsmm_status validate(const tsmm_group_item &it) {
    tsmm_plan_t p = it.plan;
    tsmm_packed_b pb = it.pb;
    if (!p || !pb) return TSMM_ERR_INVALID_ARG;
    if (pb->dtype != p->dtype || pb->k != p->k || pb->n != p->n || pb->device != p->device ||
        pb->precision != p->precision)
        return TSMM_ERR_MISMATCH;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSMM_ERR_CUDA;
    if (dev != p->device) return TSMM_ERR_MISMATCH;
    if (it.lda < std::max<int64_t>(1, p->m) || it.ldc < std::max<int64_t>(1, p->m))
        return TSMM_ERR_INVALID_ARG;
    if (p->m == 0 || p->n == 0) return TSMM_OK;
    const bool use_ab = it.alpha != 0.0 && p->k > 0;
    if (!it.C_dev || (use_ab && !it.A_dev)) return TSMM_ERR_INVALID_ARG;
    const size_t es = dtype_size(p->dtype);
    if (!is_aligned(it.C_dev, es) || (use_ab && !is_aligned(it.A_dev, es))) return TSMM_ERR_MISALIGNED;
    return TSMM_OK;
}

// 0: not groupable (its own tsmm_execute launch); 1: A described by a tensor
// map; 2: A whose base or column stride is not 16-byte aligned (each column
// moved by one bulk copy of the 16-byte-aligned span around its rows).
int group_kind(const tsmm_group_item &it) {
    tsmm_plan_t p = it.plan;
    const size_t es = dtype_size(p->dtype);
    const bool alpha_zero = it.alpha == 0.0 ||
                            (p->dtype == TSMM_F32 && static_cast<float>(it.alpha) == 0.0f);
    if (!(p->regime == 1 && p->precision == TSMM_PREC_NATIVE && p->m > 0 && p->n > 0 && p->k > 0 && !alpha_zero &&
          p->m < INT_MAX && p->k < INT_MAX && p->slabs * (int64_t)p->splits < INT_MAX))
        return 0;
    const bool tma = is_aligned(it.A_dev, 16) && (it.lda * (int64_t)es) % 16 == 0 &&
                     (it.lda * (int64_t)es) < (1LL << 40) && encoder_grouped() != nullptr;
    return tma ? 1 : 2;
}

}  // namespace

tsmm_status tsmm::execute_grouped(const tsmm_group_item *items, int count, tsmm_stream_t stream) {
    if (count < 0 || (count > 0 && !items)) return TSMM_ERR_INVALID_ARG;
    std::set<tsmm_plan_t> seen;
    for (int i = 0; i < count; ++i) {
        tsmm_status st = validate(items[i]);
        if (st != TSMM_OK) return st;
        if (!seen.insert(items[i].plan).second) return TSMM_ERR_INVALID_ARG;  // shared workspace
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // classes of groupable problems: (dtype, np, kind of A, load form) -> item indices
    std::map<std::tuple<int, int, int, int>, std::vector<int>> classes;
    for (int i = 0; i < count; ++i) {
        const int kind = group_kind(items[i]);
        if (kind != 0) {
            const tsmm_plan_t p = items[i].plan;
            const int lv = kind == 2 ? async_load_variant(p->dtype == TSMM_F32, p->np, items[i].A_dev, items[i].lda)
                                     : -1;
            classes[std::make_tuple((int)p->dtype, p->np, kind, lv)].push_back(i);
        } else {
            tsmm_status st = tsmm_execute(items[i].plan, items[i].alpha, items[i].A_dev, items[i].lda,
                                          items[i].pb, items[i].beta, items[i].C_dev, items[i].ldc,
                                          stream);
            if (st != TSMM_OK) return st;
        }
    }
    std::unique_ptr<GroupParams> gp(new (std::nothrow) GroupParams());
    if (!gp) return TSMM_ERR_OUT_OF_MEMORY;
    for (auto &cls : classes) {
        const tsmm_dtype dt = (tsmm_dtype)std::get<0>(cls.first);
        const int np = std::get<1>(cls.first);
        const bool unaligned = std::get<2>(cls.first) == 2;
        const int lv = std::get<3>(cls.first);
        const std::vector<int> &idx = cls.second;
        // launches of at most kGroupMax problems and INT_MAX work items
        size_t q = 0;
        while (q < idx.size()) {
            int64_t total = 0;
            gp->count = 0;
            for (; q < idx.size() && gp->count < kGroupMax; ++q) {
                const tsmm_group_item &it = items[idx[q]];
                tsmm_plan_t p = it.plan;
                const int64_t n_items = p->slabs * (int64_t)p->splits;
                if (total + n_items > INT_MAX) break;  // n_items < INT_MAX: the next launch takes it
                GroupProblem &g = gp->p[gp->count++];
                const size_t es = dtype_size(dt);
                const cuuint64_t gdim[2] = {(cuuint64_t)p->m, (cuuint64_t)p->k};
                const cuuint64_t gstride[1] = {(cuuint64_t)(it.lda * (int64_t)es)};
                const cuuint32_t box[2] = {(cuuint32_t)p->bm, (cuuint32_t)kTallBKS};
                const cuuint32_t estr[2] = {1, 1};
                if (!unaligned && encoder_grouped()(&g.tmA,
                                      dt == TSMM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                      2, const_cast<void *>(it.A_dev), gdim, gstride, box, estr,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                    return TSMM_ERR_CUDA;
                TallArgs &a = g.a;
                a.m = p->m;
                a.n = p->n;
                a.k = p->k;
                a.lda = it.lda;
                a.ldc = it.ldc;
                a.A = it.A_dev;
                a.Bp = it.pb->data;
                a.C = it.C_dev;
                a.alpha = it.alpha;
                a.beta = it.beta;
                a.ws = p->workspace;
                a.tickets = p->tickets;
                a.status = p->status;
                a.splits = p->splits;
                a.kchunk = p->kchunk;
                a.kp = p->kp;
                a.slabs = p->slabs;
                g.item_begin = total;
                total += n_items;
            }
            gp->total_items = total;
            cudaError_t e = dt == TSMM_F32 ? launch_grouped_f32(np, unaligned, lv, *gp, s)
                                           : launch_grouped_f64(np, unaligned, lv, *gp, s);
            if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TSMM_ERR_OUT_OF_MEMORY : TSMM_ERR_CUDA;
        }
    }
    return TSMM_OK;
}

extern "C" tsmm_status tsmm_execute_grouped(const tsmm_group_item *items, int count,
                                            tsmm_stream_t stream) {
    return tsmm::execute_grouped(items, count, stream);
}
