// Grouped regime (i) kernel: many TSMMs C_i = alpha_i A_i B_i + beta_i C_i with
// the same padded column count NP (n_i <= NP) in one launch.
//
// Each problem contributes slabs_i x splits_i work items (an m-slab and a k
// range, exactly the blocks of the single-problem kernel), and the launch has
// one block per item running the single-problem kernel's block body: the GPU's
// block scheduler hands SMs to items of unequal cost as earlier ones finish,
// and the last wave of one problem overlaps the first of the next, which
// back-to-back single launches on one stream cannot do.  The per-problem
// descriptors, each with its own tensor map for A, travel in the kernel's
// parameter block.  Split-K partials are finished by the last-arriving block
// per slab, as in the single-problem kernel, using each problem's own plan
// workspace; the results are the single launches' bit for bit.
//
// U = true: problems whose A a tensor map cannot describe (base or column
// stride not a multiple of 16 bytes) run the bulk/element-copy block body, in
// its load form LV (async_load_variant: the same for every problem of the
// launch).
#pragma once
#include <climits>
#include "tsmm_tall.cuh"

namespace tsmm {

constexpr int kGroupMax = 48;  // problems per launch (parameter block < 32 KB)

struct alignas(128) GroupProblem {
    CUtensorMap tmA;
    TallArgs a;
    int64_t item_begin;  // first global work item of this problem
};

struct GroupParams {
    GroupProblem p[kGroupMax];
    int count;
    int64_t total_items;  // <= INT_MAX: one block per item
};

// Problem holding global item `item` (linear scan: at most kGroupMax problems).
__device__ __forceinline__ int group_find(const GroupParams &gp, int64_t item) {
    int p = 0;
    while (p + 1 < gp.count && gp.p[p + 1].item_begin <= item) ++p;
    return p;
}

template <typename T, int NP, bool U, int LV>
__global__ void __launch_bounds__(TallCfg<T, NP>::THREADS, TallCfg<T, NP>::RESIDENT)
    tall_grouped_kernel(const __grid_constant__ GroupParams gp) {
    const int64_t item = blockIdx.x;
    const int p = group_find(gp, item);
    const TallArgs &a = gp.p[p].a;
    int64_t slab, split;
    udivmod(item - gp.p[p].item_begin, a.splits, slab, split);
    if constexpr (U)
        tall_async_block<T, NP, LV>(a, slab, (int)split);
    else
        tall_tma_block<T, NP>(&gp.p[p].tmA, a, slab, (int)split);
}

template <typename T, int NP, bool U, int LV>
cudaError_t launch_grouped_t(const GroupParams &gp, cudaStream_t s) {
    const int smem = U ? AsyncCfg<T, NP>::SMEM : TallCfg<T, NP>::SMEM;
    {
        const cudaError_t e =
            ensure_smem_limit(reinterpret_cast<const void *>(tall_grouped_kernel<T, NP, U, LV>), smem);
        if (e != cudaSuccess) return e;
    }
    if (gp.total_items <= 0) return cudaSuccess;
    if (gp.total_items > INT_MAX) return cudaErrorInvalidValue;
    tall_grouped_kernel<T, NP, U, LV><<<(unsigned)gp.total_items, TallCfg<T, NP>::THREADS, smem, s>>>(gp);
    return cudaGetLastError();
}

// Per-width dispatch of the grouped kernel: tensor-map A (tsmm_group_<dtype>.cu)
// and, in its load form lv, an A that a tensor map cannot describe
// (tsmm_group_async_<dtype>.cu), in translation units of their own.
template <typename T>
cudaError_t launch_grouped_tma_dispatch(int np, const GroupParams &gp, cudaStream_t s) {
#define TSMM_GROUP_CASE(NPV) \
    case NPV:                \
        return launch_grouped_t<T, NPV, false, -1>(gp, s);
    switch (np) {
        TSMM_FOR_TALL_WIDTHS(TSMM_GROUP_CASE)
        default:
            return cudaErrorInvalidValue;
    }
#undef TSMM_GROUP_CASE
}

template <typename T, int NP>
cudaError_t launch_grouped_async_np(int lv, const GroupParams &gp, cudaStream_t s) {
    return with_load_variant<T, NP>(lv, [&](auto lv_tag) {
        return launch_grouped_t<T, NP, true, decltype(lv_tag)::value>(gp, s);
    });
}

template <typename T>
cudaError_t launch_grouped_async_dispatch(int np, int lv, const GroupParams &gp, cudaStream_t s) {
#define TSMM_GROUP_CASE(NPV) \
    case NPV:                \
        return launch_grouped_async_np<T, NPV>(lv, gp, s);
    switch (np) {
        TSMM_FOR_TALL_WIDTHS(TSMM_GROUP_CASE)
        default:
            return cudaErrorInvalidValue;
    }
#undef TSMM_GROUP_CASE
}

cudaError_t launch_grouped_async_f32(int np, int lv, const GroupParams &gp, cudaStream_t s);
cudaError_t launch_grouped_async_f64(int np, int lv, const GroupParams &gp, cudaStream_t s);

}  // namespace tsmm
