// Grouped persistent regime (i) kernel: many TSMMs C_i = alpha_i A_i B_i +
// beta_i C_i with the same padded column count NP (n_i <= NP) in one launch.
//
// Each problem contributes slabs_i x splits_i work items (an m-slab and a k
// range, exactly the blocks of the single-problem kernel).  A grid of
// RESIDENT x SM-count persistent blocks walks the items
// blockIdx.x, blockIdx.x + gridDim.x, ...; the producer warp keeps its TMA ring
// running across item boundaries, so the next item's A tiles stream in while
// the consumers reduce and store the current one (the reduction uses its own
// shared-memory buffer for that reason).  The per-problem descriptors, each
// with its own tensor map for A, travel in the kernel's parameter block.
// Split-K partials are finished by the last-arriving block per slab, as in
// the single-problem kernel, using each problem's own plan workspace.
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
    int64_t total_items;
};

template <typename T, int NP>
struct GroupCfg {
    using Tc = TallCfg<T, NP>;
    static constexpr int RED_BYTES = Tc::RED * (int)sizeof(T);
    // three blocks per SM where two ring stages and the reduction buffer fit in
    // a third of the SM's shared memory and the width's tiles fit its registers
    // (more warps to hide shared-memory latency), else two with a deeper ring
    static constexpr bool THREE = tall_resident_blocks(sizeof(T) == 8, NP) == 3 &&
                                  2 * Tc::STAGE_BYTES + RED_BYTES <= 72 * 1024;
    static constexpr int RESIDENT = THREE ? 3 : 2;
    static constexpr int RING_BUDGET = (THREE ? 72 : 100) * 1024 - RED_BYTES;
    static constexpr int STAGES_RAW = RING_BUDGET / Tc::STAGE_BYTES;
    static constexpr int STAGES = STAGES_RAW < 2 ? 2 : (STAGES_RAW > 6 ? 6 : STAGES_RAW);
    static constexpr int RING_BYTES = STAGES * Tc::STAGE_BYTES;
    static constexpr int SMEM = RING_BYTES + RED_BYTES + 2 * STAGES * 8 + 16;
};

// Problem holding global item `item` (linear scan: at most kGroupMax problems).
__device__ __forceinline__ int group_find(const GroupParams &gp, int64_t item) {
    int p = 0;
    while (p + 1 < gp.count && gp.p[p + 1].item_begin <= item) ++p;
    return p;
}

template <typename T, int NP>
__global__ void __launch_bounds__(TallCfg<T, NP>::THREADS, GroupCfg<T, NP>::RESIDENT)
    tall_grouped_kernel(const __grid_constant__ GroupParams gp) {
    using Cfg = TallCfg<T, NP>;
    using GC = GroupCfg<T, NP>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sA = reinterpret_cast<T *>(smem_raw);
    T *sB = sA + GC::STAGES * Cfg::A_STAGE;
    T *red = reinterpret_cast<T *>(smem_raw + GC::RING_BYTES);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + GC::RING_BYTES + GC::RED_BYTES);
    uint64_t *empty = full + GC::STAGES;
    unsigned *flag = reinterpret_cast<unsigned *>(empty + GC::STAGES);
    unsigned *abort_flag = flag + 1;

    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        for (int s = 0; s < GC::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], Cfg::NWARPS);
        }
        *abort_flag = 0u;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == Cfg::NWARPS) {
        if (lane == 0) {
            const uint64_t pol_a = policy_evict_first();
            const uint64_t pol_b = policy_evict_last();
            int64_t g = 0;  // stages issued by this block, across items
            bool ok = true;
            for (int64_t item = blockIdx.x; item < gp.total_items && ok; item += gridDim.x) {
                const int p = group_find(gp, item);
                const TallArgs &a = gp.p[p].a;
                const int64_t local = item - gp.p[p].item_begin;
                int64_t slab, sp;
                udivmod(local, a.splits, slab, sp);
                const int64_t k0 = sp * a.kchunk;
                const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;
                const T *Bp = static_cast<const T *>(a.Bp);
                for (int64_t kk = k0; kk < k1; kk += Cfg::BKS, ++g) {
                    const int st = (int)(g % GC::STAGES);
                    if (g >= GC::STAGES &&
                        !mbar_wait_bounded(&empty[st], (int)((g / GC::STAGES) & 1) ^ 1)) {
                        atomicOr(a.status, kDevErrTimeout);
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], Cfg::STAGE_BYTES);
                    tma_load_2d(sA + st * Cfg::A_STAGE, &gp.p[p].tmA, (int32_t)(slab * Cfg::BM),
                                (int32_t)kk, &full[st], pol_a);
                    bulk_load(sB + st * Cfg::B_STAGE, Bp + kk * NP, Cfg::B_STAGE * (int)sizeof(T),
                              &full[st], pol_b);
                }
            }
        }
        return;
    }

    const int wm = warp % Cfg::WM;
    const int wk = warp / Cfg::WM;
    const int gl = lane / Cfg::LR;
    const int lr = lane % Cfg::LR;
    const int rloc = wm * Cfg::WROWS + lr * Cfg::RV;
    const int cloc = gl * Cfg::CN;
    int64_t g = 0;
    for (int64_t item = blockIdx.x; item < gp.total_items; item += gridDim.x) {
        const int p = group_find(gp, item);
        const TallArgs &a = gp.p[p].a;
        const int64_t local = item - gp.p[p].item_begin;
        int64_t slab, sp64;
        udivmod(local, a.splits, slab, sp64);
        const int split = (int)sp64;
        const int64_t k0 = (int64_t)split * a.kchunk;
        const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;

        typename TallAcc<T, NP>::type acc;
        acc.zero();
        bool ok = true;
        for (int64_t kk = k0; kk < k1; kk += Cfg::BKS, ++g) {
            const int st = (int)(g % GC::STAGES);
            if (!mbar_wait_bounded(&full[st], (int)((g / GC::STAGES) & 1))) {
                ok = false;
                break;
            }
            const T *As = sA + st * Cfg::A_STAGE;
            const T *Bs = sB + st * Cfg::B_STAGE;
#pragma unroll
            for (int c = 0; c < Cfg::KPW; ++c) {
                const int col = wk * Cfg::KPW + c;
                const Vec<T, Cfg::R> av = tall_load_rows<Cfg, T>(As + col * Cfg::BM, rloc);
                acc.fma_column(av, Bs + col * NP + cloc);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
        if (!ok && lane == 0) {
            atomicOr(a.status, kDevErrTimeout);
            atomicOr(abort_flag, 1u);
        }
        // every consumer has finished the previous item's reduction and read
        // its flags before `red` is written again
        named_barrier(1, Cfg::CONSUMERS);
        if (*abort_flag != 0u) return;
#pragma unroll
        for (int c = 0; c < Cfg::CN; ++c) {
            Vec<T, Cfg::R> v;
#pragma unroll
            for (int r = 0; r < Cfg::R; ++r) v.v[r] = acc.get(r, c);
            tall_store_rows<Cfg, T>(red + (wk * NP + cloc + c) * Cfg::BM, rloc, v);
        }
        named_barrier(1, Cfg::CONSUMERS);
        tall_finish<T, NP>(red, a, slab, split, threadIdx.x, flag);
    }
}

// persistent: RESIDENT blocks per SM loop over the items; otherwise one block
// per item, so that blocks of higher-priority streams get SMs as items finish.
template <typename T, int NP>
cudaError_t launch_grouped_t(const GroupParams &gp, int num_sms, bool persistent, cudaStream_t s) {
    using GC = GroupCfg<T, NP>;
    {
        const cudaError_t e =
            ensure_smem_limit(reinterpret_cast<const void *>(tall_grouped_kernel<T, NP>), GC::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t slots = persistent ? (int64_t)GC::RESIDENT * (num_sms > 0 ? num_sms : 1) : INT_MAX;
    const unsigned grid = (unsigned)(gp.total_items < slots ? gp.total_items : slots);
    if (grid == 0) return cudaSuccess;
    tall_grouped_kernel<T, NP><<<grid, TallCfg<T, NP>::THREADS, GC::SMEM, s>>>(gp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grouped_dispatch(int np, const GroupParams &gp, int num_sms, bool persistent,
                                    cudaStream_t s) {
    switch (np) {
        case 1: return launch_grouped_t<T, 1>(gp, num_sms, persistent, s);
        case 2: return launch_grouped_t<T, 2>(gp, num_sms, persistent, s);
        case 4: return launch_grouped_t<T, 4>(gp, num_sms, persistent, s);
        case 8: return launch_grouped_t<T, 8>(gp, num_sms, persistent, s);
        case 16: return launch_grouped_t<T, 16>(gp, num_sms, persistent, s);
        case 24: return launch_grouped_t<T, 24>(gp, num_sms, persistent, s);
        case 32: return launch_grouped_t<T, 32>(gp, num_sms, persistent, s);
        case 48: return launch_grouped_t<T, 48>(gp, num_sms, persistent, s);
        case 64: return launch_grouped_t<T, 64>(gp, num_sms, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tsmm
