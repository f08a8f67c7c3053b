// FP32 TSMM on the tensor cores from three BF16 products (precision mode
// TSMM_PREC_BF16X3), regime (i): C[m x n] = alpha*A*B + beta*C0, n <= 64.
//
// Each FP32 value x is split into x_hi = bf16(x) and x_lo = bf16(x - x_hi); the
// product A*B is accumulated in FP32 (tensor memory) as
//     A_hi*B_hi + A_hi*B_lo + A_lo*B_hi
// dropping only A_lo*B_lo and the residues of the splits (about 3*2^-16
// relative to |A||B| per product).  This mode exists for the FP32 shapes the
// FMA pipes cannot stream at HBM speed (n >= 32); it is not bit-compatible with
// the FP32 FMA path, and its bound is stated separately.
//
// Work item = one m-slab of 128 rows x one k range (the same split-K scheme as
// the FMA kernel); persistent blocks of 10 warps:
//   warp 4      producer: TMA copies of FP32 A tiles (128 rows x 64 columns)
//               and bulk copies of the pre-split B chunks (hi|lo, K-major);
//   warps 0-3   converters: read a stage's FP32 A rows into registers, then
//               overwrite the same 32 KB with the hi and lo BF16 tiles in the
//               K-major canonical UMMA layout (no second buffer, and no wait
//               on earlier MMAs);
//   warp 5      allocates tensor memory; lane 0 issues tcgen05.mma
//               (M = 128, N = NP, K = 16 per instruction, 3 per k-step) into
//               one of two accumulators and commits completions to mbarriers;
//   warps 6-9   epilogue: each thread owns one accumulator row (TMEM lane),
//               reads it with tcgen05.ld, releases the accumulator, and
//               stores alpha*acc + beta*C0 (or the split-K partial).
// Shared-memory operand layout (K-major, no swizzle): element (row, k) of a
// 64-column chunk sits at (row/8)*1024 + (k/8)*128 + (row%8)*16 + (k%8)*2
// bytes, i.e. 8x8 core matrices of 128 B, adjacent along k (LBO = 128 B) and
// 1 KB apart along rows (SBO = 1024 B).
#include <cuda_bf16.h>

#include "tsmm_device.cuh"
#include "tsmm_internal.h"

namespace tsmm {

namespace {

constexpr int kKB = kX3KB; // k per chunk (64: two 16 KB TMA boxes of FP32 A)
constexpr int kBM = 128;    // rows per block = MMA M = TMEM lanes
constexpr int kS = 4;       // stages: FP32 A arrives, is split in place into hi|lo BF16, is read by the MMAs
constexpr int kLBO = 128;
constexpr int kSBO = kKB / 8 * 128;  // 1024 B: one row group of kKB/8 core matrices

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(kLBO >> 4) << 16;
    d |= (uint64_t)(kSBO >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // no swizzle, base offset 0
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *out) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
        " [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ int kmaj_off(int row, int k) {
    return (row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2;
}

template <int NP>
struct X3Cfg {
    static constexpr int A_BYTES = kBM * kKB * 4;          // 32 KB: FP32 in, then BF16 hi | lo
    static constexpr int B_BYTES = 2 * NP * kKB * 2;       // hi + lo chunk
    static constexpr int OFF_B = kS * A_BYTES;
    static constexpr int OFF_BAR = OFF_B + kS * B_BYTES;
    static constexpr int NBAR = 3 * kS + 4 + 1;
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 32;
    static constexpr int TMEM_COLS = 2 * NP < 32 ? 32 : 2 * NP;  // double-buffered accumulator
    static constexpr int THREADS = 320;
};

}  // namespace

// Pack B (k x n, column-major) for the BF16x3 kernels: the columns are cut
// into `ntiles` tiles of NP columns (one tile for regime (i)); per tile and per
// 64-row chunk c of k, a hi tile then a lo tile, each NP rows (columns of B) x
// 64 k in the K-major layout above; zero outside the k x n matrix.
__global__ void pack_b_bf16x3_kernel(const float *__restrict__ B, int64_t k, int64_t n, int64_t ldb,
                                     unsigned char *__restrict__ dst, int np, int64_t nchunks,
                                     int64_t ntiles) {
    const int64_t per_tile = nchunks * np * kKB;
    const int64_t total = ntiles * per_tile;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / per_tile;
        const int64_t et = e - t * per_tile;
        const int64_t c = et / (np * kKB);
        const int rem = (int)(et - c * np * kKB);
        const int j = rem / kKB;
        const int kk = rem % kKB;
        const int64_t p = c * kKB + kk;
        const int64_t col = t * np + j;
        const float x = (p < k && col < n) ? B[p + col * ldb] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        unsigned char *chunk = dst + (t * nchunks + c) * (int64_t)(2 * np * kKB * 2);
        *reinterpret_cast<__nv_bfloat16 *>(chunk + kmaj_off(j, kk)) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(chunk + np * kKB * 2 + kmaj_off(j, kk)) = lo;
    }
}

// Persistent: a grid of one block per SM walks the work items (m-slab, k
// split) blockIdx.x, blockIdx.x + gridDim.x, ...  The accumulator is double
// buffered in tensor memory (2 x NP columns) and read out by four dedicated
// epilogue warps, so the MMAs of the next item run while the previous item's
// results are stored; the producer and converter rings run across items.
template <int NP>
__global__ void __launch_bounds__(320, 1)
    tall_bf16x3_kernel(const __grid_constant__ CUtensorMap tmA, const TallArgs a) {
    using Cfg = X3Cfg<NP>;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + Cfg::OFF_BAR);
    uint64_t *full = bar;             // [kS] FP32 A + B chunk landed
    uint64_t *conv = full + kS;       // [kS] hi|lo written (4 converter warps)
    uint64_t *empty = conv + kS;      // [kS] the MMAs reading the stage are done
    uint64_t *tfull = empty + kS;     // [2] accumulator ready
    uint64_t *tempty = tfull + 2;     // [2] accumulator drained
    uint64_t *done = tempty + 2;      // every issued MMA complete
    unsigned *tslot = reinterpret_cast<unsigned *>(done + 1);
    unsigned *flag = tslot + 1;
    unsigned *abort_flag = tslot + 2;
    unsigned *ep_abort = tslot + 3;    // written and read by the epilogue warps only
    unsigned *conv_abort = tslot + 4;  // written and read by the converter warps only

    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int64_t total = a.slabs * a.splits;

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmA);
        for (int s = 0; s < kS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], 4);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(done, 1);
        *abort_flag = 0u;
        *ep_abort = 0u;
        *conv_abort = 0u;
        fence_mbar_init();
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tslot)),
                     "r"((uint32_t)Cfg::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 4) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            const uint64_t pol_a = policy_evict_first();
            const uint64_t pol_b = policy_evict_last();
            const unsigned char *Bp = static_cast<const unsigned char *>(a.Bp);
            int64_t g = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x) {
                const int64_t slab = item / a.splits;
                const int64_t k0 = (item % a.splits) * a.kchunk;
                const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;
                for (int64_t kk = k0; kk < k1; kk += kKB, ++g) {
                    const int s = (int)(g % kS);
                    if (g >= kS && !mbar_wait_bounded(&empty[s], (uint32_t)((g / kS) & 1) ^ 1)) {
                        atomicOr(a.status, kDevErrTimeout);
                        ok = false;
                        break;
                    }
                    float *dstA = reinterpret_cast<float *>(smem + s * Cfg::A_BYTES);
                    mbar_arrive_expect_tx(&full[s], Cfg::A_BYTES + Cfg::B_BYTES);
                    tma_load_2d(dstA, &tmA, (int32_t)(slab * kBM), (int32_t)kk, &full[s], pol_a);
                    tma_load_2d(dstA + kBM * 32, &tmA, (int32_t)(slab * kBM), (int32_t)(kk + 32),
                                &full[s], pol_a);
                    bulk_load(smem + Cfg::OFF_B + s * Cfg::B_BYTES, Bp + (kk / kKB) * Cfg::B_BYTES,
                              Cfg::B_BYTES, &full[s], pol_b);
                }
            }
        }
        return;
    }

    if (warp == 5) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc(kBM, NP);
            int64_t g = 0;
            int j = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x, ++j) {
                const int b = j & 1;
                if (j >= 2 && !mbar_wait_bounded(&tempty[b], (uint32_t)((j >> 1) & 1) ^ 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tacc = tmem + (uint32_t)(b * NP);
                const int64_t k0 = (item % a.splits) * a.kchunk;
                const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;
                bool first = true;
                for (int64_t kk = k0; kk < k1; kk += kKB, ++g) {
                    const int s = (int)(g % kS);
                    if (!mbar_wait_bounded(&conv[s], (uint32_t)((g / kS) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ahi = smem_addr(smem + s * Cfg::A_BYTES);
                    const uint32_t alo = ahi + kBM * kKB * 2;
                    const uint32_t bhi = smem_addr(smem + Cfg::OFF_B + s * Cfg::B_BYTES);
                    const uint32_t blo = bhi + NP * kKB * 2;
#pragma unroll
                    for (int ks = 0; ks < kKB / 16; ++ks) {
                        const uint32_t off = ks * 2 * kLBO;  // 16 k = two core matrices
                        umma_bf16(tacc, umma_desc(ahi + off), umma_desc(bhi + off), idesc,
                                  first ? 0u : 1u);
                        umma_bf16(tacc, umma_desc(ahi + off), umma_desc(blo + off), idesc, 1u);
                        umma_bf16(tacc, umma_desc(alo + off), umma_desc(bhi + off), idesc, 1u);
                        first = false;
                    }
                    umma_commit(&empty[s]);  // the stage may be refilled once these finish
                }
                if (ok) umma_commit(&tfull[b]);
            }
            umma_commit(done);
            if (!ok) {
                atomicOr(a.status, kDevErrTimeout);
                atomicOr(abort_flag, 1u);
            }
            mbar_wait_bounded(done, 0);  // nothing may still write TMEM when it is freed
        }
        __syncwarp();
        tc_fence_before();
        named_barrier(2, 160);  // warps 5..9: the epilogue has read its last accumulator
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)Cfg::TMEM_COLS));
        return;
    }

    if (warp < 4) {
        // ------------------------------------------------ converters
        const int r = threadIdx.x;  // row within the slab
        int64_t g = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x) {
            const int64_t k0 = (item % a.splits) * a.kchunk;
            const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;
            for (int64_t kk = k0; kk < k1; kk += kKB, ++g) {
                const int s = (int)(g % kS);
                const bool got = mbar_wait_bounded(&full[s], (uint32_t)((g / kS) & 1));
                unsigned char *stage = smem + s * Cfg::A_BYTES;
                const float *src = reinterpret_cast<const float *>(stage);  // [64][128] FP32
                float x[kKB];
                if (got) {
#pragma unroll
                    for (int q = 0; q < kKB; ++q) x[q] = src[q * kBM + r];
                } else if (lane == 0) {
                    atomicOr(conv_abort, 1u);
                }
                // every converter has read the whole stage before any of it is
                // overwritten; the give-up decision is read between two barriers
                // so all four warps take it together
                named_barrier(1, 128);
                const bool stop = *conv_abort != 0u;
                named_barrier(1, 128);
                if (stop) {
                    ok = false;
                    break;
                }
                unsigned char *hi = stage;
                unsigned char *lo = stage + kBM * kKB * 2;
#pragma unroll
                for (int kg = 0; kg < kKB / 8; ++kg) {
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float x0 = x[kg * 8 + 2 * q];
                        const float x1 = x[kg * 8 + 2 * q + 1];
                        const __nv_bfloat162 hv = __floats2bfloat162_rn(x0, x1);
                        const float2 hf = __bfloat1622float2(hv);
                        const __nv_bfloat162 lv = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
                        h[q] = *reinterpret_cast<const uint32_t *>(&hv);
                        l[q] = *reinterpret_cast<const uint32_t *>(&lv);
                    }
                    const int off = kmaj_off(r, kg * 8);
                    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
                fence_proxy_async_smem();  // generic-proxy writes -> tensor-core reads
                __syncwarp();
                if (lane == 0) mbar_arrive(&conv[s]);
            }
        }
        if (!ok && lane == 0) {
            atomicOr(a.status, kDevErrTimeout);
            atomicOr(abort_flag, 1u);
        }
        return;
    }

    // ---------------------------------------------------- epilogue (warps 6-9)
    const int quarter = warp % 4;               // TMEM lanes 32*quarter .. +31
    const int r = quarter * 32 + lane;          // row within the slab
    const int et = (warp - 6) * 32 + lane;      // 0..127 among the epilogue threads
    const float alpha = static_cast<float>(a.alpha);
    const float beta = static_cast<float>(a.beta);
    float *C = static_cast<float *>(a.C);
    float *ws = static_cast<float *>(a.ws);
    const int64_t mpad = a.slabs * kBM;
    int j = 0;
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x, ++j) {
        const int b = j & 1;
        const bool got = mbar_wait_bounded(&tfull[b], (uint32_t)((j >> 1) & 1));
        if (!got && lane == 0) atomicOr(ep_abort, 1u);
        named_barrier(3, 128);
        const bool stop = *ep_abort != 0u;
        named_barrier(3, 128);  // every epilogue thread has read ep_abort: the choice is uniform
        if (stop) {
            if (et == 0) atomicOr(a.status, kDevErrTimeout);
            break;
        }
        tc_fence_after();
        float acc[NP];
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 16)
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * NP + c0), acc + c0);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);  // the MMAs may reuse this accumulator

        const int64_t slab = item / a.splits;
        const int split = (int)(item % a.splits);
        const int64_t i = slab * kBM + r;
        auto store = [&](int jj, float v) {
            if (i < a.m && jj < a.n) {
                float o = (alpha == 1.f) ? v : alpha * v;
                float *cp = C + i + (int64_t)jj * a.ldc;
                if (beta != 0.f) o = fmaf(beta, *cp, o);
                *cp = o;
            }
        };
        if (a.splits == 1) {
#pragma unroll
            for (int jj = 0; jj < NP; ++jj) store(jj, acc[jj]);
            continue;
        }
#pragma unroll
        for (int jj = 0; jj < NP; ++jj) ws[((int64_t)split * NP + jj) * mpad + slab * kBM + r] = acc[jj];
        __threadfence();
        named_barrier(3, 128);
        if (et == 0) {
            const unsigned ticket = atomicAdd(a.tickets + slab, 1u);
            *flag = (ticket == (unsigned)(a.splits - 1)) ? 1u : 0u;
        }
        named_barrier(3, 128);
        if (*flag == 0u) continue;
        __threadfence();
#pragma unroll
        for (int jj = 0; jj < NP; ++jj) {
            float sum = 0.f;
            for (int sp = 0; sp < a.splits; ++sp)
                sum += (sp == split) ? acc[jj]
                                     : ld_cg(ws + ((int64_t)sp * NP + jj) * mpad + slab * kBM + r);
            store(jj, sum);
        }
        if (et == 0) a.tickets[slab] = 0u;
    }
    tc_fence_before();
    named_barrier(2, 160);  // with warp 5, before it frees TMEM
}

template <int NP>
static cudaError_t launch_x3_t(const CUtensorMap *tmap, const TallArgs &a, int num_sms, cudaStream_t s) {
    using Cfg = X3Cfg<NP>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(tall_bf16x3_kernel<NP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const int64_t items = a.slabs * a.splits;
    const int64_t slots = num_sms > 0 ? num_sms : 1;
    const unsigned grid = (unsigned)(items < slots ? items : slots);
    if (grid == 0) return cudaSuccess;
    tall_bf16x3_kernel<NP><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(*tmap, a);
    return cudaGetLastError();
}

cudaError_t launch_tall_bf16x3(int np, const CUtensorMap *tmap, const TallArgs &a, int num_sms,
                               cudaStream_t s) {
    switch (np) {
        case 16: return launch_x3_t<16>(tmap, a, num_sms, s);
        case 32: return launch_x3_t<32>(tmap, a, num_sms, s);
        case 64: return launch_x3_t<64>(tmap, a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pack_b_bf16x3(int64_t k, int64_t n, const void *B, int64_t ldb, void *dst, int np,
                                 int64_t nchunks, int64_t ntiles, cudaStream_t s) {
    const int64_t total = ntiles * nchunks * np * kKB;
    if (total == 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    pack_b_bf16x3_kernel<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float *>(B), k, n, ldb,
                                                          static_cast<unsigned char *>(dst), np, nchunks,
                                                          ntiles);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Regime (ii) (k <= 128, m and n large) in the BF16x3 mode.  The cost of this
// shape is the m x n output stream (C0 in, C out); the tensor cores make the
// k-term products nearly free.  Persistent blocks walk work items = (m-tile of
// 128 rows, chunk of kRNCH n-tiles of 128 columns).  Per item the producer
// brings the FP32 A tile (128 x kp) once and the converters split it in place
// into hi|lo BF16; then the pre-split B tiles of the chunk stream through a
// double buffer, one thread issues the 3 x kp/16 MMAs of each tile (M = N =
// 128) into one of two TMEM accumulators, and eight epilogue warps (two per
// TMEM lane quarter, 64 columns each) read an accumulator, release it, and
// stream alpha*acc + beta*C0 to C with coalesced loads and stores.
namespace {

constexpr int kRNCH = 8;  // n-tiles per work item

template <int KC>  // 64-column k chunks: 1 (k <= 64) or 2 (k <= 128)
struct RX3Cfg {
    static constexpr int NT = kX3RankNT;                  // 128 columns per tile
    static constexpr int A_BYTES = KC * kBM * kKB * 4;    // FP32 in, then hi|lo per chunk, in place
    static constexpr int B_TILE = KC * 2 * NT * kKB * 2;  // hi|lo per chunk
    static constexpr int OFF_B = A_BYTES;
    static constexpr int OFF_BAR = OFF_B + 2 * B_TILE;
    static constexpr int NBAR = 3 + 2 + 2 + 2 + 2 + 1;
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 32;
    static constexpr int TMEM_COLS = 2 * NT;
    static constexpr int THREADS = 14 * 32;
};

}  // namespace

template <int KC>
__global__ void __launch_bounds__(448, 1)
    rankk_bf16x3_kernel(const __grid_constant__ CUtensorMap tmA, const RankArgs a, unsigned *status) {
    using Cfg = RX3Cfg<KC>;
    constexpr int NT = Cfg::NT;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + Cfg::OFF_BAR);
    uint64_t *a_full = bar;        // FP32 A tile landed
    uint64_t *a_conv = bar + 1;    // hi|lo written (4 converter warps)
    uint64_t *a_empty = bar + 2;   // the item's MMAs are done with A
    uint64_t *b_full = bar + 3;    // [2]
    uint64_t *b_empty = bar + 5;   // [2]
    uint64_t *tfull = bar + 7;     // [2]
    uint64_t *tempty = bar + 9;    // [2] (8 epilogue warps)
    uint64_t *done = bar + 11;
    unsigned *tslot = reinterpret_cast<unsigned *>(bar + Cfg::NBAR);
    unsigned *conv_abort = tslot + 1;
    unsigned *ep_abort = tslot + 2;

    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int64_t mtiles = (a.m + kBM - 1) / kBM;
    const int64_t ntiles = (a.n + NT - 1) / NT;
    const int64_t nch = (ntiles + kRNCH - 1) / kRNCH;
    const int64_t total = mtiles * nch;

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmA);
        mbar_init(a_full, 1);
        mbar_init(a_conv, 4);
        mbar_init(a_empty, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&b_full[b], 1);
            mbar_init(&b_empty[b], 1);
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);
        }
        mbar_init(done, 1);
        *conv_abort = 0u;
        *ep_abort = 0u;
        fence_mbar_init();
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tslot)),
                     "r"((uint32_t)Cfg::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 4) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            const uint64_t pol_a = policy_evict_last();  // A tiles are re-read by other n-chunks
            const uint64_t pol_b = policy_evict_last();
            const unsigned char *Bp = static_cast<const unsigned char *>(a.Bp);
            int64_t g = 0;
            int j = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x, ++j) {
                const int64_t mt = item / nch;
                const int64_t t0 = (item % nch) * kRNCH;
                const int64_t t1 = (t0 + kRNCH < ntiles) ? t0 + kRNCH : ntiles;
                if (j >= 1 && !mbar_wait_bounded(a_empty, (uint32_t)((j - 1) & 1))) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(a_full, Cfg::A_BYTES);
                for (int box = 0; box < 2 * KC; ++box)
                    tma_load_2d(smem + box * (kBM * 32 * 4), &tmA, (int32_t)(mt * kBM), (int32_t)(box * 32),
                                a_full, pol_a);
                for (int64_t t = t0; t < t1; ++t, ++g) {
                    const int sb = (int)(g & 1);
                    if (g >= 2 && !mbar_wait_bounded(&b_empty[sb], (uint32_t)((g >> 1) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&b_full[sb], Cfg::B_TILE);
                    bulk_load(smem + Cfg::OFF_B + sb * Cfg::B_TILE, Bp + t * Cfg::B_TILE, Cfg::B_TILE,
                              &b_full[sb], pol_b);
                }
            }
            if (!ok) atomicOr(status, kDevErrTimeout);
        }
        return;
    }

    if (warp == 5) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc(kBM, NT);
            int64_t g = 0;
            int j = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x, ++j) {
                const int64_t t0 = (item % nch) * kRNCH;
                const int64_t t1 = (t0 + kRNCH < ntiles) ? t0 + kRNCH : ntiles;
                if (!mbar_wait_bounded(a_conv, (uint32_t)(j & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int64_t t = t0; t < t1; ++t, ++g) {
                    const int sb = (int)(g & 1);
                    if (!mbar_wait_bounded(&b_full[sb], (uint32_t)((g >> 1) & 1)) ||
                        (g >= 2 && !mbar_wait_bounded(&tempty[sb], (uint32_t)((g >> 1) & 1) ^ 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tacc = tmem + (uint32_t)(sb * NT);
#pragma unroll
                    for (int c = 0; c < KC; ++c) {
                        const uint32_t ahi = smem_addr(smem + c * (kBM * kKB * 4));
                        const uint32_t alo = ahi + kBM * kKB * 2;
                        const uint32_t bhi = smem_addr(smem + Cfg::OFF_B + sb * Cfg::B_TILE + c * (2 * NT * kKB * 2));
                        const uint32_t blo = bhi + NT * kKB * 2;
#pragma unroll
                        for (int ks = 0; ks < kKB / 16; ++ks) {
                            const uint32_t off = ks * 2 * kLBO;
                            umma_bf16(tacc, umma_desc(ahi + off), umma_desc(bhi + off), idesc,
                                      (c | ks) != 0 ? 1u : 0u);
                            umma_bf16(tacc, umma_desc(ahi + off), umma_desc(blo + off), idesc, 1u);
                            umma_bf16(tacc, umma_desc(alo + off), umma_desc(bhi + off), idesc, 1u);
                        }
                    }
                    umma_commit(&b_empty[sb]);
                    umma_commit(&tfull[sb]);
                }
                if (ok) umma_commit(a_empty);
            }
            umma_commit(done);
            if (!ok) atomicOr(status, kDevErrTimeout);
            mbar_wait_bounded(done, 0);
        }
        __syncwarp();
        tc_fence_before();
        named_barrier(2, 288);  // warps 5..13
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)Cfg::TMEM_COLS));
        return;
    }

    if (warp < 4) {
        // ------------------------------------------------ converters: A tile in place
        const int r = threadIdx.x;
        int j = 0;
        for (int64_t item = blockIdx.x; item < total; item += gridDim.x, ++j) {
            const bool got = mbar_wait_bounded(a_full, (uint32_t)(j & 1));
            if (!got && lane == 0) atomicOr(conv_abort, 1u);
            named_barrier(1, 128);
            const bool stop = *conv_abort != 0u;
            named_barrier(1, 128);
            if (stop) {
                if (r == 0) atomicOr(status, kDevErrTimeout);
                break;
            }
#pragma unroll
            for (int c = 0; c < KC; ++c) {
                unsigned char *stage = smem + c * (kBM * kKB * 4);
                const float *src = reinterpret_cast<const float *>(stage);  // [64][128] FP32
                float x[kKB];
#pragma unroll
                for (int q = 0; q < kKB; ++q) x[q] = src[q * kBM + r];
                named_barrier(1, 128);  // the whole chunk is read before it is overwritten
                unsigned char *hi = stage;
                unsigned char *lo = stage + kBM * kKB * 2;
#pragma unroll
                for (int kg = 0; kg < kKB / 8; ++kg) {
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float x0 = x[kg * 8 + 2 * q];
                        const float x1 = x[kg * 8 + 2 * q + 1];
                        const __nv_bfloat162 hv = __floats2bfloat162_rn(x0, x1);
                        const float2 hf = __bfloat1622float2(hv);
                        const __nv_bfloat162 lv = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
                        h[q] = *reinterpret_cast<const uint32_t *>(&hv);
                        l[q] = *reinterpret_cast<const uint32_t *>(&lv);
                    }
                    const int off = kmaj_off(r, kg * 8);
                    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(a_conv);
        }
        return;
    }

    // ---------------------------------------------------- epilogue (warps 6-13)
    const int quarter = warp % 4;
    const int half = (warp - 6) / 4;
    const float alpha = static_cast<float>(a.alpha);
    const float beta = static_cast<float>(a.beta);
    float *C = static_cast<float *>(a.C);
    int64_t g = 0;
    bool stop = false;
    for (int64_t item = blockIdx.x; item < total && !stop; item += gridDim.x) {
        const int64_t mt = item / nch;
        const int64_t t0 = (item % nch) * kRNCH;
        const int64_t t1 = (t0 + kRNCH < ntiles) ? t0 + kRNCH : ntiles;
        const int64_t i = mt * kBM + quarter * 32 + lane;
        for (int64_t t = t0; t < t1; ++t, ++g) {
            const int tb = (int)(g & 1);
            const bool got = mbar_wait_bounded(&tfull[tb], (uint32_t)((g >> 1) & 1));
            if (!got && lane == 0) atomicOr(ep_abort, 1u);
            named_barrier(3, 256);
            stop = *ep_abort != 0u;
            named_barrier(3, 256);
            if (stop) {
                if (warp == 6 && lane == 0) atomicOr(status, kDevErrTimeout);
                break;
            }
            tc_fence_after();
            const int64_t j0 = t * NT + half * 64;
            float *crow = C + i;
            // all 64 C0 loads of this thread's half row are issued before any
            // store: 64 KB of reads in flight per SM keep HBM busy
            float c0v[64];
            if (beta != 0.f && i < a.m) {
#pragma unroll
                for (int jj = 0; jj < 64; ++jj)
                    c0v[jj] = (j0 + jj < a.n) ? crow[(j0 + jj) * a.ldc] : 0.f;
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float acc[16];
                tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tb * NT + half * 64 + b * 16),
                          acc);
                if (b == 3) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[tb]);  // the accumulator may be refilled
                }
                if (i < a.m) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int64_t jc = j0 + b * 16 + jj;
                        if (jc < a.n) {
                            float o = (alpha == 1.f) ? acc[jj] : alpha * acc[jj];
                            if (beta != 0.f) o = fmaf(beta, c0v[b * 16 + jj], o);
                            crow[jc * a.ldc] = o;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    named_barrier(2, 288);  // with warp 5, before it frees TMEM
}

template <int KC>
static cudaError_t launch_rx3_t(const CUtensorMap *tmA, const RankArgs &a, unsigned *status,
                                cudaStream_t s) {
    using Cfg = RX3Cfg<KC>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(rankk_bf16x3_kernel<KC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const int64_t mtiles = (a.m + kBM - 1) / kBM;
    const int64_t ntiles = (a.n + Cfg::NT - 1) / Cfg::NT;
    const int64_t items = mtiles * ((ntiles + kRNCH - 1) / kRNCH);
    const int64_t slots = a.num_sms > 0 ? a.num_sms : 1;
    const unsigned grid = (unsigned)(items < slots ? items : slots);
    if (grid == 0) return cudaSuccess;
    rankk_bf16x3_kernel<KC><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(*tmA, a, status);
    return cudaGetLastError();
}

cudaError_t launch_rankk_bf16x3(const CUtensorMap *tmA, const RankArgs &a, unsigned *status,
                                cudaStream_t s) {
    return a.kp <= kKB ? launch_rx3_t<1>(tmA, a, status, s) : launch_rx3_t<2>(tmA, a, status, s);
}

}  // namespace tsmm
