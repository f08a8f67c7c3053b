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

// Pack B (k x n, column-major) for this kernel: per 64-row chunk c, a hi tile
// and a lo tile, each NP rows (columns of B) x 64 k in the K-major layout
// above; zero outside the k x n matrix.
__global__ void pack_b_bf16x3_kernel(const float *__restrict__ B, int64_t k, int64_t n, int64_t ldb,
                                     unsigned char *__restrict__ dst, int np, int64_t nchunks) {
    const int64_t total = nchunks * np * kKB;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / (np * kKB);
        const int rem = (int)(e - c * np * kKB);
        const int j = rem / kKB;
        const int kk = rem % kKB;
        const int64_t p = c * kKB + kk;
        const float x = (p < k && j < n) ? B[p + j * ldb] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        unsigned char *chunk = dst + c * (int64_t)(2 * np * kKB * 2);
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
                                 int64_t nchunks, cudaStream_t s) {
    const int64_t total = nchunks * np * kKB;
    if (total == 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    pack_b_bf16x3_kernel<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float *>(B), k, n, ldb,
                                                          static_cast<unsigned char *>(dst), np, nchunks);
    return cudaGetLastError();
}

}  // namespace tsmm
