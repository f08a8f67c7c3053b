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

#include <cstring>

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

// U: an A that a tensor map cannot describe; each FP32 column of a stage then
// sits in a slot of A_STRIDE rows, at its own offset within 16 bytes.
template <int NP, bool U = false>
struct X3Cfg {
    static constexpr int A_STRIDE = U ? kBM + 8 : kBM;     // FP32 elements per column slot
    static constexpr int A_FP32_BYTES = kKB * A_STRIDE * 4;
    // FP32 in, then BF16 hi | lo (32 KB) over its start; whole KB for the MMA operands
    static constexpr int A_BYTES = (A_FP32_BYTES + 1023) / 1024 * 1024;
    static constexpr int B_BYTES = 2 * NP * kKB * 2;       // hi + lo chunk
    static constexpr int OFF_B = kS * A_BYTES;
    static constexpr int OFF_BAR = OFF_B + kS * B_BYTES;
    static constexpr int NBAR = 3 * kS + 4 + 1;
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 32;
    static constexpr int TMEM_COLS = 2 * NP < 32 ? 32 : 2 * NP;  // double-buffered accumulator
    // U: three producer warps (4, 10, 11), each moving up to 22 of a stage's 64
    // columns, one per lane: one warp issues its column copies too slowly to
    // keep up with HBM (one: 0.31 of HBM, two: 0.54); 12 warps still fit 168
    // registers a thread
    static constexpr int PRODUCERS = U ? 3 : 1;
    static constexpr int COLS_PER_PRODUCER = (kKB + PRODUCERS - 1) / PRODUCERS;
    static constexpr int THREADS = 320 + 32 * (PRODUCERS - 1);
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(!U || COLS_PER_PRODUCER <= 32, "one column per producer lane");
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
template <int NP, bool U>
__global__ void __launch_bounds__(X3Cfg<NP, U>::THREADS, 1)
    tall_bf16x3_kernel(const __grid_constant__ CUtensorMap tmA, const TallArgs a) {
    using Cfg = X3Cfg<NP, U>;
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

    // U: offset within 16 bytes of element (i0, p) of A is (abase + p * ldv) mod 4
    // (slabs start at multiples of 4 rows), so column q of a stage (which starts
    // at a multiple of 64) is at doff[q % 4]
    const int abase = (int)((reinterpret_cast<uintptr_t>(a.A) / sizeof(float)) & 3);
    const int ldv = (int)((uint64_t)a.lda & 3);

    if (threadIdx.x == 0) {
        if (!U) prefetch_tmap(&tmA);
        for (int s = 0; s < kS; ++s) {
            mbar_init(&full[s], Cfg::PRODUCERS);  // lane 0 of each producer warp
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

    if (warp == 4 || (U && warp >= 10)) {
        // ------------------------------------------------ producer(s)
        if (!U && lane == 0) {
            const uint64_t pol_a = policy_evict_first();
            const uint64_t pol_b = policy_evict_last();
            const unsigned char *Bp = static_cast<const unsigned char *>(a.Bp);
            int64_t g = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x) {
                int64_t slab, sp;
                udivmod(item, a.splits, slab, sp);
                const int64_t k0 = sp * a.kchunk;
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
        } else if (U) {
            // lane l < COLS_PER_PRODUCER of producer w moves column
            // w * COLS_PER_PRODUCER + l of each stage into its slot with one bulk copy of the 16-byte-aligned span around its rows
            // (column_span_bytes); lane 0 of each producer warp posts its warp's
            // bytes (and warp 4 the B chunk's) with its arrival before any of its
            // copies is issued; columns beyond k are zero-filled, like the tensor
            // copy's out-of-range fill; rows beyond m hold whatever the span left
            // (their results are never stored)
            const int pw = warp == 4 ? 0 : warp - 9;  // 0, 1, 2
            const uint64_t pol_a = policy_evict_first();
            const uint64_t pol_b = policy_evict_last();
            const unsigned char *Bp = static_cast<const unsigned char *>(a.Bp);
            const float *A = static_cast<const float *>(a.A);
            int64_t g = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x) {
                int64_t slab, sp;
                udivmod(item, a.splits, slab, sp);
                const int64_t k0 = sp * a.kchunk;
                const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;
                const int64_t i0 = slab * kBM;
                const int rows = (int)((a.m - i0 < kBM) ? a.m - i0 : kBM);
                for (int64_t kk = k0; kk < k1; kk += kKB, ++g) {
                    const int s = (int)(g % kS);
                    if (g >= kS) {
                        const bool got = mbar_wait_bounded(&empty[s], (uint32_t)((g / kS) & 1) ^ 1);
                        if (!__all_sync(0xffffffffu, got)) {
                            if (lane == 0) atomicOr(a.status, kDevErrTimeout);
                            ok = false;
                            break;
                        }
                    }
                    float *stageA = reinterpret_cast<float *>(smem + s * Cfg::A_BYTES);
                    const int q = Cfg::COLS_PER_PRODUCER * pw + lane;
                    const bool mine = lane < Cfg::COLS_PER_PRODUCER && q < kKB;
                    const int64_t p = kk + q;
                    float *slot0 = stageA + q * Cfg::A_STRIDE;
                    const int d = (abase + (int)(p & 3) * ldv) & 3;  // the column's offset within 16 bytes
                    const uint32_t bytes = mine && p < a.k ? column_span_bytes<float>(rows, d) : 0u;
                    if (mine && p >= a.k) {
                        for (int r = 0; r < Cfg::A_STRIDE; r += 4)
                            *reinterpret_cast<uint4 *>(slot0 + r) = make_uint4(0, 0, 0, 0);
                        fence_proxy_async_smem();  // before later copies into the slot
                    }
                    const uint32_t warp_bytes = __reduce_add_sync(0xffffffffu, bytes);
                    __syncwarp();  // the zero stores above precede lane 0's arrival
                    if (lane == 0) {
                        mbar_arrive_expect_tx(&full[s], (pw == 0 ? Cfg::B_BYTES : 0u) + warp_bytes);
                        if (pw == 0)
                            bulk_load(smem + Cfg::OFF_B + s * Cfg::B_BYTES, Bp + (kk / kKB) * Cfg::B_BYTES,
                                      Cfg::B_BYTES, &full[s], pol_b);
                    }
                    __syncwarp();
                    if (bytes != 0u) bulk_load(slot0, A + i0 + p * a.lda - d, bytes, &full[s], pol_a);
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
                int64_t slab_, sp;
                udivmod(item, a.splits, slab_, sp);
                const int64_t k0 = sp * a.kchunk;
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
            int64_t slab_, sp;
            udivmod(item, a.splits, slab_, sp);
            const int64_t k0 = sp * a.kchunk;
            const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;
            for (int64_t kk = k0; kk < k1; kk += kKB, ++g) {
                const int s = (int)(g % kS);
                const bool got = mbar_wait_bounded(&full[s], (uint32_t)((g / kS) & 1));
                unsigned char *stage = smem + s * Cfg::A_BYTES;
                const float *src = reinterpret_cast<const float *>(stage);  // [64][A_STRIDE] FP32
                float x[kKB];
                if (got) {
#pragma unroll
                    for (int q = 0; q < kKB; ++q)
                        x[q] = U ? src[q * Cfg::A_STRIDE + ((abase + (q & 3) * ldv) & 3) + r] : src[q * kBM + r];
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

        int64_t slab, sp64;
        udivmod(item, a.splits, slab, sp64);
        const int split = (int)sp64;
        const int64_t i = slab * kBM + r;
        // C = alpha*v + beta*C0 for columns c0 .. c0+15 of this thread's row: the
        // 16 C0 loads are issued together, ahead of the stores
        auto store16 = [&](int c0, const float *v) {
            if (i >= a.m) return;
            float *crow = C + i;
            float c0v[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
                c0v[jj] = (beta != 0.f && c0 + jj < a.n) ? crow[(int64_t)(c0 + jj) * a.ldc] : 0.f;
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                if (c0 + jj < a.n) {
                    float o = (alpha == 1.f) ? v[jj] : alpha * v[jj];
                    if (beta != 0.f) o = fmaf(beta, c0v[jj], o);
                    crow[(int64_t)(c0 + jj) * a.ldc] = o;
                }
            }
        };
        if (a.splits == 1) {
#pragma unroll
            for (int c0 = 0; c0 < NP; c0 += 16) store16(c0, acc + c0);
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
        // last arriver: the S partials summed in the fixed order s = 0..S-1, 16
        // columns at a time, the loads of split sp+1 in flight while split sp
        // is added
        const float *wrow = ws + slab * kBM + r;
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 16) {
            float sum[16], t[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                sum[jj] = 0.f;
                t[jj] = (split == 0) ? acc[c0 + jj] : ld_cg(wrow + (int64_t)(c0 + jj) * mpad);
            }
            for (int sp = 0; sp < a.splits; ++sp) {
                float nt[16];
                const int sn = sp + 1;
                if (sn < a.splits) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj)
                        nt[jj] = (sn == split) ? acc[c0 + jj]
                                               : ld_cg(wrow + ((int64_t)sn * NP + c0 + jj) * mpad);
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    sum[jj] += t[jj];
                    t[jj] = nt[jj];
                }
            }
            store16(c0, sum);
        }
        if (et == 0) a.tickets[slab] = 0u;
    }
    tc_fence_before();
    named_barrier(2, 160);  // with warp 5, before it frees TMEM
}

template <int NP, bool U>
static cudaError_t launch_x3_t(const CUtensorMap *tmap, const TallArgs &a, int num_sms, cudaStream_t s) {
    using Cfg = X3Cfg<NP, U>;
    {
        const cudaError_t e =
            ensure_smem_limit(reinterpret_cast<const void *>(tall_bf16x3_kernel<NP, U>), Cfg::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t items = a.slabs * a.splits;
    const int64_t slots = num_sms > 0 ? num_sms : 1;
    const unsigned grid = (unsigned)(items < slots ? items : slots);
    if (grid == 0) return cudaSuccess;
    CUtensorMap none;
    std::memset(&none, 0, sizeof(none));  // U: never read
    tall_bf16x3_kernel<NP, U><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(U ? none : *tmap, a);
    return cudaGetLastError();
}

// tmap: the tensor map of A, or nullptr for an A that one cannot describe
// (4-byte aligned; moved column by column).
cudaError_t launch_tall_bf16x3(int np, const CUtensorMap *tmap, const TallArgs &a, int num_sms,
                               cudaStream_t s) {
    const bool u = tmap == nullptr;
    switch (np) {
        case 16: return u ? launch_x3_t<16, true>(tmap, a, num_sms, s) : launch_x3_t<16, false>(tmap, a, num_sms, s);
        case 32: return u ? launch_x3_t<32, true>(tmap, a, num_sms, s) : launch_x3_t<32, false>(tmap, a, num_sms, s);
        case 64: return u ? launch_x3_t<64, true>(tmap, a, num_sms, s) : launch_x3_t<64, false>(tmap, a, num_sms, s);
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
// 128 rows, chunk of `rnch` n-tiles of 128 columns), with 16 warps:
//   warp 4      producer: the FP32 A tile (128 x kp) once per item, then the
//               pre-split B chunks (hi|lo, 64 k x 128 columns, 32 KB) of the
//               item's tiles through a ring of NB chunk buffers;
//   warps 0-3   converters: split the A tile in place into hi|lo BF16;
//   warp 5      allocates TMEM; lane 0 issues the 3 x kp/16 MMAs of a tile
//               (M = N = 128) into one of two TMEM accumulators;
//   warps 6-13  epilogue: two per TMEM lane quarter, each owning 64 columns
//               (two 32-column sub-tiles) of a tile: one tcgen05.ld of its 32
//               rows x 64 accumulator columns, then per sub-tile
//               alpha*acc + beta*C0;
//   warp 14     C0 loader (beta != 0): 128 x 32 sub-tiles of C0 into a ring
//               of CS shared-memory slots;
//   warp 15     storer: TMA stores of finished sub-tiles from their slots; a
//               slot is freed once its store has read it (`lag` = 1 keeps
//               the newest store in flight while freeing the one before).
// When C meets the TMA rules (16-byte aligned base and column stride) each
// sub-tile lives in one slot from C0 load to C store: the epilogue overwrites
// C0 with the result in place, the storer writes it out by TMA and frees the
// slot, so every global access of the output stream is a bulk copy.  Otherwise
// C0 arrives by 4-byte cp.async and the epilogue stores C directly (one
// 128-byte line per warp store).
namespace {

constexpr int kRNCHMax = 16;       // n-tiles per work item, at most
constexpr int kRSUB = kX3RankSub;  // columns per sub-tile (TMA box 128 x 32 FP32 = 16 KB)
constexpr int kRSUBS = kX3RankNT / kRSUB;

// U: an A that a tensor map cannot describe; each FP32 column of the A tile
// then sits in a slot of A_STRIDE rows at its own offset within 16 bytes (one
// B buffer fewer at KC = 2 makes room).
template <int KC, bool U = false>  // 64-column k chunks: 1 (k <= 64) or 2 (k <= 128)
struct RX3Cfg {
    static constexpr int NT = kX3RankNT;               // 128 columns per tile
    static constexpr int A_STRIDE = U ? kBM + 8 : kBM; // FP32 elements per column slot
    // one 64-column chunk: FP32 in, then hi|lo (32 KB) over its start, in place; whole KB
    static constexpr int A_CHUNK_BYTES = (kKB * A_STRIDE * 4 + 1023) / 1024 * 1024;
    static constexpr int A_BYTES = KC * A_CHUNK_BYTES;
    static constexpr int B_CHUNK = 2 * NT * kKB * 2;   // hi|lo of one 64-k chunk of one tile
    static constexpr int B_TILE = KC * B_CHUNK;
    static constexpr int NB = (KC == 1 || U) ? 2 : 3;  // B chunk buffers
    static constexpr int CS = (KC == 1 && !U) ? 8 : 4; // C slots (U, KC = 1: 8 do not fit)
    // Slot q % CS must always serve the same epilogue half (sub-tile q % 4):
    // its consumers then meet its phases in order, so parity waits cannot
    // alias (a half two phases ahead of a slot shared with the other half
    // would see the slot's older phase as complete).
    static_assert(CS % kRSUBS == 0, "each slot serves one epilogue half");
    static constexpr int SLOT = kBM * kRSUB * 4;
    static constexpr int OFF_BAR = 0;                  // barriers first
    static constexpr int OFF_A = 1024;
    static constexpr int OFF_B = OFF_A + A_BYTES;
    static constexpr int OFF_C = OFF_B + NB * B_CHUNK;
    static constexpr int NBAR = 3 + 2 * NB + 2 + 2 + 1 + 3 * CS;
    static constexpr int SMEM = OFF_C + CS * SLOT;
    static constexpr int SMEM_NO_SLOTS = OFF_C;        // beta == 0 and C not TMA-able
    static constexpr int TMEM_COLS = 2 * NT;
    static constexpr int THREADS = 16 * 32;
    static_assert(NBAR * 8 + 32 <= OFF_A, "barrier area");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// 2-D tiled tensor copy shared -> global (out-of-range parts of the box are
// not written); tracked by this thread's bulk async-groups.
__device__ __forceinline__ void tma_store_2d(const void *tmap, const void *smem_src, int32_t x, int32_t y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(tmap)),
                 "r"(x), "r"(y), "r"(smem_addr(smem_src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// every committed store has finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// every committed store but the newest has finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_but_one() {
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// every committed store is complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 64 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float *out) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]),
          "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]),
          "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]),
          "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
          "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 64; ++j) out[j] = __uint_as_float(r[j]);
}

// Warp-uniform bounded wait: every lane polls, and the warp proceeds only if
// all lanes saw the phase complete.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity) {
    return __all_sync(0xffffffffu, mbar_wait_bounded(bar, parity));
}

}  // namespace

template <int KC, bool U>
__global__ void __launch_bounds__(512, 1)
    rankk_bf16x3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmC,
                        const RankArgs a, unsigned *status, int c_tma, int rnch, int lag) {
    using Cfg = RX3Cfg<KC, U>;
    constexpr int NT = Cfg::NT;
    constexpr int NB = Cfg::NB;
    constexpr int CS = Cfg::CS;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + Cfg::OFF_BAR);
    uint64_t *a_full = bar;            // FP32 A tile landed
    uint64_t *a_conv = bar + 1;        // hi|lo written (4 converter warps)
    uint64_t *a_empty = bar + 2;       // the item's MMAs are done with A
    uint64_t *b_full = bar + 3;        // [NB]
    uint64_t *b_empty = b_full + NB;   // [NB]
    uint64_t *tfull = b_empty + NB;    // [2]
    uint64_t *tempty = tfull + 2;      // [2] (8 epilogue warps)
    uint64_t *done = tempty + 2;
    uint64_t *c_full = done + 1;       // [CS] C0 landed in the slot
    uint64_t *c_store = c_full + CS;   // [CS] results written to the slot (4 warps)
    uint64_t *c_empty = c_store + CS;  // [CS] slot free again
    unsigned *tslot = reinterpret_cast<unsigned *>(bar + Cfg::NBAR);
    unsigned *conv_abort = tslot + 1;
    float *cslots = reinterpret_cast<float *>(smem + Cfg::OFF_C);

    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int64_t mtiles = (a.m + kBM - 1) / kBM;
    const int64_t ntiles = (a.n + NT - 1) / NT;
    const int64_t nch = (ntiles + rnch - 1) / rnch;
    const int64_t total = mtiles * nch;
    const bool use_c0 = a.beta != 0.0;

    // U: offset within 16 bytes of element (i0, p) of A is (abase + p * ldv) mod 4
    // (tiles start at multiples of 4 rows, chunks at multiples of 64 columns)
    const int abase = (int)((reinterpret_cast<uintptr_t>(a.A) / sizeof(float)) & 3);
    const int ldv = (int)((uint64_t)a.lda & 3);

    if (threadIdx.x == 0) {
        if (!U) prefetch_tmap(&tmA);
        if (c_tma) prefetch_tmap(&tmC);
        mbar_init(a_full, 1);
        mbar_init(a_conv, 4);
        mbar_init(a_empty, 1);
        for (int b = 0; b < NB; ++b) {
            mbar_init(&b_full[b], 1);
            mbar_init(&b_empty[b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);
        }
        mbar_init(done, 1);
        for (int s = 0; s < CS; ++s) {
            mbar_init(&c_full[s], c_tma ? 1 : 32);
            mbar_init(&c_store[s], 4);
            mbar_init(&c_empty[s], c_tma ? 1 : 4);
        }
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
        // ------------------------------------------------ producer: A and B
        // A by tensor copies from lane 0, or (U) every lane moving columns lane,
        // lane + 32, ... of the item's A tile into their slots, each with one bulk
        // copy of the 16-byte-aligned span around its rows (column_span_bytes);
        // lane 0 posts the tile's bytes with its arrival before any copy is
        // issued, columns from k to the tile's end are zero-filled (the tensor
        // copy's out-of-range fill) and rows beyond m hold whatever the span left
        // (their results are never stored).  B chunks by bulk copies from lane 0.
        if (lane == 0 || U) {
            const uint64_t pol_a = policy_evict_last();  // A tiles are re-read by other n-chunks
            const uint64_t pol_b = policy_evict_last();
            const unsigned char *Bp = static_cast<const unsigned char *>(a.Bp);
            const float *A = static_cast<const float *>(a.A);
            int64_t gq = 0;  // B chunks issued
            int j = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x, ++j) {
                int64_t mt, ch;
                udivmod(item, nch, mt, ch);
                const int64_t t0 = ch * rnch;
                const int64_t t1 = (t0 + rnch < ntiles) ? t0 + rnch : ntiles;
                if (j >= 1) {
                    bool got = mbar_wait_bounded(a_empty, (uint32_t)((j - 1) & 1));
                    if (U) got = __all_sync(0xffffffffu, got);
                    if (!got) {
                        ok = false;
                        break;
                    }
                }
                if constexpr (!U) {
                    mbar_arrive_expect_tx(a_full, Cfg::A_BYTES);
                    for (int box = 0; box < 2 * KC; ++box)
                        tma_load_2d(smem + Cfg::OFF_A + box * (kBM * 32 * 4), &tmA, (int32_t)(mt * kBM),
                                    (int32_t)(box * 32), a_full, pol_a);
                } else {
                    const int64_t i0 = mt * kBM;
                    const int rows = (int)((a.m - i0 < kBM) ? a.m - i0 : kBM);
                    constexpr int PER_LANE = KC * kKB / 32;
                    uint32_t bytes[PER_LANE];
                    int dd[PER_LANE];
                    uint32_t sum = 0;
#pragma unroll
                    for (int h = 0; h < PER_LANE; ++h) {
                        const int p = lane + 32 * h;  // column of the tile
                        float *slot0 = reinterpret_cast<float *>(smem + Cfg::OFF_A + (p / kKB) * Cfg::A_CHUNK_BYTES) +
                                       (p % kKB) * Cfg::A_STRIDE;
                        dd[h] = (abase + (p & 3) * ldv) & 3;  // the column's offset within 16 bytes
                        bytes[h] = p < a.k ? column_span_bytes<float>(rows, dd[h]) : 0u;
                        if (p >= a.k) {
                            for (int r = 0; r < Cfg::A_STRIDE; r += 4)
                                *reinterpret_cast<uint4 *>(slot0 + r) = make_uint4(0, 0, 0, 0);
                            fence_proxy_async_smem();  // before later copies into the slot
                        }
                        sum += bytes[h];
                    }
                    const uint32_t tile_bytes = __reduce_add_sync(0xffffffffu, sum);
                    __syncwarp();  // the zero stores above precede lane 0's arrival
                    if (lane == 0) mbar_arrive_expect_tx(a_full, tile_bytes);
                    __syncwarp();
#pragma unroll
                    for (int h = 0; h < PER_LANE; ++h) {
                        const int p = lane + 32 * h;
                        if (bytes[h] != 0u)
                            bulk_load(reinterpret_cast<float *>(smem + Cfg::OFF_A + (p / kKB) * Cfg::A_CHUNK_BYTES) +
                                          (p % kKB) * Cfg::A_STRIDE,
                                      A + i0 + (int64_t)p * a.lda - dd[h], bytes[h], a_full, pol_a);
                    }
                }
                if (lane == 0) {
                    for (int64_t t = t0; t < t1 && ok; ++t) {
                        for (int c = 0; c < KC; ++c, ++gq) {
                            const int sb = (int)(gq % NB);
                            if (gq >= NB &&
                                !mbar_wait_bounded(&b_empty[sb], (uint32_t)((gq / NB) & 1) ^ 1)) {
                                ok = false;
                                break;
                            }
                            mbar_arrive_expect_tx(&b_full[sb], Cfg::B_CHUNK);
                            bulk_load(smem + Cfg::OFF_B + sb * Cfg::B_CHUNK,
                                      Bp + t * Cfg::B_TILE + c * Cfg::B_CHUNK, Cfg::B_CHUNK, &b_full[sb], pol_b);
                        }
                    }
                }
                if (U) ok = __shfl_sync(0xffffffffu, ok, 0);
            }
            if (lane == 0) {
                if (!ok) atomicOr(status, kDevErrTimeout);
                // copies still in flight land before the block may exit
                if (j >= 1) mbar_wait_bounded(a_full, (uint32_t)((j - 1) & 1));
                for (int64_t q = gq > NB ? gq - NB : 0; q < gq; ++q)
                    mbar_wait_bounded(&b_full[q % NB], (uint32_t)((q / NB) & 1));
            }
        }
        return;
    }

    if (warp == 14) {
        // ------------------------------------------------ C0 loader
        if (!use_c0) return;
        const uint64_t pol_c = policy_evict_first();
        const float *C = static_cast<const float *>(a.C);
        int64_t q = 0;  // sub-tiles issued
        bool ok = true;
        for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x) {
            int64_t mt, ch;
            udivmod(item, nch, mt, ch);
            const int64_t t0 = ch * rnch;
            const int64_t t1 = (t0 + rnch < ntiles) ? t0 + rnch : ntiles;
            for (int64_t t = t0; t < t1 && ok; ++t) {
                for (int sub = 0; sub < kRSUBS; ++sub, ++q) {
                    const int st = (int)(q % CS);
                    if (q >= CS && !warp_wait(&c_empty[st], (uint32_t)((q / CS) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    float *slot = cslots + st * (kBM * kRSUB);
                    const int64_t col0 = t * NT + sub * kRSUB;
                    if (c_tma) {
                        if (lane == 0) {
                            mbar_arrive_expect_tx(&c_full[st], Cfg::SLOT);
                            tma_load_2d(slot, &tmC, (int32_t)(mt * kBM), (int32_t)col0, &c_full[st], pol_c);
                        }
                    } else {
                        // element (row r, column c) of the slot sits at r + c * kBM; this
                        // lane copies rows lane + 32 rr of every column, walking one
                        // column pointer by ldc (a warp copy is one 128-byte run of C)
                        const int64_t i0 = mt * kBM;
                        bool rin[kBM / 32];
#pragma unroll
                        for (int rr = 0; rr < kBM / 32; ++rr) rin[rr] = i0 + lane + 32 * rr < a.m;
                        const float *colp = C + i0 + lane + col0 * a.ldc;
                        float *dst = slot + lane;
                        for (int c = 0; c < kRSUB; ++c, colp += a.ldc, dst += kBM) {
                            const bool cin = col0 + c < a.n;
#pragma unroll
                            for (int rr = 0; rr < kBM / 32; ++rr) {
                                const bool in = cin && rin[rr];
                                cp_async_elem(dst + 32 * rr, in ? colp + 32 * rr : C, in, 4);
                            }
                        }
                        cp_async_arrive_noinc(&c_full[st]);
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicOr(status, kDevErrTimeout);
        if (!c_tma) asm volatile("cp.async.wait_all;" ::: "memory");
        if (lane == 0)
            for (int64_t r = q > CS ? q - CS : 0; r < q; ++r)
                mbar_wait_bounded(&c_full[r % CS], (uint32_t)((r / CS) & 1));
        return;
    }

    if (warp == 15) {
        // ------------------------------------------------ storer (TMA mode)
        if (!c_tma || lane != 0) return;
        int64_t q = 0;  // sub-tiles stored
        bool ok = true;
        for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x) {
            int64_t mt, ch;
            udivmod(item, nch, mt, ch);
            const int64_t t0 = ch * rnch;
            const int64_t t1 = (t0 + rnch < ntiles) ? t0 + rnch : ntiles;
            for (int64_t t = t0; t < t1 && ok; ++t) {
                for (int sub = 0; sub < kRSUBS; ++sub, ++q) {
                    const int st = (int)(q % CS);
                    if (!mbar_wait_bounded(&c_store[st], (uint32_t)((q / CS) & 1))) {
                        ok = false;
                        break;
                    }
                    const int64_t col0 = t * NT + sub * kRSUB;
                    if (col0 < a.n)  // boxes wholly past the last column are not issued
                        tma_store_2d(&tmC, cslots + st * (kBM * kRSUB), (int32_t)(mt * kBM), (int32_t)col0);
                    bulk_commit();
                    if (lag == 0) {
                        bulk_wait_read_all();
                        mbar_arrive(&c_empty[st]);
                    } else if (q >= 1) {
                        bulk_wait_read_but_one();
                        mbar_arrive(&c_empty[(q - 1) % CS]);
                    }
                }
            }
        }
        if (!ok) atomicOr(status, kDevErrTimeout);
        bulk_wait_all();
        return;
    }

    if (warp == 5) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc(kBM, NT);
            int64_t g = 0, gq = 0;
            int j = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x, ++j) {
                int64_t mt_, ch;
                udivmod(item, nch, mt_, ch);
                const int64_t t0 = ch * rnch;
                const int64_t t1 = (t0 + rnch < ntiles) ? t0 + rnch : ntiles;
                if (!mbar_wait_bounded(a_conv, (uint32_t)(j & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int64_t t = t0; t < t1 && ok; ++t, ++g) {
                    const int tb = (int)(g & 1);
                    if (g >= 2 && !mbar_wait_bounded(&tempty[tb], (uint32_t)((g >> 1) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    const uint32_t tacc = tmem + (uint32_t)(tb * NT);
                    for (int c = 0; c < KC; ++c, ++gq) {
                        const int sb = (int)(gq % NB);
                        if (!mbar_wait_bounded(&b_full[sb], (uint32_t)((gq / NB) & 1))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t ahi = smem_addr(smem + Cfg::OFF_A + c * Cfg::A_CHUNK_BYTES);
                        const uint32_t alo = ahi + kBM * kKB * 2;
                        const uint32_t bhi = smem_addr(smem + Cfg::OFF_B + sb * Cfg::B_CHUNK);
                        const uint32_t blo = bhi + NT * kKB * 2;
#pragma unroll
                        for (int ks = 0; ks < kKB / 16; ++ks) {
                            const uint32_t off = ks * 2 * kLBO;
                            umma_bf16(tacc, umma_desc(ahi + off), umma_desc(bhi + off), idesc,
                                      (c | ks) != 0 ? 1u : 0u);
                            umma_bf16(tacc, umma_desc(ahi + off), umma_desc(blo + off), idesc, 1u);
                            umma_bf16(tacc, umma_desc(alo + off), umma_desc(bhi + off), idesc, 1u);
                        }
                        umma_commit(&b_empty[sb]);
                    }
                    if (ok) umma_commit(&tfull[tb]);
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
                unsigned char *stage = smem + Cfg::OFF_A + c * Cfg::A_CHUNK_BYTES;
                const float *src = reinterpret_cast<const float *>(stage);  // [64][A_STRIDE] FP32
                float x[kKB];
#pragma unroll
                for (int q = 0; q < kKB; ++q)
                    x[q] = U ? src[q * Cfg::A_STRIDE + ((abase + (q & 3) * ldv) & 3) + r] : src[q * kBM + r];
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
    // Each warp decides on its own to stop after a timed-out wait: the only
    // named barrier it meets afterwards is the final one with warp 5.
    const int quarter = warp % 4;
    const int half = (warp - 6) / 4;  // columns half*64 .. half*64+63 of each tile
    const float alpha = static_cast<float>(a.alpha);
    const float beta = static_cast<float>(a.beta);
    float *C = static_cast<float *>(a.C);
    int64_t g = 0, gc = 0;
    bool ok = true;
    for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x) {
        int64_t mt, ch;
        udivmod(item, nch, mt, ch);
        const int64_t t0 = ch * rnch;
        const int64_t t1 = (t0 + rnch < ntiles) ? t0 + rnch : ntiles;
        const int64_t i = mt * kBM + quarter * 32 + lane;
        float *crow = C + i;
        for (int64_t t = t0; t < t1 && ok; ++t, ++g, gc += kRSUBS) {
            const int tb = (int)(g & 1);
            if (!warp_wait(&tfull[tb], (uint32_t)((g >> 1) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            float acc[64];
            tmem_ld64(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tb * NT + half * 64), acc);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[tb]);  // the accumulator may be refilled
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float *v = acc + h * 32;
                const int64_t q = gc + half * 2 + h;  // this sub-tile's ring index
                const int st = (int)(q % CS);
                const uint32_t par = (uint32_t)((q / CS) & 1);
                float *slot = cslots + st * (kBM * kRSUB) + quarter * 32 + lane;  // column 0, own row
                if (use_c0 ? !warp_wait(&c_full[st], par)
                           : (c_tma && q >= CS && !warp_wait(&c_empty[st], par ^ 1))) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    v[jj] = alpha * v[jj];
                    if (use_c0) v[jj] = fmaf(beta, slot[jj * kBM], v[jj]);
                }
                if (c_tma) {
                    // result replaces C0 in the slot; the storer writes it out
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) slot[jj * kBM] = v[jj];
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&c_store[st]);
                } else {
                    if (use_c0) {
                        release_reads_to_async_copy();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&c_empty[st]);
                    }
                    const int64_t jb = t * NT + half * 64 + h * 32;
                    if (i < a.m) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj)
                            if (jb + jj < a.n) crow[(jb + jj) * a.ldc] = v[jj];
                    }
                }
            }
        }
    }
    if (!ok && lane == 0) atomicOr(status, kDevErrTimeout);
    tc_fence_before();
    named_barrier(2, 288);  // with warp 5, before it frees TMEM
}

template <int KC, bool U>
static cudaError_t launch_rx3_t(const CUtensorMap *tmA, const CUtensorMap *tmC, const RankArgs &a,
                                unsigned *status, cudaStream_t s) {
    using Cfg = RX3Cfg<KC, U>;
    {
        const cudaError_t e =
            ensure_smem_limit(reinterpret_cast<const void *>(rankk_bf16x3_kernel<KC, U>), Cfg::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t mtiles = (a.m + kBM - 1) / kBM;
    const int64_t ntiles = (a.n + Cfg::NT - 1) / Cfg::NT;
    const int64_t slots = a.num_sms > 0 ? a.num_sms : 1;
    // n-tiles per item: long items amortise the A tile's load and split, but
    // keep at least ~4 items per block for balance
    int64_t rnch = mtiles * ntiles / (4 * slots);
    rnch = rnch < 1 ? 1 : (rnch > kRNCHMax ? kRNCHMax : rnch);
    const int64_t items = mtiles * ((ntiles + rnch - 1) / rnch);
    const unsigned grid = (unsigned)(items < slots ? items : slots);
    if (grid == 0) return cudaSuccess;
    CUtensorMap none;
    memset(&none, 0, sizeof(none));
    const int smem = (tmC || a.beta != 0.0) ? Cfg::SMEM : Cfg::SMEM_NO_SLOTS;
    // with only 4 slots and C0 to prefetch, free each slot as early as possible
    const int lag = (Cfg::CS == 4 && a.beta != 0.0) ? 0 : 1;
    rankk_bf16x3_kernel<KC, U><<<grid, Cfg::THREADS, smem, s>>>(U ? none : *tmA, tmC ? *tmC : none, a, status,
                                                             tmC ? 1 : 0, (int)rnch, lag);
    return cudaGetLastError();
}

// tmA: the tensor map of A, or nullptr for an A that one cannot describe
// (4-byte aligned; moved column by column).
cudaError_t launch_rankk_bf16x3(const CUtensorMap *tmA, const CUtensorMap *tmC, const RankArgs &a,
                                unsigned *status, cudaStream_t s) {
    if (tmA == nullptr)
        return a.kp <= kKB ? launch_rx3_t<1, true>(tmA, tmC, a, status, s)
                           : launch_rx3_t<2, true>(tmA, tmC, a, status, s);
    return a.kp <= kKB ? launch_rx3_t<1, false>(tmA, tmC, a, status, s)
                       : launch_rx3_t<2, false>(tmA, tmC, a, status, s);
}

}  // namespace tsmm
