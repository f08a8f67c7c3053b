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
// Block = one m-slab of 128 rows x one k range (the same split-K scheme as the
// FMA kernel), 6 warps:
//   warp 4      producer: TMA copies of FP32 A tiles (128 rows x 64 columns)
//               and bulk copies of the pre-split B chunks (hi|lo, K-major);
//   warps 0-3   converters: split A into hi/lo BF16 written in the K-major
//               canonical UMMA layout; afterwards the epilogue, each thread
//               owning one accumulator row (TMEM lane);
//   warp 5      allocates tensor memory; lane 0 issues tcgen05.mma
//               (M = 128, N = NP, K = 16 per instruction, 3 per k-step) and
//               commits completions to mbarriers.
// Shared-memory operand layout (K-major, no swizzle): element (row, k) of a
// 64-column chunk sits at (row/8)*1024 + (k/8)*128 + (row%8)*16 + (k%8)*2
// bytes, i.e. 8x8 core matrices of 128 B, adjacent along k (LBO = 128 B) and
// 1 KB apart along rows (SBO = 1024 B).
#include <cuda_bf16.h>

#include "tsmm_device.cuh"
#include "tsmm_internal.h"

namespace tsmm {

namespace {

constexpr int kKB = 64;     // k per chunk
constexpr int kBM = 128;    // rows per block = MMA M = TMEM lanes
constexpr int kS32 = 3;     // FP32 A ring
constexpr int kSB = 2;      // BF16 A ring
constexpr int kLBO = 128;
constexpr int kSBO = 1024;

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
    static constexpr int A32_BYTES = kBM * kKB * 4;        // 32 KB
    static constexpr int ABF_BYTES = 2 * kBM * kKB * 2;    // hi + lo, 32 KB
    static constexpr int B_BYTES = 2 * NP * kKB * 2;       // hi + lo chunk
    static constexpr int OFF_ABF = kS32 * A32_BYTES;
    static constexpr int OFF_B = OFF_ABF + kSB * ABF_BYTES;
    static constexpr int OFF_BAR = OFF_B + kS32 * B_BYTES;
    static constexpr int NBAR = 4 * kS32 + 2 * kSB + 1;
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16;
    static constexpr int TMEM_COLS = NP < 32 ? 32 : NP;
    static constexpr int THREADS = 192;
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

template <int NP>
__global__ void __launch_bounds__(192, 1)
    tall_bf16x3_kernel(const __grid_constant__ CUtensorMap tmA, const TallArgs a) {
    using Cfg = X3Cfg<NP>;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + Cfg::OFF_BAR);
    uint64_t *full32 = bar;
    uint64_t *empty32 = full32 + kS32;
    uint64_t *fullB = empty32 + kS32;
    uint64_t *emptyB = fullB + kS32;
    uint64_t *fullA = emptyB + kS32;
    uint64_t *emptyA = fullA + kSB;
    uint64_t *done = emptyA + kSB;
    unsigned *tslot = reinterpret_cast<unsigned *>(done + 1);
    unsigned *flag = tslot + 1;
    unsigned *abort_flag = tslot + 2;

    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int64_t slab = blockIdx.x;
    const int split = blockIdx.y;
    const int64_t k0 = (int64_t)split * a.kchunk;
    const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;
    const int nchunks = (int)((k1 - k0) / kKB);

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmA);
        for (int s = 0; s < kS32; ++s) {
            mbar_init(&full32[s], 1);
            mbar_init(&empty32[s], 4);
            mbar_init(&fullB[s], 1);
            mbar_init(&emptyB[s], 1);
        }
        for (int s = 0; s < kSB; ++s) {
            mbar_init(&fullA[s], 4);
            mbar_init(&emptyA[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0u;
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
            for (int c = 0; c < nchunks; ++c) {
                const int s = c % kS32;
                const uint32_t par = ((c / kS32) & 1) ^ 1;
                if (c >= kS32 && (!mbar_wait_bounded(&empty32[s], par) || !mbar_wait_bounded(&emptyB[s], par))) {
                    atomicOr(a.status, kDevErrTimeout);
                    break;
                }
                const int64_t kk = k0 + (int64_t)c * kKB;
                float *dstA = reinterpret_cast<float *>(smem + s * Cfg::A32_BYTES);
                mbar_arrive_expect_tx(&full32[s], Cfg::A32_BYTES);
                tma_load_2d(dstA, &tmA, (int32_t)(slab * kBM), (int32_t)kk, &full32[s], pol_a);
                tma_load_2d(dstA + kBM * 32, &tmA, (int32_t)(slab * kBM), (int32_t)(kk + 32), &full32[s],
                            pol_a);
                mbar_arrive_expect_tx(&fullB[s], Cfg::B_BYTES);
                bulk_load(smem + Cfg::OFF_B + s * Cfg::B_BYTES, Bp + (kk / kKB) * Cfg::B_BYTES,
                          Cfg::B_BYTES, &fullB[s], pol_b);
            }
        }
        return;
    }

    if (warp == 5) {
        // ------------------------------------------------ MMA issuer
        bool ok = true;
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc(kBM, NP);
            for (int c = 0; c < nchunks && ok; ++c) {
                const int sa = c % kSB;
                const int sb = c % kS32;
                if (!mbar_wait_bounded(&fullA[sa], (c / kSB) & 1) ||
                    !mbar_wait_bounded(&fullB[sb], (c / kS32) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ahi = smem_addr(smem + Cfg::OFF_ABF + sa * Cfg::ABF_BYTES);
                const uint32_t alo = ahi + kBM * kKB * 2;
                const uint32_t bhi = smem_addr(smem + Cfg::OFF_B + sb * Cfg::B_BYTES);
                const uint32_t blo = bhi + NP * kKB * 2;
#pragma unroll
                for (int ks = 0; ks < kKB / 16; ++ks) {
                    const uint32_t off = ks * 2 * kLBO;  // 16 k = two core matrices
                    umma_bf16(tmem, umma_desc(ahi + off), umma_desc(bhi + off), idesc, (c | ks) != 0);
                    umma_bf16(tmem, umma_desc(ahi + off), umma_desc(blo + off), idesc, 1u);
                    umma_bf16(tmem, umma_desc(alo + off), umma_desc(bhi + off), idesc, 1u);
                }
                umma_commit(&emptyA[sa]);  // this chunk's A hi/lo slot is free once these finish
                umma_commit(&emptyB[sb]);  // ... and its B slot
            }
            umma_commit(done);  // all issued products complete (also on the give-up path)
            if (!ok) {
                atomicOr(a.status, kDevErrTimeout);
                atomicOr(abort_flag, 1u);
            }
        }
        __syncwarp();
        // wait for the epilogue to finish reading TMEM, then free it
        tc_fence_before();
        named_barrier(2, 160);
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)Cfg::TMEM_COLS));
        return;
    }

    // ---------------------------------------------------- converters (warps 0-3)
    const int r = threadIdx.x;  // row of the slab, = TMEM lane
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int s = c % kS32;
        const int sa = c % kSB;
        if (!mbar_wait_bounded(&full32[s], (c / kS32) & 1) ||
            (c >= kSB && !mbar_wait_bounded(&emptyA[sa], ((c / kSB) & 1) ^ 1))) {
            ok = false;
            break;
        }
        const float *src = reinterpret_cast<const float *>(smem + s * Cfg::A32_BYTES);  // [64][128]
        unsigned char *hi = smem + Cfg::OFF_ABF + sa * Cfg::ABF_BYTES;
        unsigned char *lo = hi + kBM * kKB * 2;
#pragma unroll
        for (int kg = 0; kg < kKB / 8; ++kg) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float x0 = src[(kg * 8 + 2 * q) * kBM + r];
                const float x1 = src[(kg * 8 + 2 * q + 1) * kBM + r];
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
        if (lane == 0) {
            mbar_arrive(&fullA[sa]);
            mbar_arrive(&empty32[s]);
        }
    }
    if (!ok && lane == 0) {
        atomicOr(a.status, kDevErrTimeout);
        atomicOr(abort_flag, 1u);
    }

    // ---------------------------------------------------- epilogue (warps 0-3)
    float acc[NP];
    bool have = ok && mbar_wait_bounded(done, 0);
    tc_fence_after();
    if (have) {
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 16)
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc + c0);
    }
    tc_fence_before();
    named_barrier(2, 160);  // TMEM may be freed now
    named_barrier(1, 128);
    if (!have && lane == 0) atomicOr(abort_flag, 1u);
    named_barrier(1, 128);
    if (*abort_flag != 0u) {
        if (threadIdx.x == 0) atomicOr(a.status, kDevErrTimeout);
        return;
    }

    const float alpha = static_cast<float>(a.alpha);
    const float beta = static_cast<float>(a.beta);
    const int64_t row0 = slab * kBM;
    const int64_t i = row0 + r;
    float *C = static_cast<float *>(a.C);
    auto store = [&](int j, float v) {
        if (i < a.m && j < a.n) {
            float o = (alpha == 1.f) ? v : alpha * v;
            float *cp = C + i + (int64_t)j * a.ldc;
            if (beta != 0.f) o = fmaf(beta, *cp, o);
            *cp = o;
        }
    };
    if (a.splits == 1) {
#pragma unroll
        for (int j = 0; j < NP; ++j) store(j, acc[j]);
        return;
    }
    const int64_t mpad = a.slabs * kBM;
    float *ws = static_cast<float *>(a.ws);
#pragma unroll
    for (int j = 0; j < NP; ++j) ws[((int64_t)split * NP + j) * mpad + row0 + r] = acc[j];
    __threadfence();
    named_barrier(1, 128);
    if (threadIdx.x == 0) {
        const unsigned ticket = atomicAdd(a.tickets + slab, 1u);
        *flag = (ticket == (unsigned)(a.splits - 1)) ? 1u : 0u;
    }
    named_barrier(1, 128);
    if (*flag == 0u) return;
    __threadfence();
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        float s = 0.f;
        for (int sp = 0; sp < a.splits; ++sp)
            s += (sp == split) ? acc[j] : ld_cg(ws + ((int64_t)sp * NP + j) * mpad + row0 + r);
        store(j, s);
    }
    if (threadIdx.x == 0) a.tickets[slab] = 0u;
}

template <int NP>
static cudaError_t launch_x3_t(const CUtensorMap *tmap, const TallArgs &a, cudaStream_t s) {
    using Cfg = X3Cfg<NP>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(tall_bf16x3_kernel<NP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((unsigned)a.slabs, (unsigned)a.splits);
    tall_bf16x3_kernel<NP><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(*tmap, a);
    return cudaGetLastError();
}

cudaError_t launch_tall_bf16x3(int np, const CUtensorMap *tmap, const TallArgs &a, cudaStream_t s) {
    switch (np) {
        case 16: return launch_x3_t<16>(tmap, a, s);
        case 32: return launch_x3_t<32>(tmap, a, s);
        case 64: return launch_x3_t<64>(tmap, a, s);
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
