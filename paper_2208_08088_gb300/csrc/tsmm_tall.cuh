// Regime (i) kernel: C[m x n] = alpha * A[m x k] * B[k x n] + beta * C0, n <= 64.
//
// Mapping of the paper's tiled algorithm (Section IV.A, Fig. 2) to the GPU:
//   * GEPB_t (a block of m_t rows per CPU thread) -> a thread block owns an
//     m-slab of BM rows and a contiguous k range.  n is never split across
//     blocks (the paper leaves n untiled when n <= n_c, Section IV.A.2), so each
//     block stages the full-width rows of packed B it needs in shared memory,
//     the counterpart of each core keeping its B block in its own L1.
//   * No barrier between k iterations thanks to pre-packing (Section IV.A.2)
//     -> blocks never wait for each other: the k splits of a slab are combined
//     by whichever block finishes last (an atomic arrival ticket; nobody
//     spins), in the fixed order s = 0..S-1.
//   * Register-blocked m_r x n_r inner kernels (Section IV.B) -> each thread
//     keeps an R x CN register tile of C; A arrives through a multi-stage TMA
//     pipeline (the GPU form of the paper's prefetching, Section IV.B.3), and B
//     rows are read from shared memory as broadcasts.
//
// Block layout: kTallConsumerWarps consumer warps + 1 producer warp.  The
// producer issues, per stage, one 2-D tensor copy of A (BM rows x BKS columns,
// zero-filled outside the matrix) and one bulk copy of BKS packed B rows.
// Consumer warps are arranged WM (along m) x WK (along k); lanes are arranged
// LR (along m) x G (along n).  After the k loop the WK partial tiles are summed
// in shared memory in warp order, then either stored (one split) or written to
// the split-K workspace and finished by the last-arriving block.
#pragma once
#include <type_traits>

#include "tsmm_device.cuh"
#include "tsmm_internal.h"

namespace tsmm {

template <typename T, int NP>
struct TallCfg {
    static constexpr int VEC = 16 / (int)sizeof(T);   // elements per 16-byte vector
    // The FMA-bound FP32 shapes (n >= 32) use 8-row thread tiles: 8 x 8 (32
    // packed fmas per 4 shared-memory loads of 16 bytes; a 16-byte load costs
    // four shared-memory wavefronts whatever its address pattern, and the
    // 4 x 16 tile's 5 loads per 32 fmas saturate them before the FMA pipe), and
    // 8 x 12 for the width 48 (5 loads per 48 packed fmas; n = 48 at
    // m = k = 32768: 1.52 -> 1.46 ms against 4 x 12).  A thread's 8 rows are two
    // groups of 4, half a warp tile apart, so the lanes along m read adjacent
    // 16-byte words of A (no bank shared).  FP32 width 24 and FP64 widths 24
    // and 48 use VEC x 12 tiles.
    static constexpr bool WIDE = sizeof(T) == 4 && (NP == 32 || NP == 48 || NP == 64);
    static constexpr int R = WIDE ? 8 : VEC;  // rows per thread
    static constexpr int CN = WIDE ? (NP == 48 ? 12 : 8)
                                   : ((NP == 24 || NP == 48) ? 12 : (NP < 16 ? NP : 16));  // columns per thread
    static constexpr int G = NP / CN;                  // lane groups along n
    static constexpr int LR = 32 / G;                  // lanes along m
    static constexpr int WROWS = LR * R;               // rows per warp
    static constexpr int RG = WIDE ? 2 : 1;            // row groups per thread
    static constexpr int RV = R / RG;                  // rows per group (one vector)
    static constexpr int GSTRIDE = WROWS / RG;         // distance between a thread's groups
    // local row of this thread's row r, given rloc = wm*WROWS + lr*RV
    static __host__ __device__ constexpr int row(int rloc, int r) { return rloc + (r / RV) * GSTRIDE + r % RV; }
    static constexpr int BM = tall_block_rows(sizeof(T) == 8, NP);
    static constexpr int WM = BM / WROWS;              // warps along m
    static constexpr int NWARPS = kTallConsumerWarps;
    static constexpr int WK = NWARPS / WM;             // warps along k
    static constexpr int BKS = kTallBKS;
    static constexpr int KPW = BKS / WK;               // stage columns per warp
    static constexpr int BV = CN < VEC ? CN : VEC;     // B vector width
    static constexpr int A_STAGE = BM * BKS;           // elements
    static constexpr int B_STAGE = BKS * NP;           // elements
    static constexpr int STAGE_BYTES = (A_STAGE + B_STAGE) * (int)sizeof(T);
    // Resident blocks per SM the ring is sized for: FMA-bound shapes (FP32,
    // n >= 32) want more warps to hide shared-memory latency and need less data
    // in flight, so they get a shorter ring and three blocks per SM.
    static constexpr int RESIDENT = tall_resident_blocks(sizeof(T) == 8, NP);
    static constexpr int SMEM_BUDGET = RESIDENT >= 3 ? 72 * 1024 : 100 * 1024;
    static constexpr int STAGES_RAW = SMEM_BUDGET / STAGE_BYTES;
    static constexpr int STAGES = STAGES_RAW < 2 ? 2 : (STAGES_RAW > 6 ? 6 : STAGES_RAW);
    static constexpr int RED = WK * NP * BM;           // reduction buffer elements
    static constexpr int DATA_BYTES = STAGES * STAGE_BYTES > RED * (int)sizeof(T)
                                          ? STAGES * STAGE_BYTES
                                          : RED * (int)sizeof(T);
    static constexpr int SMEM = DATA_BYTES + 2 * STAGES * 8 + 16;
    static constexpr int THREADS = (NWARPS + 1) * 32;
    static constexpr int CONSUMERS = NWARPS * 32;
    static_assert(G * CN == NP, "column split");
    static_assert(WM * WROWS == BM && WM <= NWARPS && WK * WM == NWARPS, "warp split");
    static_assert(WK * KPW == BKS, "stage split");
    static_assert(BM * (int)sizeof(T) % 16 == 0, "TMA box row bytes");
};

// A thread's R rows of one A column (cb: the column's first element) and
// the store of R row values of one C column, in the thread's row layout.
template <typename Cfg, typename T>
__device__ __forceinline__ Vec<T, Cfg::R> tall_load_rows(const T *cb, int rloc) {
    Vec<T, Cfg::R> v;
#pragma unroll
    for (int gi = 0; gi < Cfg::RG; ++gi) {
        const Vec<T, Cfg::RV> part = ld_vec<T, Cfg::RV>(cb + rloc + gi * Cfg::GSTRIDE);
#pragma unroll
        for (int r = 0; r < Cfg::RV; ++r) v.v[gi * Cfg::RV + r] = part.v[r];
    }
    return v;
}
template <typename Cfg, typename T>
__device__ __forceinline__ void tall_store_rows(T *cb, int rloc, const Vec<T, Cfg::R> &v) {
#pragma unroll
    for (int gi = 0; gi < Cfg::RG; ++gi) {
        Vec<T, Cfg::RV> part;
#pragma unroll
        for (int r = 0; r < Cfg::RV; ++r) part.v[r] = v.v[gi * Cfg::RV + r];
        st_vec<T, Cfg::RV>(cb + rloc + gi * Cfg::GSTRIDE, part);
    }
}

// Sum of the WK per-warp partial tiles, then store / split-K finish.
// `red` holds WK tiles laid out [WK][NP][BM]; on return red[0..NP*BM) is reused.
template <typename T, int NP>
__device__ __forceinline__ void tall_finish(T *red, const TallArgs &a, int64_t slab, int split,
                                            int ctid, unsigned *smem_flag) {
    using Cfg = TallCfg<T, NP>;
    constexpr int R = Cfg::R;
    constexpr int CHUNKS = NP * Cfg::BM / R;
    const T alpha = static_cast<T>(a.alpha);
    const T beta = static_cast<T>(a.beta);
    const int64_t row0 = slab * Cfg::BM;

    // 1) cross-warp sum in warp order w = 0..WK-1
    if (Cfg::WK > 1) {
        for (int q = ctid; q < CHUNKS; q += Cfg::CONSUMERS) {
            Vec<T, R> s = ld_vec<T, R>(red + q * R);
#pragma unroll
            for (int w = 1; w < Cfg::WK; ++w) {
                Vec<T, R> t = ld_vec<T, R>(red + w * NP * Cfg::BM + q * R);
#pragma unroll
                for (int r = 0; r < R; ++r) s.v[r] += t.v[r];
            }
            st_vec<T, R>(red + q * R, s);
        }
        named_barrier(1, Cfg::CONSUMERS);
    }

    // C = alpha*v + beta*C0 for R rows of one column: one vector access when
    // the chunk lies inside C and is aligned, else the R C0 loads issued
    // together, ahead of the stores
    auto store = [&](int q, const Vec<T, R> &v) {
        const int j = (q * R) / Cfg::BM;
        const int il = (q * R) % Cfg::BM;
        if (j >= a.n) return;
        T *c = static_cast<T *>(a.C) + row0 + il + (int64_t)j * a.ldc;
        const int64_t rows = a.m - (row0 + il);  // rows of this chunk inside C
        if (rows >= R && reinterpret_cast<uintptr_t>(c) % sizeof(Vec<T, R>) == 0) {
            Vec<T, R> o;
            const Vec<T, R> c0 = beta != T(0) ? ld_vec<T, R>(c) : Vec<T, R>{};
#pragma unroll
            for (int r = 0; r < R; ++r) {
                o.v[r] = alpha * v.v[r];
                if (beta != T(0)) o.v[r] = fma(beta, c0.v[r], o.v[r]);
            }
            st_vec<T, R>(c, o);
            return;
        }
        T c0[R];
#pragma unroll
        for (int r = 0; r < R; ++r) c0[r] = (beta != T(0) && r < rows) ? c[r] : T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < rows) {
                T out = alpha * v.v[r];
                if (beta != T(0)) out = fma(beta, c0[r], out);
                c[r] = out;
            }
        }
    };

    if (a.splits == 1) {
        for (int q = ctid; q < CHUNKS; q += Cfg::CONSUMERS) store(q, ld_vec<T, R>(red + q * R));
        return;
    }

    // 2) split-K: publish this block's partial tile, take an arrival ticket
    const int64_t mpad = a.slabs * Cfg::BM;
    T *ws = static_cast<T *>(a.ws);
    for (int q = ctid; q < CHUNKS; q += Cfg::CONSUMERS) {
        const int j = (q * R) / Cfg::BM;
        const int il = (q * R) % Cfg::BM;
        st_vec<T, R>(ws + ((int64_t)split * NP + j) * mpad + row0 + il, ld_vec<T, R>(red + q * R));
    }
    __threadfence();
    named_barrier(1, Cfg::CONSUMERS);
    if (ctid == 0) {
        const unsigned ticket = atomicAdd(a.tickets + slab, 1u);
        *smem_flag = (ticket == (unsigned)(a.splits - 1)) ? 1u : 0u;
    }
    named_barrier(1, Cfg::CONSUMERS);
    if (*smem_flag == 0u) return;

    // 3) last arriver: sum the S partial tiles in the fixed order s = 0..S-1
    __threadfence();
    for (int q = ctid; q < CHUNKS; q += Cfg::CONSUMERS) {
        const int j = (q * R) / Cfg::BM;
        const int il = (q * R) % Cfg::BM;
        // partial of split sp (this block's own from shared memory)
        auto partial = [&](int sp) {
            Vec<T, R> t;
            if (sp == split) {
                t = ld_vec<T, R>(red + q * R);
            } else {
                const T *src = ws + ((int64_t)sp * NP + j) * mpad + row0 + il;
#pragma unroll
                for (int r = 0; r < R; ++r) t.v[r] = ld_cg(src + r);
            }
            return t;
        };
        Vec<T, R> s;
#pragma unroll
        for (int r = 0; r < R; ++r) s.v[r] = T(0);
        Vec<T, R> t = partial(0);
        for (int sp = 0; sp < a.splits; ++sp) {
            // the loads of split sp+1 are in flight while split sp is added
            const Vec<T, R> nt = partial(sp + 1 < a.splits ? sp + 1 : sp);
#pragma unroll
            for (int r = 0; r < R; ++r) s.v[r] += t.v[r];
            t = nt;
        }
        store(q, s);
    }
    if (ctid == 0) a.tickets[slab] = 0u;  // ready for the next launch on this stream
}

// Register tile of one thread: R rows x CN columns of C.  acc(r, c) +=
// A[r] * B[c] for one A column at a time, each product an IEEE fma in the
// working precision.  FP32 tiles with CN >= 2 store column pairs as float2 and
// use the packed FP32x2 fma (fma.rn.f32x2): the same two roundings as two
// scalar fmas, in half the issue slots, which leaves room for the shared-
// memory loads of A and B in the FMA-bound cases (n >= 16).
template <typename T, int R, int CN, int BV>
struct AccTile {
    T v[R][CN];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < CN; ++c) v[r][c] = T(0);
    }
    __device__ __forceinline__ void fma_column(const Vec<T, R> &av, const T *bsrc) {
#pragma unroll
        for (int c0 = 0; c0 < CN; c0 += BV) {
            const Vec<T, BV> bv = ld_vec<T, BV>(bsrc + c0);
#pragma unroll
            for (int c = 0; c < BV; ++c)
#pragma unroll
                for (int r = 0; r < R; ++r) v[r][c0 + c] = fma(av.v[r], bv.v[c], v[r][c0 + c]);
        }
    }
    __device__ __forceinline__ T get(int r, int c) const { return v[r][c]; }
};

template <int R, int CN>
struct AccTilePairs {
    float2 v[R][CN / 2];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < CN / 2; ++c) v[r][c] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void fma_column(const Vec<float, R> &av, const float *bsrc) {
        float2 ad[R];
#pragma unroll
        for (int r = 0; r < R; ++r) ad[r] = make_float2(av.v[r], av.v[r]);
        constexpr int BV = CN < 4 ? CN : 4;
#pragma unroll
        for (int c0 = 0; c0 < CN; c0 += BV) {
            const Vec<float, BV> bv = ld_vec<float, BV>(bsrc + c0);
#pragma unroll
            for (int c = 0; c < BV; c += 2) {
                const float2 b2 = make_float2(bv.v[c], bv.v[c + 1]);
#pragma unroll
                for (int r = 0; r < R; ++r)
                    v[r][(c0 + c) / 2] = __ffma2_rn(ad[r], b2, v[r][(c0 + c) / 2]);
            }
        }
    }
    __device__ __forceinline__ float get(int r, int c) const {
        return (c & 1) ? v[r][c / 2].y : v[r][c / 2].x;
    }
};

template <typename T, int NP>
struct TallAcc {
    using Cfg = TallCfg<T, NP>;
    using type = AccTile<T, Cfg::R, Cfg::CN, Cfg::BV>;
};
template <int NP>
struct TallAcc<float, NP> {
    using Cfg = TallCfg<float, NP>;
    using type = typename std::conditional<(Cfg::CN >= 2), AccTilePairs<Cfg::R, Cfg::CN>,
                                           AccTile<float, Cfg::R, Cfg::CN, Cfg::BV>>::type;
};

// One block's work item (m-slab `slab`, k range `split`) with A described by
// the tensor map *tmA (a kernel parameter); the body of the single-problem
// kernel and of the grouped kernel.
template <typename T, int NP>
__device__ __forceinline__ void tall_tma_block(const CUtensorMap *tmA, const TallArgs &a, int64_t slab,
                                               int split) {
    using Cfg = TallCfg<T, NP>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sA = reinterpret_cast<T *>(smem_raw);
    T *sB = sA + Cfg::STAGES * Cfg::A_STAGE;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + Cfg::DATA_BYTES);
    uint64_t *empty = full + Cfg::STAGES;
    unsigned *flag = reinterpret_cast<unsigned *>(empty + Cfg::STAGES);
    unsigned *abort_flag = flag + 1;

    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int64_t k0 = (int64_t)split * a.kchunk;
    const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;
    const int iters = (int)((k1 - k0) / Cfg::BKS);

    if (threadIdx.x == 0) {
        prefetch_tmap(tmA);
        for (int s = 0; s < Cfg::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], Cfg::NWARPS);
        }
        *abort_flag = 0u;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == Cfg::NWARPS) {
        // ---------------- producer warp: one elected lane issues the copies
        if (lane == 0) {
            const uint64_t pol_a = policy_evict_first();
            const uint64_t pol_b = policy_evict_last();
            const T *Bp = static_cast<const T *>(a.Bp);
            for (int it = 0; it < iters; ++it) {
                const int st = it % Cfg::STAGES;
                if (it >= Cfg::STAGES) {
                    if (!mbar_wait_bounded(&empty[st], ((it / Cfg::STAGES) & 1) ^ 1)) {
                        atomicOr(a.status, kDevErrTimeout);
                        break;
                    }
                }
                const int64_t kk = k0 + (int64_t)it * Cfg::BKS;
                mbar_arrive_expect_tx(&full[st], Cfg::STAGE_BYTES);
                tma_load_2d(sA + st * Cfg::A_STAGE, tmA, (int32_t)(slab * Cfg::BM), (int32_t)kk,
                            &full[st], pol_a);
                bulk_load(sB + st * Cfg::B_STAGE, Bp + kk * NP, Cfg::B_STAGE * (int)sizeof(T),
                          &full[st], pol_b);
            }
        }
        return;
    }

    // ---------------- consumer warps
    const int wm = warp % Cfg::WM;
    const int wk = warp / Cfg::WM;
    const int g = lane / Cfg::LR;
    const int lr = lane % Cfg::LR;
    const int rloc = wm * Cfg::WROWS + lr * Cfg::RV;  // first local row of this thread
    const int cloc = g * Cfg::CN;                    // first column of this thread

    typename TallAcc<T, NP>::type acc;
    acc.zero();

    bool ok = true;
    for (int it = 0; it < iters; ++it) {
        const int st = it % Cfg::STAGES;
        if (!mbar_wait_bounded(&full[st], (it / Cfg::STAGES) & 1)) {
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
        release_reads_to_async_copy();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
    if (!ok && lane == 0) {
        atomicOr(a.status, kDevErrTimeout);
        atomicOr(abort_flag, 1u);
    }

    // all stages consumed (or abandoned): every consumer warp gets here, since
    // each wait above is bounded, so the named barrier cannot hang
    named_barrier(1, Cfg::CONSUMERS);
    if (*abort_flag != 0u) return;  // tile not written; the host sees TSMM_ERR_TIMEOUT
    T *red = sA;
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

template <typename T, int NP>
__global__ void __launch_bounds__(TallCfg<T, NP>::THREADS, TallCfg<T, NP>::RESIDENT)
    tall_tma_kernel(const __grid_constant__ CUtensorMap tmA, const TallArgs a) {
    tall_tma_block<T, NP>(&tmA, a, blockIdx.x, (int)blockIdx.y);
}

// Same decomposition without a tensor map, for an A that one cannot describe
// (its base or its column stride lda*sizeof(T) not a multiple of 16 bytes, as
// for a column-major A with lda = m and m not a multiple of 4 -- most of a
// random serving mix).  The structure is the TMA kernel's: consumer warps, a
// producer warp and a ring of mbarrier-guarded stages of BM rows x BKS columns.
// Each of the producer's 32 lanes moves one column of a stage with one bulk
// copy (cp.async.bulk, the tensor copy's engine): a column of A may start at
// any element address, so it is copied together with the 16-byte-aligned span
// around its rows (column_span_bytes) and sits in shared memory at its own
// offset within 16 bytes (d elements into its slot).  Lane 0 posts the bytes of
// the whole stage with its arrival before any lane issues its copy.  Columns
// beyond k are zero-filled; rows beyond m hold whatever the span or an earlier
// stage left (their results are never stored).  Consumers read the rows at the
// column's offset.  B's packed rows come in one bulk copy per stage.  The thread
// tiles, reduction and split-K finish are the TMA kernel's.
template <typename T, int NP>
struct AsyncCfg {
    using Cfg = TallCfg<T, NP>;
    static constexpr int V = 16 / (int)sizeof(T);        // elements per 16 bytes
    static constexpr int APAD = Cfg::BM + 2 * V;          // a column's slot: offset + rows + the tail chunk
    static constexpr int A_STAGE = Cfg::BKS * APAD;
    static constexpr int STAGE_BYTES = (A_STAGE + Cfg::B_STAGE) * (int)sizeof(T);
    // all the shared memory the resident blocks can have (228 KB per SM, 1 KB per block reserved)
    static constexpr int BUDGET = Cfg::RESIDENT >= 3 ? 74 * 1024 : 112 * 1024;
    static constexpr int STAGES_RAW = BUDGET / STAGE_BYTES;
    static constexpr int STAGES = STAGES_RAW < 2 ? 2 : (STAGES_RAW > 6 ? 6 : STAGES_RAW);
    static constexpr int RED_BYTES = Cfg::RED * (int)sizeof(T);
    static constexpr int DATA_BYTES =
        STAGES * STAGE_BYTES > RED_BYTES ? STAGES * STAGE_BYTES : RED_BYTES;
    static constexpr int SMEM = DATA_BYTES + 2 * STAGES * 8 + 16;
    static_assert(Cfg::BKS == 32, "one producer lane per column");
    static_assert(Cfg::KPW % V == 0, "a warp's first stage column is a multiple of V");
    static_assert(Cfg::RESIDENT * (SMEM + 1024) <= 228 * 1024, "resident blocks per SM");
};

// f(std::integral_constant<int, I>{}) for I = B .. E-1, unrolled at compile time.
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// An FP32 thread's rows of one stage column whose rows start D elements past
// the 16-byte-aligned slot start.  rloc and the group stride are multiples of
// 4, so every group of 4 rows sits D elements past a 16-byte boundary and takes
// one 16-byte load (D = 0), two 8-byte loads (D = 2) or 4 + 8 + 4 bytes (D
// odd): the same shared-memory wavefronts as element loads, in a quarter to
// three quarters of the instructions.
template <typename Cfg, int D>
__device__ __forceinline__ Vec<float, Cfg::R> load_rows_at(const float *slot, int rloc) {
    static_assert(Cfg::RV == 4, "groups of 4 rows");
    Vec<float, Cfg::R> v;
#pragma unroll
    for (int gi = 0; gi < Cfg::RG; ++gi) {
        const float *p = slot + D + rloc + gi * Cfg::GSTRIDE;
        float x[4];
        if constexpr (D == 0) {
            const float4 q = *reinterpret_cast<const float4 *>(p);
            x[0] = q.x, x[1] = q.y, x[2] = q.z, x[3] = q.w;
        } else if constexpr (D == 2) {
            const float2 q0 = *reinterpret_cast<const float2 *>(p);
            const float2 q1 = *reinterpret_cast<const float2 *>(p + 2);
            x[0] = q0.x, x[1] = q0.y, x[2] = q1.x, x[3] = q1.y;
        } else {
            const float2 q = *reinterpret_cast<const float2 *>(p + 1);  // 8-byte aligned for D = 1, 3
            x[0] = p[0], x[1] = q.x, x[2] = q.y, x[3] = p[3];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) v.v[gi * 4 + r] = x[r];
    }
    return v;
}

// LV >= 0 (FP32 widths of 16 and more, chosen on the host by
// async_load_variant): A's base is 16-byte aligned and lda = LV mod 4, so
// column c of a stage sits (c * LV) mod 4 elements into its slot, known at
// compile time, and its rows are read with load_rows_at.  LV = -1: any A, the
// offsets computed at run time and the rows read element by element.
template <typename T, int NP, int LV = -1>
__device__ __forceinline__ void tall_async_block(const TallArgs &a, int64_t slab, int split) {
    using Cfg = TallCfg<T, NP>;
    using AC = AsyncCfg<T, NP>;
    constexpr int S = AC::STAGES;
    constexpr int V = AC::V;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sA = reinterpret_cast<T *>(smem_raw);
    T *sB = sA + S * AC::A_STAGE;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + AC::DATA_BYTES);
    uint64_t *empty = full + S;
    unsigned *flag = reinterpret_cast<unsigned *>(empty + S);
    unsigned *abort_flag = flag + 1;

    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int64_t k0 = (int64_t)split * a.kchunk;
    const int64_t k1 = (k0 + a.kchunk < a.kp) ? k0 + a.kchunk : a.kp;
    const int iters = (int)((k1 - k0) / Cfg::BKS);
    const int64_t i0 = slab * Cfg::BM;
    const int rows = (int)((a.m - i0 < Cfg::BM) ? a.m - i0 : Cfg::BM);  // rows of this slab inside A
    const T *A = static_cast<const T *>(a.A);
    // offset within 16 bytes of element (i0, p): (d0 + p*lda) mod V
    const int d0 = (int)(((reinterpret_cast<uintptr_t>(A) / sizeof(T)) + (uint64_t)i0) & (V - 1));
    const int ldv = (int)((uint64_t)a.lda & (V - 1));
    auto col_off = [&](int64_t p) { return (d0 + (int)((uint64_t)p & (V - 1)) * ldv) & (V - 1); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);  // lane 0 of the producer warp
            mbar_init(&empty[s], Cfg::NWARPS);
        }
        *abort_flag = 0u;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == Cfg::NWARPS) {
        // ---------------- producer warp: lane c moves column c of each stage
        const uint64_t pol_a = policy_evict_first();
        const uint64_t pol_b = policy_evict_last();
        const T *Bp = static_cast<const T *>(a.Bp);
        for (int it = 0; it < iters; ++it) {
            const int st = it % S;
            if (it >= S) {
                const bool got = mbar_wait_bounded(&empty[st], ((it / S) & 1) ^ 1);
                if (!__all_sync(0xffffffffu, got)) {
                    if (lane == 0) atomicOr(a.status, kDevErrTimeout);
                    break;
                }
            }
            const int64_t kk = k0 + (int64_t)it * Cfg::BKS;
            const int64_t p = kk + lane;
            const int d = col_off(p);
            T *slot0 = sA + st * AC::A_STAGE + lane * AC::APAD;  // row r at slot0[d + r]
            const uint32_t bytes = p < a.k ? column_span_bytes<T>(rows, d) : 0u;
            if (p >= a.k) {
                // beyond k: zeros, as B's padding (the whole slot)
                for (int r = 0; r < AC::APAD; r += V) *reinterpret_cast<uint4 *>(slot0 + r) = make_uint4(0, 0, 0, 0);
                fence_proxy_async_smem();  // before later copies into the slot
            }
            // the stage's bytes are expected once, by lane 0's arrival, before any
            // copy of it is issued; the zero stores above precede that arrival
            const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
            __syncwarp();
            if (lane == 0) {
                mbar_arrive_expect_tx(&full[st], Cfg::B_STAGE * (uint32_t)sizeof(T) + total);
                bulk_load(sB + st * Cfg::B_STAGE, Bp + kk * NP, Cfg::B_STAGE * (int)sizeof(T), &full[st], pol_b);
            }
            __syncwarp();
            if (p < a.k) bulk_load(slot0, A + i0 + p * a.lda - d, bytes, &full[st], pol_a);
        }
        return;
    }

    // ---------------- consumer warps
    const int wm = warp % Cfg::WM;
    const int wk = warp / Cfg::WM;
    const int g = lane / Cfg::LR;
    const int lr = lane % Cfg::LR;
    const int rloc = wm * Cfg::WROWS + lr * Cfg::RV;
    const int cloc = g * Cfg::CN;
    typename TallAcc<T, NP>::type acc;
    acc.zero();
    // every stage starts at a multiple of BKS (k splits are whole stages), so a
    // column's offset within 16 bytes depends only on its index mod V
    int doff[V];
#pragma unroll
    for (int j = 0; j < V; ++j) doff[j] = col_off(k0 + j);

    static_assert(LV < 0 || (sizeof(T) == 4 && NP >= 16), "compile-time offsets: FP32 widths of 16 and more");
    bool ok = true;
    for (int it = 0; it < iters; ++it) {
        const int st = it % S;
        if (!mbar_wait_bounded(&full[st], (it / S) & 1)) {
            ok = false;
            break;
        }
        const T *As = sA + st * AC::A_STAGE;
        const T *Bs = sB + st * Cfg::B_STAGE;
        static_for<0, Cfg::KPW>([&](auto c_tag) {
            constexpr int c = decltype(c_tag)::value;
            const int col = wk * Cfg::KPW + c;  // col = c mod V: KPW % V == 0
            Vec<T, Cfg::R> av;
            if constexpr (LV >= 0) {
                av = load_rows_at<Cfg, (c * LV) % V>(As + col * AC::APAD, rloc);
            } else {
                const T *colp = As + col * AC::APAD + doff[c % V];
#pragma unroll
                for (int r = 0; r < Cfg::R; ++r) av.v[r] = colp[Cfg::row(rloc, r)];
            }
            acc.fma_column(av, Bs + col * NP + cloc);
        });
        release_reads_to_async_copy();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
    if (!ok && lane == 0) {
        atomicOr(a.status, kDevErrTimeout);
        atomicOr(abort_flag, 1u);
    }
    // every consumer warp gets here (each wait above is bounded)
    named_barrier(1, Cfg::CONSUMERS);
    if (*abort_flag != 0u) return;  // tile not written; the host sees TSMM_ERR_TIMEOUT
    T *red = sA;
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

template <typename T, int NP, int LV>
__global__ void __launch_bounds__(TallCfg<T, NP>::THREADS, TallCfg<T, NP>::RESIDENT)
    tall_async_kernel(const TallArgs a) {
    tall_async_block<T, NP, LV>(a, blockIdx.x, (int)blockIdx.y);
}

template <typename T, int NP>
cudaError_t launch_tall_tma_t(const CUtensorMap *tmap, const TallArgs &a, cudaStream_t s) {
    using Cfg = TallCfg<T, NP>;
    {
        const cudaError_t e =
            ensure_smem_limit(reinterpret_cast<const void *>(tall_tma_kernel<T, NP>), Cfg::SMEM);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)a.slabs, (unsigned)a.splits);
    tall_tma_kernel<T, NP><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(*tmap, a);
    return cudaGetLastError();
}

template <typename T, int NP, int LV>
cudaError_t launch_tall_async_lv(const TallArgs &a, cudaStream_t s) {
    const int smem = AsyncCfg<T, NP>::SMEM;
    {
        const cudaError_t e =
            ensure_smem_limit(reinterpret_cast<const void *>(tall_async_kernel<T, NP, LV>), smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)a.slabs, (unsigned)a.splits);
    tall_async_kernel<T, NP, LV><<<grid, TallCfg<T, NP>::THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// Calls f(std::integral_constant<int, LV>) for the load form lv of
// async_load_variant (only -1 where no other form is instantiated).
template <typename T, int NP, typename F>
auto with_load_variant(int lv, F &&f) {
    if constexpr (sizeof(T) == 4 && NP >= 16) {
        switch (lv) {
            case 0:
                return f(std::integral_constant<int, 0>{});
            case 1:
                return f(std::integral_constant<int, 1>{});
            case 2:
                return f(std::integral_constant<int, 2>{});
            case 3:
                return f(std::integral_constant<int, 3>{});
            default:
                break;
        }
    }
    return f(std::integral_constant<int, -1>{});
}

template <typename T, int NP>
cudaError_t launch_tall_async_t(const TallArgs &a, cudaStream_t s) {
    const int lv = async_load_variant(sizeof(T) == 4, NP, a.A, a.lda);
    return with_load_variant<T, NP>(lv, [&](auto lv_tag) {
        return launch_tall_async_lv<T, NP, decltype(lv_tag)::value>(a, s);
    });
}

// Per-width dispatch of the two regime (i) kernels.  Each dtype's TMA and
// bulk-copy kernels are instantiated in translation units of their own
// (tsmm_tall_<dtype>.cu, tsmm_tall_async_<dtype>.cu) so that they compile in
// parallel.
#define TSMM_FOR_TALL_WIDTHS(X) X(1) X(2) X(4) X(8) X(16) X(24) X(32) X(48) X(64)

template <typename T>
cudaError_t launch_tall_tma_dispatch(int np, const CUtensorMap *tmap, const TallArgs &a, cudaStream_t s) {
#define TSMM_TALL_CASE(NPV) \
    case NPV:               \
        return launch_tall_tma_t<T, NPV>(tmap, a, s);
    switch (np) {
        TSMM_FOR_TALL_WIDTHS(TSMM_TALL_CASE)
        default:
            return cudaErrorInvalidValue;
    }
#undef TSMM_TALL_CASE
}

template <typename T>
cudaError_t launch_tall_async_dispatch(int np, const TallArgs &a, cudaStream_t s) {
#define TSMM_TALL_CASE(NPV) \
    case NPV:               \
        return launch_tall_async_t<T, NPV>(a, s);
    switch (np) {
        TSMM_FOR_TALL_WIDTHS(TSMM_TALL_CASE)
        default:
            return cudaErrorInvalidValue;
    }
#undef TSMM_TALL_CASE
}

cudaError_t launch_tall_async_f32(int np, const TallArgs &a, cudaStream_t s);  // tsmm_tall_async_f32.cu
cudaError_t launch_tall_async_f64(int np, const TallArgs &a, cudaStream_t s);  // tsmm_tall_async_f64.cu

}  // namespace tsmm
