// Regime (ii) kernel: C[m x n] = alpha * A[m x k] * B[k x n] + beta * C0 with
// k <= 128 and m, n large (a rank-k update; TSMM with the skinny operand on
// the inner dimension, Section I).  The whole k extent of a C tile is
// contracted on chip, so the kernel streams C0 in and C out exactly once:
// the traffic floor of this shape is the 2*m*n output read/write, not A or B.
//
// Thread block: 256 consumer threads own a BMT x 64 tile of C.  Each thread
// keeps a (2*VEC) x 4 register tile: two row groups {tm*VEC + r} and
// {BMT/2 + tm*VEC + r} (one 16-byte vector each) and the columns {tn*4 + c},
// so that both the shared-memory operand reads and the global C stores of a
// half-warp cover one contiguous 256-byte run.
//
// TMA path (A 16-byte aligned with lda*s a multiple of 16): one producer warp
// streams k in chunks of KC = 32 -- a 2-D tensor copy of A (BMT x KC) and a
// bulk copy of the packed B rows (KC x 64) per chunk -- through a ring of
// STAGES mbarrier-guarded buffers.  For the output-bound small-k shapes
// (PREFETCH_C0) it also fetches the whole C0 tile with one tensor copy at block
// start, so the C0 read overlaps the A/B traffic and the products; otherwise
// the epilogue loads C0 in batches ahead of its stores.  An A that a tensor
// map cannot describe is first copied into an aligned scratch buffer by the
// host-side dispatch (tsmm_execute); the plain-load kernel below covers it only
// when no scratch can be had.
#include <type_traits>

#include "tsmm_device.cuh"
#include "tsmm_internal.h"

namespace tsmm {

template <typename T>
struct RankCfg {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int TM = 2 * VEC;         // rows per thread (two row groups)
    static constexpr int TN = 4;               // columns per thread
    static constexpr int BMT = 16 * TM;        // 128 (f32) / 64 (f64)
    static constexpr int BNT = kRankNT;        // 64
    static constexpr int KC = 32;
    static constexpr int CONSUMERS = 256;
    static constexpr int A_CHUNK = BMT * KC;   // elements
    static constexpr int B_CHUNK = KC * BNT;
    static constexpr int C_TILE = BMT * BNT;
    static_assert(BNT == 16 * TN, "tile width");
};

// Register tile of one thread: rows {rg*BMT/2 + tm*VEC + r} (rg = 0, 1;
// r < VEC) x columns {tn*4 + c} (c < 4); row index R = rg*VEC + r.  Each
// product is an IEEE fma in the working precision.  The FP32 tile keeps row
// pairs as float2 and uses the packed FP32x2 fma (same roundings as two scalar
// fmas, half the issue slots), with each B value duplicated into both halves.
template <typename T>
struct RankAcc {
    using Cfg = RankCfg<T>;
    T v[Cfg::TM][Cfg::TN];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < Cfg::TM; ++r)
#pragma unroll
            for (int c = 0; c < Cfg::TN; ++c) v[r][c] = T(0);
    }
    // one k-chunk from shared memory (As: [KC][BMT], Bs: [KC][BNT])
    __device__ __forceinline__ void chunk(const T *As, const T *Bs, int kcnt, int tm, int tn) {
        constexpr int V = Cfg::VEC;
#pragma unroll 4
        for (int pc = 0; pc < kcnt; ++pc) {
            const Vec<T, V> a0 = ld_vec<T, V>(As + pc * Cfg::BMT + tm * V);
            const Vec<T, V> a1 = ld_vec<T, V>(As + pc * Cfg::BMT + Cfg::BMT / 2 + tm * V);
            const Vec<T, 4> b0 = *reinterpret_cast<const Vec<T, 4> *>(Bs + pc * Cfg::BNT + tn * 4);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
#pragma unroll
                for (int r = 0; r < V; ++r) {
                    v[r][c] = fma(a0.v[r], b0.v[c], v[r][c]);
                    v[V + r][c] = fma(a1.v[r], b0.v[c], v[V + r][c]);
                }
            }
        }
    }
    __device__ __forceinline__ T get(int r, int c) const { return v[r][c]; }
    // start from C0 given in the epilogue's layout (c0v[c][rg].v[r] is row rg*VEC + r)
    __device__ __forceinline__ void init(const Vec<T, Cfg::VEC> (&c0v)[4][2]) {
#pragma unroll
        for (int c = 0; c < Cfg::TN; ++c)
#pragma unroll
            for (int rg = 0; rg < 2; ++rg)
#pragma unroll
                for (int r = 0; r < Cfg::VEC; ++r) v[rg * Cfg::VEC + r][c] = c0v[c][rg].v[r];
    }
};

template <>
struct RankAcc<float> {
    using Cfg = RankCfg<float>;
    float2 v[Cfg::TM / 2][Cfg::TN];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < Cfg::TM / 2; ++r)
#pragma unroll
            for (int c = 0; c < Cfg::TN; ++c) v[r][c] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void chunk(const float *As, const float *Bs, int kcnt, int tm, int tn) {
#pragma unroll 4
        for (int pc = 0; pc < kcnt; ++pc) {
            const float4 a0 = *reinterpret_cast<const float4 *>(As + pc * Cfg::BMT + tm * 4);
            const float4 a1 = *reinterpret_cast<const float4 *>(As + pc * Cfg::BMT + Cfg::BMT / 2 + tm * 4);
            const float4 b = *reinterpret_cast<const float4 *>(Bs + pc * Cfg::BNT + tn * 4);
            const float2 ap[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w),
                                  make_float2(a1.x, a1.y), make_float2(a1.z, a1.w)};
            const float2 bd[4] = {make_float2(b.x, b.x), make_float2(b.y, b.y),
                                  make_float2(b.z, b.z), make_float2(b.w, b.w)};
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int rp = 0; rp < 4; ++rp) v[rp][c] = __ffma2_rn(ap[rp], bd[c], v[rp][c]);
        }
    }
    __device__ __forceinline__ float get(int r, int c) const {
        return (r & 1) ? v[r / 2][c].y : v[r / 2][c].x;
    }
    __device__ __forceinline__ void init(const Vec<float, Cfg::VEC> (&c0v)[4][2]) {
#pragma unroll
        for (int c = 0; c < Cfg::TN; ++c)
#pragma unroll
            for (int rg = 0; rg < 2; ++rg)
#pragma unroll
                for (int r = 0; r < Cfg::VEC; r += 2)
                    v[(rg * Cfg::VEC + r) / 2][c] = make_float2(c0v[c][rg].v[r], c0v[c][rg].v[r + 1]);
    }
};

// Epilogue C = alpha*acc + beta*C0 in two phases so that C0 can come from a
// shared-memory buffer that is released between them.  Phase 1 gathers this
// thread's C0 values -- from the tile sC ([BNT][BMT], as the tensor copy lays it
// out) when given, else from global memory, all loads ahead of any store so
// they do not wait behind stores to the same array; phase 2 stores.
// The 16 bytes of consecutive elements at p, where p sits D elements past a
// 16-byte boundary (D known at compile time): one 16-byte access for D = 0,
// else the widest aligned pieces -- for FP32 two 8-byte accesses (D = 2) or
// 4 + 8 + 4 bytes (D odd), for FP64 two 8-byte accesses.
template <typename T, int D>
__device__ __forceinline__ Vec<T, 16 / sizeof(T)> ld_group(const T *p) {
    constexpr int V = 16 / (int)sizeof(T);
    Vec<T, V> v;
    if constexpr (D == 0) {
        v = ld_vec<T, V>(p);
    } else if constexpr (sizeof(T) == 4 && D == 2) {
        const float2 q0 = *reinterpret_cast<const float2 *>(p);
        const float2 q1 = *reinterpret_cast<const float2 *>(p + 2);
        v.v[0] = q0.x, v.v[1] = q0.y, v.v[2] = q1.x, v.v[3] = q1.y;
    } else if constexpr (sizeof(T) == 4) {
        const float2 q = *reinterpret_cast<const float2 *>(p + 1);
        v.v[0] = p[0], v.v[1] = q.x, v.v[2] = q.y, v.v[3] = p[3];
    } else {
#pragma unroll
        for (int r = 0; r < V; ++r) v.v[r] = p[r];
    }
    return v;
}
template <typename T, int D>
__device__ __forceinline__ void st_group(T *p, const Vec<T, 16 / sizeof(T)> &v) {
    constexpr int V = 16 / (int)sizeof(T);
    if constexpr (D == 0) {
        st_vec<T, V>(p, v);
    } else if constexpr (sizeof(T) == 4 && D == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v.v[0], v.v[1]);
        *reinterpret_cast<float2 *>(p + 2) = make_float2(v.v[2], v.v[3]);
    } else if constexpr (sizeof(T) == 4) {
        p[0] = v.v[0];
        *reinterpret_cast<float2 *>(p + 1) = make_float2(v.v[1], v.v[2]);
        p[3] = v.v[3];
    } else {
#pragma unroll
        for (int r = 0; r < V; ++r) p[r] = v.v[r];
    }
}

// f(std::integral_constant<int, I>{}) for I = B .. E-1, unrolled at compile time.
template <int B, int E, typename F>
__device__ __forceinline__ void rank_static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        rank_static_for<B + 1, E>(f);
    }
}

// Epilogue of the 8 x 4-tile kernels.  LVC (the form of C's accesses): -1 for
// any C (element accesses), else C's base is 16-byte aligned and ldc = LVC mod
// V, so the thread's group of V rows in column c (c = column mod 4, the same
// for the whole warp) sits (c * LVC) mod V elements past a 16-byte boundary and
// is read and written with ld_group / st_group.  LVC = 0 is the aligned case.
template <typename T>
struct RankEpilogue {
    using Cfg = RankCfg<T>;
    static constexpr int V = Cfg::VEC;
    Vec<T, V> c0v[4][2];

    template <int LVC>
    __device__ __forceinline__ void load(const RankArgs &a, int64_t i0, int64_t tile, int tm, int tn,
                                         const T *sC, T beta) {
        const T *C = static_cast<const T *>(a.C);
        rank_static_for<0, 4>([&](auto c_tag) {
            constexpr int c = decltype(c_tag)::value;
            const int jl = tn * 4 + c;
            const int64_t j = tile * Cfg::BNT + jl;
#pragma unroll
            for (int rg = 0; rg < 2; ++rg) {
                const int il = rg * (Cfg::BMT / 2) + tm * V;
                const int64_t i = i0 + il;
#pragma unroll
                for (int r = 0; r < V; ++r) c0v[c][rg].v[r] = T(0);
                if (beta == T(0) || j >= a.n) continue;
                if (sC) {
                    c0v[c][rg] = ld_vec<T, V>(sC + jl * Cfg::BMT + il);
                } else if (LVC >= 0 && i + V <= a.m) {
                    c0v[c][rg] = ld_group<T, LVC >= 0 ? (c * LVC) % V : 0>(C + i + j * a.ldc);
                } else {
#pragma unroll
                    for (int r = 0; r < V; ++r)
                        if (i + r < a.m) c0v[c][rg].v[r] = C[i + r + j * a.ldc];
                }
            }
        });
    }

    // alpha == 1 is a separate code path (the test is uniform), so the
    // epilogue issues no multiply by 1 and no per-element select: at small k
    // in FP64 the epilogue's arithmetic shares the FP64 pipe with the k
    // products of each output.
    template <int LVC>
    __device__ __forceinline__ void store(const RankAcc<T> &acc, const RankArgs &a, int64_t i0,
                                          int64_t tile, int tm, int tn, T alpha, T beta) const {
        if (alpha == T(1)) store_t<true, LVC>(acc, a, i0, tile, tm, tn, alpha, beta);
        else store_t<false, LVC>(acc, a, i0, tile, tm, tn, alpha, beta);
    }

    template <bool ALPHA1, int LVC>
    __device__ __forceinline__ void store_t(const RankAcc<T> &acc, const RankArgs &a, int64_t i0,
                                            int64_t tile, int tm, int tn, T alpha, T beta) const {
        T *C = static_cast<T *>(a.C);
        rank_static_for<0, 4>([&](auto c_tag) {
            constexpr int c = decltype(c_tag)::value;
            const int64_t j = tile * Cfg::BNT + tn * 4 + c;
            if (j >= a.n) return;
#pragma unroll
            for (int rg = 0; rg < 2; ++rg) {
                const int64_t i = i0 + rg * (Cfg::BMT / 2) + tm * V;
                Vec<T, V> o;
#pragma unroll
                for (int r = 0; r < V; ++r) {
                    const T x = acc.get(rg * V + r, c);
                    o.v[r] = ALPHA1 ? x : alpha * x;  // alpha*x == x exactly when alpha is 1
                    if (beta != T(0)) o.v[r] = fma(beta, c0v[c][rg].v[r], o.v[r]);
                }
                T *cp = C + i + j * a.ldc;
                if (LVC >= 0 && i + V <= a.m) {
                    st_group<T, LVC >= 0 ? (c * LVC) % V : 0>(cp, o);
                } else {
#pragma unroll
                    for (int r = 0; r < V; ++r)
                        if (i + r < a.m) cp[r] = o.v[r];
                }
            }
        });
    }
};

template <typename T, int STAGES, bool PREFETCH_C0>
struct RankTmaCfg {
    using Cfg = RankCfg<T>;
    static constexpr int STAGE_ELEMS = Cfg::A_CHUNK + Cfg::B_CHUNK;
    static constexpr int CBUF = PREFETCH_C0 ? 2 : 0;   // double-buffered C0 tiles
    static constexpr int DATA_BYTES = (STAGES * STAGE_ELEMS + CBUF * Cfg::C_TILE) * (int)sizeof(T);
    static constexpr int NBAR = 2 * STAGES + 2 * CBUF;
    static constexpr int SMEM = DATA_BYTES + NBAR * 8 + 16;
    static constexpr int THREADS = Cfg::CONSUMERS + 32;
    static constexpr int RESIDENT = 2;                  // blocks per SM (registers, shared memory)
};

// Persistent: each block walks tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// (tile t covers rows (t % mtiles)*BMT and columns (t / mtiles)*BNT).  The
// producer warp runs ahead of the consumers by up to STAGES k-chunks and, with
// PREFETCH_C0, by one C0 tile, so the next tile's loads overlap this tile's
// products and stores.
template <typename T, int STAGES, bool PREFETCH_C0, bool C0_INIT, int LVC>
__global__ void __launch_bounds__(RankCfg<T>::CONSUMERS + 32, 2)
    rankk_tma_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmC, const RankArgs a, unsigned *status) {
    using Cfg = RankCfg<T>;
    using TC = RankTmaCfg<T, STAGES, PREFETCH_C0>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sStage = reinterpret_cast<T *>(smem_raw);
    T *sC = sStage + STAGES * TC::STAGE_ELEMS;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + TC::DATA_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *cfull = empty + STAGES;  // CBUF entries
    uint64_t *cempty = cfull + TC::CBUF;

    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int64_t mtiles = (a.m + Cfg::BMT - 1) / Cfg::BMT;
    const int64_t ntiles_total = mtiles * ((a.n + Cfg::BNT - 1) / Cfg::BNT);
    const int nchunks = (int)((a.k + Cfg::KC - 1) / Cfg::KC);
    const bool want_c0 = PREFETCH_C0 && a.beta != 0.0;

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmA);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], Cfg::CONSUMERS / 32);
        }
        for (int b = 0; b < TC::CBUF; ++b) {
            mbar_init(&cfull[b], 1);
            mbar_init(&cempty[b], Cfg::CONSUMERS / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == Cfg::CONSUMERS / 32) {
        if (lane == 0) {
            const uint64_t pol_stream = policy_evict_first();
            const uint64_t pol_keep = policy_evict_last();
            int64_t g = 0;  // k-chunks issued so far by this block
            int j = 0;      // tiles issued so far by this block
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles_total && ok; t += gridDim.x, ++j) {
                int64_t tile, mt;
                udivmod(t, mtiles, tile, mt);
                const int64_t i0 = mt * Cfg::BMT;
                if (want_c0) {
                    const int b = j % 2;
                    if (j >= 2 && !mbar_wait_bounded(&cempty[b], ((j / 2) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    T *dst = sC + b * Cfg::C_TILE;
                    mbar_arrive_expect_tx(&cfull[b], Cfg::C_TILE * (int)sizeof(T));
                    tma_load_2d(dst, &tmC, (int32_t)i0, (int32_t)(tile * Cfg::BNT), &cfull[b],
                                pol_stream);
                }
                const T *Bt = static_cast<const T *>(a.Bp) + tile * a.kp * Cfg::BNT;
                for (int c = 0; c < nchunks; ++c, ++g) {
                    const int st = (int)(g % STAGES);
                    if (g >= STAGES && !mbar_wait_bounded(&empty[st], (int)((g / STAGES) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    const int64_t kc = (int64_t)c * Cfg::KC;
                    const int brows = (int)((a.kp - kc < Cfg::KC) ? a.kp - kc : Cfg::KC);
                    T *sA = sStage + st * TC::STAGE_ELEMS;
                    T *sB = sA + Cfg::A_CHUNK;
                    mbar_arrive_expect_tx(&full[st],
                                          (Cfg::A_CHUNK + brows * Cfg::BNT) * (int)sizeof(T));
                    tma_load_2d(sA, &tmA, (int32_t)i0, (int32_t)kc, &full[st], pol_keep);
                    bulk_load(sB, Bt + kc * Cfg::BNT, brows * Cfg::BNT * (int)sizeof(T), &full[st],
                              pol_keep);
                }
            }
            if (!ok) atomicOr(status, kDevErrTimeout);
        }
        return;
    }

    const int tid = threadIdx.x;
    const int tm = tid % 16;
    const int tn = tid / 16;
    const T ealpha = static_cast<T>(a.alpha);  // converted once, not per tile
    const T ebeta = static_cast<T>(a.beta);
    // C0_INIT (FP64, alpha = beta = 1, C0 prefetched a tile ahead): the
    // accumulators start from C0, so the epilogue has no arithmetic left -- at
    // small k the k fmas per output and the epilogue's one share the FP64 pipe.
    // The sum is C0 + a1*b1 + ... in fma order: another order of the same terms.
    static_assert(!C0_INIT || PREFETCH_C0, "C0 comes from the prefetched tile");
    int64_t g = 0;
    int j = 0;
    for (int64_t t = blockIdx.x; t < ntiles_total; t += gridDim.x, ++j) {
        int64_t tile, mt;
        udivmod(t, mtiles, tile, mt);
        const int64_t i0 = mt * Cfg::BMT;
        RankAcc<T> acc;
        bool ok = true;
        if constexpr (C0_INIT) {
            const int b = j % 2;
            if (!mbar_wait_bounded(&cfull[b], (j / 2) & 1)) {
                if (lane == 0) atomicOr(status, kDevErrTimeout);
                return;  // this warp's part of the tile is not written; the host sees TSMM_ERR_TIMEOUT
            }
            RankEpilogue<T> e0;
            e0.template load<LVC>(a, i0, tile, tm, tn, sC + b * Cfg::C_TILE, ebeta);
            release_reads_to_async_copy();
            __syncwarp();
            if (lane == 0) mbar_arrive(&cempty[b]);  // C0 buffer b may be refilled
            acc.init(e0.c0v);
        } else {
            acc.zero();
        }
        for (int c = 0; c < nchunks; ++c, ++g) {
            const int st = (int)(g % STAGES);
            if (!mbar_wait_bounded(&full[st], (int)((g / STAGES) & 1))) {
                ok = false;
                break;
            }
            const int64_t kc = (int64_t)c * Cfg::KC;
            const int kcnt = (int)((a.k - kc < Cfg::KC) ? a.k - kc : Cfg::KC);
            const T *sA = sStage + st * TC::STAGE_ELEMS;
            acc.chunk(sA, sA + Cfg::A_CHUNK, kcnt, tm, tn);
            release_reads_to_async_copy();
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
        if constexpr (C0_INIT) {
            if (!ok) {
                if (lane == 0) atomicOr(status, kDevErrTimeout);
                return;
            }
            RankEpilogue<T>().template store<LVC>(acc, a, i0, tile, tm, tn, T(1), T(0));  // C0 is in acc
            continue;
        }
        RankEpilogue<T> ep;
        const int b = j % 2;
        if (ok && want_c0 && !mbar_wait_bounded(&cfull[b], (j / 2) & 1)) ok = false;
        if (!ok) {
            if (lane == 0) atomicOr(status, kDevErrTimeout);
            return;  // this warp's part of the tile is not written; the host sees TSMM_ERR_TIMEOUT
        }
        ep.template load<LVC>(a, i0, tile, tm, tn, want_c0 ? sC + b * Cfg::C_TILE : nullptr, ebeta);
        if (want_c0) {
            release_reads_to_async_copy();
            __syncwarp();
            if (lane == 0) mbar_arrive(&cempty[b]);  // C0 buffer b may be refilled
        }
        ep.template store<LVC>(acc, a, i0, tile, tm, tn, ealpha, ebeta);
    }
}

// Plain-load kernel for an A that a tensor map cannot describe.
template <typename T, int LVC>
__global__ void __launch_bounds__(256, 2) rankk_plain_kernel(const RankArgs a, bool vec_a) {
    using Cfg = RankCfg<T>;
    constexpr int V = Cfg::VEC;
    constexpr int BMT = Cfg::BMT;
    constexpr int BNT = Cfg::BNT;
    constexpr int KC = Cfg::KC;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);  // [KC][BMT]
    T *Bs = As + KC * BMT;                     // [KC][BNT]

    const int tid = threadIdx.x;
    const int tm = tid % 16;
    const int tn = tid / 16;
    const int64_t i0 = (int64_t)blockIdx.x * BMT;
    const int64_t tile = blockIdx.y;
    const T *A = static_cast<const T *>(a.A);
    const T *Bt = static_cast<const T *>(a.Bp) + tile * a.kp * BNT;

    RankAcc<T> acc;
    acc.zero();
    const T ealpha = static_cast<T>(a.alpha);
    const T ebeta = static_cast<T>(a.beta);

    for (int64_t kc = 0; kc < a.k; kc += KC) {
        for (int e = tid * V; e < KC * BMT; e += Cfg::CONSUMERS * V) {
            const int pc = e / BMT;
            const int il = e % BMT;
            const int64_t p = kc + pc;
            const int64_t i = i0 + il;
            Vec<T, V> v;
            if (vec_a && p < a.k && i + V <= a.m) {
                v = ld_vec<T, V>(A + i + p * a.lda);
            } else {
#pragma unroll
                for (int r = 0; r < V; ++r)
                    v.v[r] = (p < a.k && i + r < a.m) ? A[i + r + p * a.lda] : T(0);
            }
            st_vec<T, V>(As + e, v);
        }
        for (int e = tid * V; e < KC * BNT; e += Cfg::CONSUMERS * V) {
            const int64_t p = kc + e / BNT;
            Vec<T, V> v;
            if (p < a.kp) {
                v = ld_vec<T, V>(Bt + p * BNT + (e % BNT));
            } else {
#pragma unroll
                for (int r = 0; r < V; ++r) v.v[r] = T(0);
            }
            st_vec<T, V>(Bs + e, v);
        }
        __syncthreads();
        const int kcnt = (a.k - kc < KC) ? (int)(a.k - kc) : KC;
        acc.chunk(As, Bs, kcnt, tm, tn);
        __syncthreads();
    }
    RankEpilogue<T> ep;
    ep.template load<LVC>(a, i0, tile, tm, tn, nullptr, ebeta);
    ep.template store<LVC>(acc, a, i0, tile, tm, tn, ealpha, ebeta);
}

// FP32, k > 32 (FMA-bound).  A 16-byte shared-memory load costs
// four wavefronts whatever its address pattern, and the SM serves one per
// cycle; the 8 x 4 register tiles above need 1.5 per cycle at the FMA peak,
// so this kernel uses 8 x 8 tiles (1.0 per cycle): 4 consumer warps own the
// same 128 x 64 C tile as a 2 x 2 grid of 64 x 32 warp tiles, lane
// (lm = lane % 8, ln = lane / 8) owning rows {wm*64 + lm*4 + r, +32} and
// columns {wn*32 + ln*4 + c, +16} (r, c < 4); a warp's A reads cover one
// 128-byte line, its B reads 64 bytes.  For k > 32, k streams in chunks of 32
// through 3 stages (24 KB each) and the C tile has one 32 KB buffer: two blocks
// (8 consumer warps) per SM, each chunk unrolled whole.  Chunks of 16 (3 stages
// of 12 KB) fit three blocks per SM, but each chunk's wait and release costs a
// fixed stretch of issue: their main loop ran at ~0.72 of the FMA peak against
// ~0.79 for chunks of 32.  For k in 17..32 the chunks of 16 stay (two chunks
// per tile, so the C0 copy overlaps the second).
//
// TMA_EPI (C meets the TMA rules): the producer brings the C0 tile into the
// buffer with one tensor copy while the tile's products run; the epilogue
// overwrites it in place with alpha*acc + beta*C0.  The producer then writes it
// out with a TMA store and, once the store has read the buffer, issues the next
// tile's C0 copy into it -- from the next tile's second chunk on, so the copy has
// that tile's chunks to land (without it, the copy issued one chunk before the
// epilogue was still in flight at half of the k = 64 epilogues).  With beta = 1
// and k > 32 there is no C0 copy: the epilogue writes alpha*acc into the buffer and the
// producer adds it to C with a TMA reduce-add (cp.reduce.async.bulk.tensor
// .add), which reads C0 and writes C in L2 -- the same single rounding of
// C0 + alpha*acc as the fma(1, C0, alpha*acc) of the other form -- so the tile
// never waits for C0.
// Otherwise the epilogue moves C0 and C with 16-byte loads and stores.
namespace {
template <bool TMA_EPI, int KC_>
struct WideCfg {
    static constexpr int BMT = 128;
    static constexpr int BNT = kRankNT;  // 64
    static constexpr int KC = KC_;
    static constexpr int RESIDENT = KC == 16 ? 3 : 2;  // blocks per SM
    static constexpr int STAGES = 3;
    static constexpr int CONSUMERS = 128;
    static constexpr int THREADS = CONSUMERS + 32;
    static constexpr int A_CHUNK = BMT * KC;
    static constexpr int B_CHUNK = KC * BNT;
    static constexpr int STAGE_ELEMS = A_CHUNK + B_CHUNK;
    static constexpr int C_ELEMS = TMA_EPI ? BMT * BNT : 0;  // [BNT][BMT], as the tensor copy lays it out
    static constexpr int DATA_BYTES = (STAGES * STAGE_ELEMS + C_ELEMS) * 4;
    static constexpr int NBAR = 2 * STAGES + 2;
    static constexpr int SMEM = DATA_BYTES + NBAR * 8 + 16;
    static_assert(RESIDENT * (SMEM + 1024) <= 228 * 1024, "resident blocks per SM");
};

struct WideAcc {
    // [row][column pair]: rows r0..r0+3 (0..3) and r0+32..r0+35 (4..7); column
    // pairs (c0, c0+1), (c0+2, c0+3), (c0+16, c0+17), (c0+18, c0+19).  Each A
    // value is duplicated into both halves of a packed operand and B supplies
    // adjacent column pairs as they lie in shared memory.
    float2 v[8][4];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) v[r][q] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void step(const float *As, const float *Bs, int pc, int r0, int c0) {
        const float4 a0 = *reinterpret_cast<const float4 *>(As + pc * 128 + r0);
        const float4 a1 = *reinterpret_cast<const float4 *>(As + pc * 128 + r0 + 32);
        const float4 b0 = *reinterpret_cast<const float4 *>(Bs + pc * kRankNT + c0);
        const float4 b1 = *reinterpret_cast<const float4 *>(Bs + pc * kRankNT + c0 + 16);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float2 bp[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                              make_float2(b1.z, b1.w)};
        float2 ad[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) ad[r] = make_float2(av[r], av[r]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int r = 0; r < 8; ++r) v[r][q] = __ffma2_rn(ad[r], bp[q], v[r][q]);
    }
    // a full chunk is unrolled whole, so its loads can be scheduled early
    template <int KC>
    __device__ __forceinline__ void chunk(const float *As, const float *Bs, int kcnt, int r0, int c0) {
        if (kcnt == KC) {
#pragma unroll(KC == 16 ? 8 : KC)
            for (int pc = 0; pc < KC; ++pc) step(As, Bs, pc, r0, c0);
        } else {
#pragma unroll 4
            for (int pc = 0; pc < kcnt; ++pc) step(As, Bs, pc, r0, c0);
        }
    }
    // the 4 rows of row group rg (0: r0.., 1: r0+32..) in column c (0..7)
    __device__ __forceinline__ float4 rows(int rg, int c) const {
        const int q = c / 2;
        if (c & 1) return make_float4(v[rg * 4][q].y, v[rg * 4 + 1][q].y, v[rg * 4 + 2][q].y, v[rg * 4 + 3][q].y);
        return make_float4(v[rg * 4][q].x, v[rg * 4 + 1][q].x, v[rg * 4 + 2][q].x, v[rg * 4 + 3][q].x);
    }
};

__device__ __forceinline__ float4 axpby4(float alpha, float4 x, float beta, float4 c0, bool use_c0) {
    x.x *= alpha;  // alpha*x == x exactly when alpha is 1
    x.y *= alpha;
    x.z *= alpha;
    x.w *= alpha;
    if (use_c0) {
        x.x = fmaf(beta, c0.x, x.x);
        x.y = fmaf(beta, c0.y, x.y);
        x.z = fmaf(beta, c0.z, x.z);
        x.w = fmaf(beta, c0.w, x.w);
    }
    return x;
}

__device__ __forceinline__ void tma_reduce_add_2d_commit(const void *tmap, const void *smem_src, int32_t x,
                                                         int32_t y) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(tmap)),
                 "r"(x), "r"(y), "r"(smem_addr(smem_src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void tma_store_2d_commit(const void *tmap, const void *smem_src, int32_t x,
                                                    int32_t y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(tmap)),
                 "r"(x), "r"(y), "r"(smem_addr(smem_src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
}  // namespace

template <bool TMA_EPI, int KC, int LVC>
__global__ void __launch_bounds__(WideCfg<TMA_EPI, KC>::THREADS, WideCfg<TMA_EPI, KC>::RESIDENT)
    rankk_wide_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmC,
                      const RankArgs a, unsigned *status) {
    using W = WideCfg<TMA_EPI, KC>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *sStage = reinterpret_cast<float *>(smem_raw);
    float *cbuf = sStage + W::STAGES * W::STAGE_ELEMS;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + W::DATA_BYTES);
    uint64_t *empty = full + W::STAGES;
    uint64_t *cfull = empty + W::STAGES;  // C0 landed (or buffer free, beta == 0)
    uint64_t *cstore = cfull + 1;         // results written (4 consumer warps)

    const int warp = threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    const int64_t mtiles = (a.m + W::BMT - 1) / W::BMT;
    const int64_t ntiles_total = mtiles * ((a.n + W::BNT - 1) / W::BNT);
    const int nchunks = (int)((a.k + W::KC - 1) / W::KC);
    const bool use_c0 = a.beta != 0.0;
    // C = C0 + alpha*acc by a TMA reduce-add of the buffer into C (no C0 copy);
    // FMA-bound shapes only: for k <= 32 the output stream bounds the kernel and the
    // read-modify-write in L2 streamed slower than the C0 copy (0.43 vs 0.35 ms at
    // m = n = 16384, k = 32)
    const bool add_c0 = TMA_EPI && KC == 32 && use_c0 && static_cast<float>(a.beta) == 1.0f;

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmA);
        if (TMA_EPI) prefetch_tmap(&tmC);
        for (int s = 0; s < W::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], W::CONSUMERS / 32);
        }
        mbar_init(cfull, 1);
        mbar_init(cstore, W::CONSUMERS / 32);
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == W::CONSUMERS / 32) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            const uint64_t pol_keep = policy_evict_last();
            const uint64_t pol_stream = policy_evict_first();
            int64_t g = 0;
            int j = 0;
            bool ok = true;
            int32_t prev_x = 0, prev_y = 0;  // C coordinates of the previous tile
            // write tile j's results out (they are complete once every consumer warp
            // arrived on cstore) and wait until the store has read the buffer
            auto store_tile = [&](int jj, int32_t x, int32_t y) -> bool {
                if (!mbar_wait_bounded(cstore, (uint32_t)(jj & 1))) return false;
                if (add_c0)
                    tma_reduce_add_2d_commit(&tmC, cbuf, x, y);
                else
                    tma_store_2d_commit(&tmC, cbuf, x, y);
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                return true;
            };
            for (int64_t t = blockIdx.x; t < ntiles_total && ok; t += gridDim.x, ++j) {
                int64_t tile, mt;
                udivmod(t, mtiles, tile, mt);
                const int64_t i0 = mt * W::BMT;
                const float *Bt = static_cast<const float *>(a.Bp) + tile * a.kp * W::BNT;
                for (int c = 0; c < nchunks; ++c, ++g) {
                    const int st = (int)(g % W::STAGES);
                    if (g >= W::STAGES &&
                        !mbar_wait_bounded(&empty[st], (uint32_t)((g / W::STAGES) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    const int64_t kc = (int64_t)c * W::KC;
                    const int brows = (int)((a.kp - kc < W::KC) ? a.kp - kc : W::KC);
                    float *sA = sStage + st * W::STAGE_ELEMS;
                    mbar_arrive_expect_tx(&full[st], (W::A_CHUNK + brows * W::BNT) * 4);
                    tma_load_2d(sA, &tmA, (int32_t)i0, (int32_t)kc, &full[st], pol_keep);
                    bulk_load(sA + W::A_CHUNK, Bt + kc * W::BNT, brows * W::BNT * 4, &full[st], pol_keep);
                    // after the tile's second chunk (k >= kRankWideMinK: there always is
                    // one): the previous tile's store, then this tile's C0
                    if (TMA_EPI && c == 1) {
                        if (j >= 1 && !store_tile(j - 1, prev_x, prev_y)) {
                            ++g;  // this chunk is in flight: the drain below waits for it
                            ok = false;
                            break;
                        }
                        prev_x = (int32_t)i0;
                        prev_y = (int32_t)(tile * W::BNT);
                        if (use_c0 && !add_c0) {
                            mbar_arrive_expect_tx(cfull, W::C_ELEMS * 4);
                            tma_load_2d(cbuf, &tmC, (int32_t)i0, (int32_t)(tile * W::BNT), cfull, pol_stream);
                        } else {
                            mbar_arrive(cfull);
                        }
                    }
                }
            }
            // the last tile's store
            if (TMA_EPI && ok && j >= 1 && !store_tile(j - 1, prev_x, prev_y)) ok = false;
            if (!ok) atomicOr(status, kDevErrTimeout);
            // copies in flight land before the block may exit
            for (int64_t q = g > W::STAGES ? g - W::STAGES : 0; q < g; ++q)
                mbar_wait_bounded(&full[q % W::STAGES], (uint32_t)((q / W::STAGES) & 1));
            if (TMA_EPI && j >= 1) mbar_wait_bounded(cfull, (uint32_t)((j - 1) & 1));
            if (TMA_EPI) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        }
        return;
    }

    // ---------------------------------------------------- consumers
    const int lm = lane & 7;
    const int ln = lane >> 3;
    const int r0 = (warp & 1) * 64 + lm * 4;   // local rows r0..r0+3 and r0+32..r0+35
    const int c0 = (warp >> 1) * 32 + ln * 4;  // local columns c0..c0+3 and c0+16..c0+19
    const float alpha = static_cast<float>(a.alpha);
    const float beta = static_cast<float>(a.beta);
    const bool alpha1 = alpha == 1.0f;  // alpha*x == x exactly: no multiply
    float *C = static_cast<float *>(a.C);
    int st = 0;       // ring slot of the next chunk
    uint32_t ph = 0;  // and the parity of its phase
    int j = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles_total && ok; t += gridDim.x, ++j) {
        int64_t tile, mt;
        udivmod(t, mtiles, tile, mt);
        const int64_t i0 = mt * W::BMT;
        WideAcc acc;
        acc.zero();
        for (int c = 0; c < nchunks; ++c) {
            if (!mbar_wait_bounded(&full[st], ph)) {
                ok = false;
                break;
            }
            const int kc = c * W::KC;  // k <= kRankMaxK
            const int kcnt = (int)a.k - kc < W::KC ? (int)a.k - kc : W::KC;
            const float *sA = sStage + st * W::STAGE_ELEMS;
            acc.chunk<W::KC>(sA, sA + W::A_CHUNK, kcnt, r0, c0);
            release_reads_to_async_copy();
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
            if (++st == W::STAGES) {
                st = 0;
                ph ^= 1u;
            }
        }
        if (!ok) break;
        if constexpr (TMA_EPI) {
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(cfull, (uint32_t)(j & 1)))) {
                ok = false;
                break;
            }
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                const int cl = c0 + (cc < 4 ? cc : 12 + cc);
#pragma unroll
                for (int rg = 0; rg < 2; ++rg) {
                    float4 *p = reinterpret_cast<float4 *>(cbuf + cl * W::BMT + r0 + rg * 32);
                    const bool with_c0 = use_c0 && !add_c0;
                    const float4 x = acc.rows(rg, cc);
                    if (alpha1 && !with_c0) {
                        *p = x;
                    } else {
                        const float4 c0v = with_c0 ? *p : make_float4(0.f, 0.f, 0.f, 0.f);
                        *p = axpby4(alpha, x, beta, c0v, with_c0);
                    }
                }
            }
            // results in the buffer, visible to the tensor copy: the producer stores them
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(cstore);
        } else {
            // plain epilogue in two halves of 4 columns: all C0 loads of a half before its
            // stores; column cc of a half is cc mod 4 of the tile, so with LVC >= 0 its rows
            // sit (cc * LVC) mod 4 elements past a 16-byte boundary (RankEpilogue's forms)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                Vec<float, 4> c0v[4][2];
                rank_static_for<0, 4>([&](auto cc_tag) {
                    constexpr int cc = decltype(cc_tag)::value;
                    const int64_t jg = tile * W::BNT + c0 + h * 16 + cc;
#pragma unroll
                    for (int rg = 0; rg < 2; ++rg) {
                        const int64_t i = i0 + r0 + rg * 32;
#pragma unroll
                        for (int r = 0; r < 4; ++r) c0v[cc][rg].v[r] = 0.f;
                        if (!use_c0 || jg >= a.n) continue;
                        const float *src = C + i + jg * a.ldc;
                        if (LVC >= 0 && i + 4 <= a.m) {
                            c0v[cc][rg] = ld_group<float, LVC >= 0 ? (cc * LVC) % 4 : 0>(src);
                        } else {
#pragma unroll
                            for (int r = 0; r < 4; ++r)
                                if (i + r < a.m) c0v[cc][rg].v[r] = src[r];
                        }
                    }
                });
                rank_static_for<0, 4>([&](auto cc_tag) {
                    constexpr int cc = decltype(cc_tag)::value;
                    const int64_t jg = tile * W::BNT + c0 + h * 16 + cc;
                    if (jg >= a.n) return;
#pragma unroll
                    for (int rg = 0; rg < 2; ++rg) {
                        const int64_t i = i0 + r0 + rg * 32;
                        const float4 x = acc.rows(rg, h * 4 + cc);
                        const Vec<float, 4> &cv = c0v[cc][rg];
                        const float4 o =
                            axpby4(alpha, x, beta, make_float4(cv.v[0], cv.v[1], cv.v[2], cv.v[3]), use_c0);
                        float *dst = C + i + jg * a.ldc;
                        if (LVC >= 0 && i + 4 <= a.m) {
                            Vec<float, 4> ov;
                            ov.v[0] = o.x, ov.v[1] = o.y, ov.v[2] = o.z, ov.v[3] = o.w;
                            st_group<float, LVC >= 0 ? (cc * LVC) % 4 : 0>(dst, ov);
                        } else {
                            if (i < a.m) dst[0] = o.x;
                            if (i + 1 < a.m) dst[1] = o.y;
                            if (i + 2 < a.m) dst[2] = o.z;
                            if (i + 3 < a.m) dst[3] = o.w;
                        }
                    }
                });
            }
        }
    }
    if (!ok && lane == 0) atomicOr(status, kDevErrTimeout);
}

template <bool TMA_EPI, int KC, int LVC>
static cudaError_t launch_rankk_wide_t(const CUtensorMap *tmA, const CUtensorMap *tmC, const RankArgs &a,
                                       unsigned *status, cudaStream_t s) {
    using W = WideCfg<TMA_EPI, KC>;
    {
        const cudaError_t e =
            ensure_smem_limit(reinterpret_cast<const void *>(rankk_wide_kernel<TMA_EPI, KC, LVC>), W::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t tiles = ((a.m + W::BMT - 1) / W::BMT) * ((a.n + W::BNT - 1) / W::BNT);
    const int64_t slots = W::RESIDENT * (int64_t)(a.num_sms > 0 ? a.num_sms : 1);
    const unsigned grid = (unsigned)(tiles < slots ? tiles : slots);
    rankk_wide_kernel<TMA_EPI, KC, LVC><<<grid, W::THREADS, W::SMEM, s>>>(*tmA, *tmC, a, status);
    return cudaGetLastError();
}

template <typename T, int STAGES, bool PF, bool C0I, int LVC>
static cudaError_t launch_rankk_tma_t(const CUtensorMap *tmA, const CUtensorMap *tmC,
                                      const RankArgs &a, unsigned *status, cudaStream_t s) {
    using Cfg = RankCfg<T>;
    using TC = RankTmaCfg<T, STAGES, PF>;
    {
        const cudaError_t e = ensure_smem_limit(
            reinterpret_cast<const void *>(rankk_tma_kernel<T, STAGES, PF, C0I, LVC>), TC::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t tiles = ((a.m + Cfg::BMT - 1) / Cfg::BMT) * ((a.n + Cfg::BNT - 1) / Cfg::BNT);
    const int64_t slots = (int64_t)TC::RESIDENT * (a.num_sms > 0 ? a.num_sms : 1);
    const unsigned grid = (unsigned)(tiles < slots ? tiles : slots);
    rankk_tma_kernel<T, STAGES, PF, C0I, LVC><<<grid, TC::THREADS, TC::SMEM, s>>>(*tmA, *tmC, a, status);
    return cudaGetLastError();
}

// Calls f(std::integral_constant<int, LVC>) for the form lvc of C's accesses
// (RankEpilogue): FP32 -1..3, FP64 -1..1.
template <typename T, typename F>
static cudaError_t with_c_form(int lvc, F &&f) {
    switch (lvc) {
        case 0:
            return f(std::integral_constant<int, 0>{});
        case 1:
            return f(std::integral_constant<int, 1>{});
        case 2:
            if constexpr (sizeof(T) == 4) return f(std::integral_constant<int, 2>{});
            break;
        case 3:
            if constexpr (sizeof(T) == 4) return f(std::integral_constant<int, 3>{});
            break;
        default:
            break;
    }
    return f(std::integral_constant<int, -1>{});
}

template <typename T>
static cudaError_t launch_rankk_t(const CUtensorMap *tmA, const CUtensorMap *tmC, const RankArgs &a,
                                  unsigned *status, cudaStream_t s) {
    using Cfg = RankCfg<T>;
    const bool vec_a = (reinterpret_cast<uintptr_t>(a.A) % 16 == 0) &&
                       ((a.lda * (int64_t)sizeof(T)) % 16 == 0);
    // form of C's accesses: ldc mod (16 bytes / element) for a 16-byte aligned base, else -1
    const int lvc = reinterpret_cast<uintptr_t>(a.C) % 16 == 0 ? (int)((uint64_t)a.ldc % (16 / sizeof(T))) : -1;
    if (tmA) {
        // FP32 from k = kRankWideMinK on: the 8 x 8-tile kernel (its A tensor map's box is
        // 128 x rank_wide_kc(k)); C by TMA when its tensor map exists, else in form lvc
        if (rank_wide(sizeof(T) == 4 ? TSMM_F32 : TSMM_F64, 2, 0, a.k)) {
            if (rank_wide_kc(a.k) == 16) {
                if (tmC) return launch_rankk_wide_t<true, 16, 0>(tmA, tmC, a, status, s);
                return with_c_form<T>(lvc, [&](auto f) {
                    return launch_rankk_wide_t<false, 16, decltype(f)::value>(tmA, tmA, a, status, s);
                });
            }
            if (tmC) return launch_rankk_wide_t<true, 32, 0>(tmA, tmC, a, status, s);
            return with_c_form<T>(lvc, [&](auto f) {
                return launch_rankk_wide_t<false, 32, decltype(f)::value>(tmA, tmA, a, status, s);
            });
        }
        // output-bound shapes: one k chunk, C0 prefetched by TMA when it is read
        if (a.k <= Cfg::KC) {
            if (tmC && a.beta != 0.0) {
                if constexpr (std::is_same<T, double>::value)
                    if (a.alpha == 1.0 && a.beta == 1.0)
                        return launch_rankk_tma_t<T, 1, true, true, 0>(tmA, tmC, a, status, s);
                return launch_rankk_tma_t<T, 1, true, false, 0>(tmA, tmC, a, status, s);
            }
            return with_c_form<T>(lvc, [&](auto f) {
                return launch_rankk_tma_t<T, 1, false, false, decltype(f)::value>(tmA, tmA, a, status, s);
            });
        }
        return with_c_form<T>(lvc, [&](auto f) {
            return launch_rankk_tma_t<T, 2, false, false, decltype(f)::value>(tmA, tmA, a, status, s);
        });
    }
    const int smem = Cfg::KC * (Cfg::BMT + Cfg::BNT) * (int)sizeof(T);
    dim3 grid((unsigned)((a.m + Cfg::BMT - 1) / Cfg::BMT), (unsigned)((a.n + Cfg::BNT - 1) / Cfg::BNT));
    if (lvc == 0) rankk_plain_kernel<T, 0><<<grid, Cfg::CONSUMERS, smem, s>>>(a, vec_a);
    else rankk_plain_kernel<T, -1><<<grid, Cfg::CONSUMERS, smem, s>>>(a, vec_a);
    return cudaGetLastError();
}

cudaError_t launch_rankk(tsmm_dtype dt, const CUtensorMap *tmA, const CUtensorMap *tmC,
                         const RankArgs &a, unsigned *status, cudaStream_t s) {
    return dt == TSMM_F32 ? launch_rankk_t<float>(tmA, tmC, a, status, s)
                          : launch_rankk_t<double>(tmA, tmC, a, status, s);
}

}  // namespace tsmm
