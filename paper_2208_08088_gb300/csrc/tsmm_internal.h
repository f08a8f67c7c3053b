// Internal (host-side) declarations shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

#include "../../include/tsmm.h"

namespace tsmm {

// ---- tiling constants shared by planner, packer and kernels -------------------
// Regime (i): A columns per pipeline stage; packed B rows are padded to it.
constexpr int kTallBKS = 32;
// Regime (i): consumer warps per thread block (the producer warp is extra).
constexpr int kTallConsumerWarps = 4;
// Regime (ii): packed B tile width (columns) and k granule.
constexpr int kRankNT = 64;
constexpr int kRankKGran = 8;
constexpr int kRankMaxK = 128;
constexpr int kTallMaxN = 64;

inline size_t dtype_size(tsmm_dtype d) { return d == TSMM_F64 ? 8 : 4; }

// Smallest power of two >= n.
inline int pow2_ceil(int64_t n) {
    int np = 1;
    while (np < n) np <<= 1;
    return np;
}

// Padded column count of the regime-(i) kernel that serves n columns: one of
// 1, 2, 4, 8, 16, 24, 32, 48, 64 (the FMA-bound widths 24 and 48 save a
// quarter of the padded work for n in 17..24 and 33..48).
inline int tall_np(int64_t n) {
    if (n > 16 && n <= 24) return 24;
    if (n > 32 && n <= 48) return 48;
    return pow2_ceil(n);
}

// Rows per thread block (m-slab) of the regime-(i) kernel.  FP32 widths up to
// 32 take 256 rows: the consumer warps then split the slab by rows more and the
// stage's k columns less (widths 24 and 32: each warp reads whole 32-column
// stages instead of two warps splitting every stage, one stage wait per 16
// k-steps -- n = 24: 0.83 -> 0.79 ms, n = 32: 1.01 -> 0.98 ms at m = k = 32768;
// widths up to 16: 4 -> 2 warps per stage, 0.5-1.5 % faster; width 48 with
// its 8 x 12 tiles likewise).  The FP32 width 64 takes 128 (its warps already
// own whole stages), FP64 64.
constexpr int tall_block_rows(bool f64, int np) { return f64 ? 64 : (np == 64 ? 128 : 256); }
inline int tall_bm(tsmm_dtype d, int np) { return tall_block_rows(d == TSMM_F64, np); }

// Thread blocks of the regime-(i) TMA kernel resident per SM (its shared-memory
// ring is sized for this): 3 for the FMA-bound FP32 widths 32 and 64 (8 x 8
// tiles fit 136 registers), else 2 (the width 48's 8 x 12 tiles need ~160).
constexpr int tall_resident_blocks(bool f64, int np) { return (!f64 && (np == 32 || np == 64)) ? 3 : 2; }

// Load form of the regime (i) kernel for an A that a tensor map cannot describe
// (its bulk/element-copy kernel): for FP32 widths of 16 and more with A's base
// 16-byte aligned, lda mod 4 -- every column's offset within 16 bytes is then
// fixed by its index mod 4, and the kernel is compiled for it -- else -1
// (offsets computed at run time).
inline int async_load_variant(bool f32, int np, const void *A, int64_t lda) {
    if (!f32 || np < 16 || reinterpret_cast<uintptr_t>(A) % 16 != 0) return -1;
    return (int)((uint64_t)lda & 3u);
}

// Regime of a (k, n) pair: 1 = tall (n <= 64), 2 = rank-k (k <= 128), 0 = unsupported.
inline int regime_of(int64_t k, int64_t n) {
    if (n <= kTallMaxN) return 1;
    if (k <= kRankMaxK) return 2;
    return 0;
}

inline int64_t round_up(int64_t x, int64_t g) { return (x + g - 1) / g * g; }

// Raises a kernel's dynamic shared-memory limit to `bytes` once per (kernel,
// device); thread-safe (the server thread and callers' threads launch alike).
inline cudaError_t ensure_smem_limit(const void *kernel, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kernel, dev})) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert({kernel, dev});
    return e;
}

}  // namespace tsmm

struct tsmm_packed_b_s {
    tsmm_dtype dtype;
    int precision;   // tsmm_precision
    int64_t k, n;
    int64_t kp;      // padded rows
    int64_t w;       // tile width (columns)
    int64_t ntiles;  // number of column tiles
    int regime;
    int device;
    void *data;      // device storage, kp * w * ntiles elements
    size_t bytes;
};

struct tsmm_plan_s {
    int64_t m, n, k;
    tsmm_dtype dtype;
    int precision;   // tsmm_precision
    int regime;
    int device;
    int num_sms;
    // regime (i)
    int np;          // padded n
    int bm;          // rows per thread block
    int64_t slabs;   // ceil(m / bm)
    int splits;      // k splits (S)
    int64_t kchunk;  // packed-B rows per split (multiple of kTallBKS)
    int64_t kp;      // padded k
    // regime (ii)
    int64_t mtiles, ntiles;
    // device scratch owned by the plan
    void *workspace;           // splits * np * slabs * bm elements (regime (i), splits > 1)
    size_t workspace_bytes;
    unsigned *tickets;         // one arrival counter per slab
    unsigned *status;          // device error word
    // one-entry caches of the TMA descriptors for A and (regime (ii)) C
    const void *tmap_ptr;
    int64_t tmap_lda;
    CUtensorMap tmap;
    const void *tmapc_ptr;
    int64_t tmapc_ldc;
    CUtensorMap tmapc;
};

namespace tsmm {

struct TallArgs {
    int64_t m, n, k, lda, ldc;
    const void *A;
    const void *Bp;     // packed B, kp x np row-major
    void *C;
    double alpha, beta;
    void *ws;
    unsigned *tickets;
    unsigned *status;
    int splits;
    int64_t kchunk, kp, slabs;
};

// Launchers (return cudaSuccess or the launch error).  `tma` selects the
// TMA-pipelined kernel (tmap must describe A) or the plain-load kernel.
cudaError_t launch_tall_f32(bool tma, int np, const CUtensorMap *tmap, const TallArgs &a,
                            cudaStream_t s);
cudaError_t launch_tall_f64(bool tma, int np, const CUtensorMap *tmap, const TallArgs &a,
                            cudaStream_t s);

struct RankArgs {
    int64_t m, n, k, lda, ldc, kp;
    const void *A;
    const void *Bp;  // packed B, ntiles x (kp x kRankNT)
    void *C;
    double alpha, beta;
    int num_sms;     // persistent grid size = resident blocks x SMs
};
// tmA: tensor map of A (box bm x 32) or nullptr for the plain-load kernel;
// The FP32 regime (ii) kernel for k >= kRankWideMinK streams k in chunks of
// rank_wide_kc(k): 16 up to k = 32 (three blocks per SM), 32 above (two blocks
// per SM), so that every tile has at least two chunks.  Its A tensor map box is
// bm x rank_wide_kc(k); every other kernel's is bm x kTallBKS.
constexpr int kRankWideMinK = 17;
constexpr int rank_wide_kc(int64_t k) { return k <= 32 ? 16 : 32; }
inline bool rank_wide(tsmm_dtype d, int regime, int precision, int64_t k) {
    return d == TSMM_F32 && regime == 2 && precision == 0 && k >= kRankWideMinK;
}
inline int a_box_k(tsmm_dtype d, int regime, int precision, int64_t k) {
    return rank_wide(d, regime, precision, k) ? rank_wide_kc(k) : kTallBKS;
}
// tmC: tensor map of C (box bm x kRankNT) when C meets the TMA rules, else nullptr.
cudaError_t launch_rankk(tsmm_dtype dt, const CUtensorMap *tmA, const CUtensorMap *tmC,
                         const RankArgs &a, unsigned *status, cudaStream_t s);

// Plan construction with an optional forced split count (0 = planner's choice).
tsmm_status create_plan(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype, int forced_splits,
                        tsmm_plan_t *out, int precision = 0);

// Plan fields without any device allocation: every member except workspace,
// tickets and status, plus the ticket bytes the plan needs; split-K workspaces
// are capped at max_workspace bytes.  (Used by create_plan and the server.)
tsmm_status plan_layout(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype, int forced_splits,
                        int precision, int dev, int sms, int64_t max_workspace, tsmm_plan_s *p,
                        size_t *ticket_bytes_out);

// BF16x3 precision mode (tsmm_bf16x3.cu): k granule of its packed B and plan.
constexpr int kX3KB = 64;
inline int x3_np(int64_t n) {
    const int np = pow2_ceil(n);  // an MMA N of 16, 32 or 64
    return np < 16 ? 16 : np;
}
cudaError_t launch_tall_bf16x3(int np, const CUtensorMap *tmap, const TallArgs &a, int num_sms,
                               cudaStream_t s);
cudaError_t launch_pack_b_bf16x3(int64_t k, int64_t n, const void *B, int64_t ldb, void *dst, int np,
                                 int64_t nchunks, int64_t ntiles, cudaStream_t s);
// Regime (ii) in the BF16x3 mode: tile width of its packed B, and the kernel.
// tmC: tensor map of C (box 128 x kX3RankSub) when C meets the TMA rules
// (C0 loads and C stores by TMA), else nullptr (C0 by 4-byte cp.async, C by
// plain stores).
constexpr int kX3RankNT = 128;
constexpr int kX3RankSub = 32;
cudaError_t launch_rankk_bf16x3(const CUtensorMap *tmA, const CUtensorMap *tmC, const RankArgs &a,
                                unsigned *status, cudaStream_t s);

// Process-wide plan cache (tsmm_tune.cu): tuned split counts keyed by
// (dtype, m, n, k, SM count).  Lookup returns 0 when absent.
int plan_cache_lookup(tsmm_dtype dtype, int64_t m, int64_t n, int64_t k, int sms);
void plan_cache_store(tsmm_dtype dtype, int64_t m, int64_t n, int64_t k, int sms, int splits);

// tsmm_execute_grouped (tsmm_group_api.cu), for the server.
tsmm_status execute_grouped(const tsmm_group_item *items, int count, tsmm_stream_t stream);

// Split-K factor of the regime (i) kernel (planner model in tsmm_api.cu);
// `resident` = thread blocks per SM.
int choose_splits(int64_t slabs, int64_t kstages, int num_sms, int64_t max_splits,
                  int resident = 2);

cudaError_t launch_pack_b(tsmm_dtype dt, int64_t k, int64_t n, const void *B, int64_t ldb,
                          void *dst, int64_t kp, int64_t w, int64_t ntiles, cudaStream_t s);
cudaError_t launch_scale(tsmm_dtype dt, int64_t m, int64_t n, double beta, void *C, int64_t ldc,
                         cudaStream_t s);
cudaError_t launch_copy_columns(tsmm_dtype dt, const void *src, int64_t lds, int64_t m, int64_t k, void *dst,
                                int64_t ldd, cudaStream_t s);

}  // namespace tsmm
