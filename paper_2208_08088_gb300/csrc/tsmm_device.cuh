// Device-side building blocks for sm_103a: mbarrier, bulk / tensor TMA copies,
// bounded waits, and small vector helpers.  Hand-written inline PTX.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsmm {

// Device error record: kernels OR these bits into the plan's status word.
enum : uint32_t { kDevErrTimeout = 1u };

// A wait on an mbarrier phase gives up after kWaitNs of global time (one
// second) or kMaxPolls polls, whichever comes first.  A poll is an
// mbarrier.try_wait, which suspends the thread for a hardware-defined interval
// while the phase is incomplete (about 3.8 us on GB300, measured), so the poll
// cap alone would be about a minute; the clock makes the bound one second, far
// above any legitimate wait (microseconds) and short enough that a lost
// transaction costs the caller a TSMM_ERR_TIMEOUT, not a hung GPU.
constexpr uint32_t kMaxPolls = 1u << 24;
constexpr uint64_t kWaitNs = 1000000000ull;

// Quotient and remainder of a / b for 0 <= a, 0 < b.  A 64-bit division is a
// long sequence that occupies the (slow) FP64 pipe on this GPU; per-tile index
// math takes the 32-bit path whenever both operands fit.
__device__ __forceinline__ void udivmod(int64_t a, int64_t b, int64_t &q, int64_t &r) {
    if (((static_cast<uint64_t>(a) | static_cast<uint64_t>(b)) >> 32) == 0) {
        const uint32_t q32 = static_cast<uint32_t>(a) / static_cast<uint32_t>(b);
        q = q32;
        r = static_cast<int64_t>(static_cast<uint32_t>(a) - q32 * static_cast<uint32_t>(b));
    } else {
        q = a / b;
        r = a - q * b;
    }
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make mbarrier initialisation visible to the async proxy (TMA).
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// Element copy global -> shared; a zero source size writes zeros and reads nothing.
__device__ __forceinline__ void cp_async_elem(void *smem_dst, const void *gsrc, bool valid, int bytes) {
    const uint32_t n = valid ? (uint32_t)bytes : 0u;
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(smem_dst)), "l"(gsrc), "r"(n)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(smem_dst)), "l"(gsrc), "r"(n)
                     : "memory");
}
// The barrier counts this thread's arrival once all its earlier cp.async copies have landed.
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// A consumer's release of a shared-memory buffer that a tensor or bulk copy
// (the async proxy) refills: its reads of the buffer (generic proxy) are
// ordered before that copy by this fence, issued by every reading thread before
// the warp's arrival on the buffer's "empty" barrier.  Without it a read still
// in flight when the barrier completes can return the refilled data.
__device__ __forceinline__ void release_reads_to_async_copy() { fence_proxy_async_smem(); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity to complete: at most max_polls
// polls and kWaitNs of global time.  Returns false (and leaves the barrier
// alone) on timeout.  The first poll is the fast path (no clock read).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint32_t max_polls = kMaxPolls) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; i < max_polls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

// L2 cache policies for the streamed operand (read once) and reused data.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 2-D tiled tensor copy global -> shared, completion counted on `bar`.
// x is the innermost (contiguous) coordinate; the caller guarantees
// x * sizeof(element) is a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const void *tmap, int32_t x, int32_t y,
                                            uint64_t *bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_addr(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Contiguous bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completion counted on `bar`.
__device__ __forceinline__ void bulk_load(void *smem_dst, const void *gsrc, uint32_t bytes,
                                          uint64_t *bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(gsrc)), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// One column of A whose first element sits d elements past a 16-byte boundary,
// as one bulk copy of the 16-byte-aligned span around its rows [0, rows): from
// (first element - d) to the next 16-byte boundary after the last row, so row r
// lands at slot[d + r] of a 16-byte-aligned slot.  The span's extra bytes (under
// 16 on either side) lie in the same 16-byte chunks as the column's own
// elements, hence on the same pages (they cannot fault), and land in slot
// positions that hold no row.  Returns the copy's size.
template <typename T>
__device__ __forceinline__ uint32_t column_span_bytes(int rows, int d) {
    constexpr int V = 16 / (int)sizeof(T);
    return (uint32_t)((d + rows + V - 1) / V * 16);
}

__device__ __forceinline__ void prefetch_tmap(const void *tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

// Named barrier over a subset of the block's warps (id 0 is __syncthreads).
__device__ __forceinline__ void named_barrier(uint32_t id, uint32_t threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Vector of N consecutive elements for 16-byte (or smaller) shared/global access.
template <typename T, int N>
struct alignas(sizeof(T) * N) Vec {
    T v[N];
};

template <typename T, int N>
__device__ __forceinline__ Vec<T, N> ld_vec(const T *p) {
    return *reinterpret_cast<const Vec<T, N> *>(p);
}

template <typename T, int N>
__device__ __forceinline__ void st_vec(T *p, const Vec<T, N> &v) {
    *reinterpret_cast<Vec<T, N> *>(p) = v;
}

// L2-coherent load that bypasses L1 (split-K partials written by other CTAs).
template <typename T>
__device__ __forceinline__ T ld_cg(const T *p) {
    return __ldcg(p);
}

}  // namespace tsmm
