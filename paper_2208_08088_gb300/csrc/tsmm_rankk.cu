// Regime (ii) kernel: C[m x n] = alpha * A[m x k] * B[k x n] + beta * C0 with
// k <= 128 and m, n large (a rank-k update; TSMM with the skinny operand on
// the inner dimension, Section I).  The whole k extent of a C tile is
// contracted on chip, so the kernel streams C0 in and C out exactly once:
// the traffic floor of this shape is the 2*m*n output read/write, not A or B.
//
// Thread block: 256 threads own a BMT x 128 tile of C.  Each thread keeps a
// (2*VEC) x 8 register tile split in two row groups {tm*VEC + r} and
// {BMT/2 + tm*VEC + r} and two column groups {tn*4 + c} and {64 + tn*4 + c}, so
// that both the shared-memory operand reads and the global C0 loads / C stores
// of a half-warp cover one contiguous 256-byte run.  k is consumed in chunks of
// KC = 32 staged through shared memory.
#include "tsmm_device.cuh"
#include "tsmm_internal.h"

namespace tsmm {

template <typename T>
struct RankCfg {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int TM = 2 * VEC;         // rows per thread (two row groups)
    static constexpr int TN = 8;               // columns per thread (two column groups)
    static constexpr int BMT = 16 * TM;        // 128 (f32) / 64 (f64)
    static constexpr int BNT = kRankNT;        // 128
    static constexpr int KC = 32;
    static constexpr int THREADS = 256;
    static constexpr int SMEM = KC * (BMT + BNT) * (int)sizeof(T);
    static_assert(BNT == 16 * TN, "tile width");
};

template <typename T>
__global__ void __launch_bounds__(256, 2) rankk_kernel(const RankArgs a, bool vec_a, bool vec_c) {
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

    T acc[Cfg::TM][Cfg::TN];
#pragma unroll
    for (int r = 0; r < Cfg::TM; ++r)
#pragma unroll
        for (int c = 0; c < Cfg::TN; ++c) acc[r][c] = T(0);

    for (int64_t kc = 0; kc < a.k; kc += KC) {
        // ---- stage A[i0 .. i0+BMT) x [kc .. kc+KC) as As[p][i]
        for (int e = tid * V; e < KC * BMT; e += Cfg::THREADS * V) {
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
        // ---- stage packed B rows [kc .. kc+KC) of this column tile as Bs[p][j]
        for (int e = tid * V; e < KC * BNT; e += Cfg::THREADS * V) {
            const int pc = e / BNT;
            const int64_t p = kc + pc;
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
#pragma unroll 4
        for (int pc = 0; pc < kcnt; ++pc) {
            const Vec<T, V> a0 = ld_vec<T, V>(As + pc * BMT + tm * V);
            const Vec<T, V> a1 = ld_vec<T, V>(As + pc * BMT + BMT / 2 + tm * V);
            const Vec<T, 4> b0 = *reinterpret_cast<const Vec<T, 4> *>(Bs + pc * BNT + tn * 4);
            const Vec<T, 4> b1 = *reinterpret_cast<const Vec<T, 4> *>(Bs + pc * BNT + 64 + tn * 4);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
#pragma unroll
                for (int r = 0; r < V; ++r) {
                    acc[r][c] = fma(a0.v[r], b0.v[c], acc[r][c]);
                    acc[V + r][c] = fma(a1.v[r], b0.v[c], acc[V + r][c]);
                    acc[r][4 + c] = fma(a0.v[r], b1.v[c], acc[r][4 + c]);
                    acc[V + r][4 + c] = fma(a1.v[r], b1.v[c], acc[V + r][4 + c]);
                }
            }
        }
        __syncthreads();
    }

    // ---- epilogue: C = alpha*acc + beta*C0, one pass over the tile
    const T alpha = static_cast<T>(a.alpha);
    const T beta = static_cast<T>(a.beta);
    T *C = static_cast<T *>(a.C);
#pragma unroll
    for (int cg = 0; cg < 2; ++cg) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = tile * BNT + cg * 64 + tn * 4 + c;
            if (j >= a.n) continue;
#pragma unroll
            for (int rg = 0; rg < 2; ++rg) {
                const int64_t i = i0 + rg * (BMT / 2) + tm * V;
                T *cp = C + i + j * a.ldc;
                if (vec_c && i + V <= a.m) {
                    Vec<T, V> o;
#pragma unroll
                    for (int r = 0; r < V; ++r) o.v[r] = alpha * acc[rg * V + r][cg * 4 + c];
                    if (beta != T(0)) {
                        const Vec<T, V> c0 = ld_vec<T, V>(cp);
#pragma unroll
                        for (int r = 0; r < V; ++r) o.v[r] = fma(beta, c0.v[r], o.v[r]);
                    }
                    st_vec<T, V>(cp, o);
                } else {
#pragma unroll
                    for (int r = 0; r < V; ++r) {
                        if (i + r < a.m) {
                            T o = alpha * acc[rg * V + r][cg * 4 + c];
                            if (beta != T(0)) o = fma(beta, cp[r], o);
                            cp[r] = o;
                        }
                    }
                }
            }
        }
    }
}

template <typename T>
static cudaError_t launch_rankk_t(const RankArgs &a, cudaStream_t s) {
    using Cfg = RankCfg<T>;
    const bool vec_a = (reinterpret_cast<uintptr_t>(a.A) % 16 == 0) &&
                       ((a.lda * (int64_t)sizeof(T)) % 16 == 0);
    const bool vec_c = (reinterpret_cast<uintptr_t>(a.C) % 16 == 0) &&
                       ((a.ldc * (int64_t)sizeof(T)) % 16 == 0);
    dim3 grid((unsigned)((a.m + Cfg::BMT - 1) / Cfg::BMT), (unsigned)((a.n + Cfg::BNT - 1) / Cfg::BNT));
    rankk_kernel<T><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a, vec_a, vec_c);
    return cudaGetLastError();
}

cudaError_t launch_rankk(tsmm_dtype dt, const RankArgs &a, cudaStream_t s) {
    return dt == TSMM_F32 ? launch_rankk_t<float>(a, s) : launch_rankk_t<double>(a, s);
}

}  // namespace tsmm
