/*
 * tsmm.h -- C ABI of the GB300 (sm_103a) pre-packed tall-and-skinny GEMM.
 *
 * The operation is Eq. 1 of "AutoTSMM: An Auto-tuning Framework for Building
 * High-Performance Tall-and-Skinny Matrix-Matrix Multiplication on CPUs"
 * (Li et al., arXiv 2208.08088):
 *
 *       C = alpha * A * B + beta * C0            A: m x k,  B: k x n,  C: m x n
 *
 * split, as the paper's Algorithm 1 ("Workflow of the pre-pack TSMM") splits
 * it, into a packing step that runs once per B (PACKB, called there with
 * alpha = 1) and a compute step that is executed many times against the
 * packed operand (COMPUTE); the plan object is the GPU counterpart of the
 * paper's runtime "execution plan" (Section III) that is generated once per
 * problem shape and reused.
 *
 * Two shape regimes are supported (TSMM as defined in Section I: one operand
 * has a dimension far smaller than the others):
 *   regime (i)  n <= 64           (A tall: m and k large)   -- streaming kernel
 *   regime (ii) n > 64, k <= 128  (rank-k update: m, n large) -- output-bound kernel
 * Any other shape returns TSMM_ERR_UNSUPPORTED_SHAPE.
 *
 * Conventions shared by every entry point
 *   - All matrices are column-major with explicit leading dimensions
 *     (lda >= max(1,m), ldb >= max(1,k), ldc >= max(1,m)).
 *   - Pointers named *_dev are device pointers on the current CUDA device.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Every entry point that takes a stream only enqueues work on it and
 *     returns without waiting; the returned status covers argument checks and
 *     launch errors, not the outcome of the asynchronous work.
 *   - alpha and beta are passed as double; for TSMM_F32 they are rounded to
 *     float first.  alpha is applied once, in the epilogue (Eq. 1), never folded
 *     into the packed B, so one packed B serves every alpha.
 *   - BLAS conventions for the special cases: beta == 0 means C0 is not read
 *     (C may hold NaN); alpha == 0 or k == 0 means A and B are not read and
 *     C = beta*C0; m == 0 or n == 0 is a no-op returning TSMM_OK.
 *   - Results are deterministic: split-K partial sums are combined in a fixed
 *     order, so the same inputs give the same bits on every call.
 *   - Out-parameters are written only when the call returns TSMM_OK.  No call
 *     aborts or throws; every failure is a status code.
 *   - Accuracy: every entry satisfies |C - C_exact| <= 4*k*u*(|alpha| sum_p
 *     |A[i,p]||B[p,j]| + |beta||C0[i,j]|) with u = 2^-24 (F32) / 2^-53 (F64);
 *     products are accumulated with IEEE fma in the working precision (no
 *     TF32, no reduced-precision tensor-core path).
 */
#ifndef TSMM_H
#define TSMM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TSMM_API __attribute__((visibility("default")))
#else
#define TSMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { TSMM_F32 = 0, TSMM_F64 = 1 } tsmm_dtype;

typedef enum {
    TSMM_OK = 0,
    TSMM_ERR_INVALID_ARG = 1,      /* bad size, leading dimension, NULL pointer or dtype */
    TSMM_ERR_UNSUPPORTED_SHAPE = 2,/* neither n <= 64 nor k <= 128 */
    TSMM_ERR_MISMATCH = 3,         /* plan and packed B disagree on (k, n, dtype) or device */
    TSMM_ERR_MISALIGNED = 4,       /* pointer not aligned to the element size */
    TSMM_ERR_OUT_OF_MEMORY = 5,    /* device allocation failed */
    TSMM_ERR_CUDA = 6,             /* a CUDA runtime/driver call failed */
    TSMM_ERR_TIMEOUT = 7           /* a bounded device-side wait gave up (see tsmm_plan_check) */
} tsmm_status;

/*
 * Arithmetic of a plan / packed B.  NATIVE: IEEE fma in the working precision
 * (the contract stated above).  BF16X3 (TSMM_F32, both regimes): the
 * tensor-core mode C = alpha*(A_hi*B_hi + A_hi*B_lo + A_lo*B_hi) + beta*C0
 * with x_hi = bf16(x), x_lo = bf16(x - x_hi) and FP32 accumulation in tensor
 * memory (tcgen05.mma).  It drops A_lo*B_lo and the split residues, about
 * 3*2^-16 of |A||B| per product, so it does NOT meet the native bound for
 * small k; its documented bound is |C - C_exact| <= (2^-13 + 4*k*2^-24) *
 * (|alpha| sum_p |A[i,p]||B[p,j]| + |beta||C0[i,j]|).  Inf/NaN inputs may turn
 * into NaN (the split of an infinity is Inf - Inf).  Both regimes take any A
 * aligned to 4 bytes: an A that a tensor map cannot describe (base or lda*4
 * not a multiple of 16) is moved column by column, with the same result.
 */
typedef enum { TSMM_PREC_NATIVE = 0, TSMM_PREC_BF16X3 = 1 } tsmm_precision;

typedef void *tsmm_stream_t; /* a cudaStream_t */
typedef struct tsmm_packed_b_s *tsmm_packed_b;
typedef struct tsmm_plan_s *tsmm_plan_t;

/* Human-readable name of a status code (static string, never NULL). */
TSMM_API const char *tsmm_status_string(tsmm_status status);

/* Library version as major*10000 + minor*100 + patch. */
TSMM_API int tsmm_version(void);

/* The CUDA runtime's message for the last CUDA failure that one of this
   thread's calls turned into TSMM_ERR_CUDA / TSMM_ERR_OUT_OF_MEMORY (static
   string, never NULL; "no error" before any). */
TSMM_API const char *tsmm_last_cuda_error(void);

/*
 * tsmm_pack_b -- PACKB of Algorithm 1: copy B (k x n, column-major, leading
 * dimension ldb, device memory) into a library-owned, device-resident panel
 * layout that the compute kernels read with contiguous accesses (the pre-pack
 * module of Section IV.A.3).  The copy is bit-preserving and unscaled.
 *
 * Allocates the packed storage on the current device, enqueues one pack kernel
 * on `stream` and returns the handle in *out.  The caller keeps ownership of
 * B_dev and may free it once `stream` has passed the pack.  The handle owns its
 * storage until tsmm_packed_b_destroy.  k == 0 or n == 0 is allowed (an empty
 * handle).  Errors: INVALID_ARG (negative sizes, ldb < max(1,k), NULL out, or
 * NULL B_dev with k*n > 0), UNSUPPORTED_SHAPE, MISALIGNED (B_dev not aligned to
 * the element size), OUT_OF_MEMORY, CUDA.
 *
 * Packed layout (private to the library, described for test readers): the
 * n columns are cut into `ntiles` tiles of `w` columns (regime (i): one tile,
 * w = the kernel's padded column count, n rounded up to one of 1, 2, 4, 8, 16,
 * 24, 32, 48, 64; regime (ii): w = 64).  Tile t is a
 * row-major kp x w block (kp = k rounded up to the kernel's k granule) at
 * element offset t*kp*w; element (p, jj) of tile t holds B[p, t*w + jj], and is
 * +0.0 where p >= k or t*w + jj >= n.
 */
TSMM_API tsmm_status tsmm_pack_b(tsmm_dtype dtype, int64_t k, int64_t n, const void *B_dev, int64_t ldb,
                        tsmm_stream_t stream, tsmm_packed_b *out);

/*
 * tsmm_pack_b_ex -- tsmm_pack_b with an explicit precision mode.  BF16X3 packs
 * B once as hi and lo BF16 copies in the tensor-core operand layout: the
 * columns are cut into `ntiles` tiles of w columns (regime (i): one tile, w = n
 * rounded up to a power of two, at least 16; regime (ii): w = 128); per tile and
 * per 64-row chunk c of k (kp = k rounded up to 64), a hi tile then a lo tile,
 * each w x 64 BF16 values, element (column j, row kk) at byte (j/8)*1024 +
 * (kk/8)*128 + (j%8)*16 + (kk%8)*2 of the tile; chunk c of tile t starts at byte
 * (t*kp/64 + c) * 4*w*64.  INVALID_ARG for BF16X3 with TSMM_F64.
 */
TSMM_API tsmm_status tsmm_pack_b_ex(tsmm_dtype dtype, tsmm_precision precision, int64_t k, int64_t n,
                                    const void *B_dev, int64_t ldb, tsmm_stream_t stream,
                                    tsmm_packed_b *out);

/* Release a packed B (waits for the device to be done with it).  NULL is a no-op. */
TSMM_API tsmm_status tsmm_packed_b_destroy(tsmm_packed_b pb);

/*
 * Describe a packed B: its dtype, k, n, kp, w, ntiles (see tsmm_pack_b), the
 * device pointer of its storage and the storage size in bytes.  Any output
 * pointer may be NULL.  The storage stays owned by the handle.
 */
TSMM_API tsmm_status tsmm_packed_b_info(tsmm_packed_b pb, tsmm_dtype *dtype, int64_t *k, int64_t *n,
                               int64_t *kp, int64_t *w, int64_t *ntiles, const void **data_dev,
                               size_t *bytes);

/*
 * Copy the packed storage of `pb` (tsmm_packed_b_info's `bytes` bytes) into host
 * memory at host_dst, synchronously (waits for the pack to finish).  For tests
 * and inspection.  Errors: INVALID_ARG (NULL pb, NULL host_dst with a non-empty
 * pack, or `bytes` smaller than the packed size), CUDA.
 */
TSMM_API tsmm_status tsmm_packed_b_read(tsmm_packed_b pb, void *host_dst, size_t bytes);

/*
 * tsmm_plan -- the runtime "execution plan" of Section III / IV.A: chooses the
 * kernel (regime (i) or (ii)), its tile shape, and the split of the k
 * dimension across thread blocks (the GPU analogue of the cache-blocked
 * designer and multi-thread optimizer: blocks are split along m and k, never
 * along n, Section IV.A.2), and allocates the split-K workspace and the
 * per-tile arrival counters on the current device.
 *
 * The plan's shape and kernel choice are fixed once created; it owns its
 * workspace and caches the tensor maps of the last A and C it ran with (each
 * launch takes its own copy), so calls with one plan must come from one host
 * thread at a time, and two executions that may overlap on the device
 * (different streams) need two plans.  Errors: INVALID_ARG (negative sizes,
 * bad dtype, NULL out), UNSUPPORTED_SHAPE, OUT_OF_MEMORY, CUDA.
 */
TSMM_API tsmm_status tsmm_plan(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype, tsmm_plan_t *out);

/*
 * tsmm_plan_ex -- tsmm_plan with an explicit precision mode; the plan and the
 * packed B given to tsmm_execute must have the same mode (else MISMATCH).
 */
TSMM_API tsmm_status tsmm_plan_ex(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype,
                                  tsmm_precision precision, tsmm_plan_t *out);

/* Release a plan (waits for the device to be done with it).  NULL is a no-op. */
TSMM_API tsmm_status tsmm_plan_destroy(tsmm_plan_t plan);

/*
 * Describe a plan: regime (1 or 2), padded column count np, rows per thread
 * block bm, number of k splits, and the workspace size in bytes.  Any output
 * pointer may be NULL.
 */
TSMM_API tsmm_status tsmm_plan_info(tsmm_plan_t plan, int *regime, int *np, int *bm, int *splits,
                           size_t *workspace_bytes);

/*
 * tsmm_execute -- COMPUTE of Algorithm 1:  C = alpha * A * packedB + beta * C0,
 * where C0 is the prior content of C (in place, as in Eq. 1).
 *
 * A_dev: m x k, column-major, leading dimension lda, device memory, read only.
 * C_dev: m x n, column-major, leading dimension ldc, read (if beta != 0) and
 * written.  A and C must not overlap.  `pb` must have been packed with the
 * plan's (k, n, dtype) on the same device (else TSMM_ERR_MISMATCH).
 *
 * A 16-byte aligned A with lda*sizeof(element) a multiple of 16 is staged by
 * tensor copies.  Any other A (pointers must still be aligned to the element
 * size, else MISALIGNED) is staged column by column by bulk copies in regime
 * (i), and in regime (ii) copied first into an aligned scratch buffer taken
 * from the device's stream-ordered memory pool (cudaMallocAsync on `stream`,
 * released by cudaFreeAsync after the kernel; if that allocation fails, a
 * slower kernel with plain loads reads A directly).  Enqueues one kernel on
 * `stream` (two when regime (ii) copies A first) and returns.
 */
TSMM_API tsmm_status tsmm_execute(tsmm_plan_t plan, double alpha, const void *A_dev, int64_t lda,
                         tsmm_packed_b pb, double beta, void *C_dev, int64_t ldc,
                         tsmm_stream_t stream);

/*
 * Synchronize the device and report whether any kernel launched with this plan
 * has recorded a device-side error since the previous check (a bounded wait
 * that ran out of iterations reports TSMM_ERR_TIMEOUT); clears the record.
 */
TSMM_API tsmm_status tsmm_plan_check(tsmm_plan_t plan);

/* Number of kernel launches `tsmm_execute` with this plan enqueues for an A that
 * a tensor map can describe (for accounting; regime (ii) with any other A adds
 * the copy kernel). */
TSMM_API int tsmm_plan_launches_per_execute(tsmm_plan_t plan);

/*
 * One problem of a grouped execution: the arguments of one tsmm_execute call.
 */
typedef struct tsmm_group_item {
    tsmm_plan_t plan;
    double alpha;
    const void *A_dev;
    int64_t lda;
    tsmm_packed_b pb;
    double beta;
    void *C_dev;
    int64_t ldc;
} tsmm_group_item;

/*
 * tsmm_execute_grouped -- run `count` independent TSMMs (uneven shapes, each
 * with its own plan, packed B, alpha, beta, A and C) with as few kernel
 * launches as possible: the grouped execution of many pre-packed products that
 * the paper's reuse argument (Section III) motivates.  Regime (i) problems in
 * the native precision are batched per (dtype, padded column count, whether
 * a tensor map can describe A: base 16-byte aligned and lda*sizeof(element) a
 * multiple of 16) into launches of one grouped kernel, at most 48 problems per
 * launch, with one thread block per work item (m-slab x k-split) of every
 * problem, so that items of unequal cost share the GPU as its block scheduler
 * hands out SMs; any other problem runs as its own tsmm_execute launch on the
 * same stream.  Results equal tsmm_execute's bit for bit.  Every item is validated
 * as tsmm_execute would before anything is launched; two items may not share a
 * plan (INVALID_ARG), since a plan's split-K workspace serves one problem at a
 * time.  Asynchronous on `stream`.
 */
TSMM_API tsmm_status tsmm_execute_grouped(const tsmm_group_item *items, int count,
                                          tsmm_stream_t stream);

/*
 * tsmm_autotune -- the performance evaluator of Section III: time candidate
 * execution plans for this shape on the caller's operands and keep the
 * fastest.  For regime (i) the candidates are split-K factors (the planner's
 * model evaluated for 1..4 resident blocks per SM, its halves and doubles, no
 * split, and factors that fill whole waves of the GPU); each candidate runs
 * once untimed and `reps` times between CUDA events on `stream` with alpha = 1,
 * beta = 0, so C is overwritten.  Blocks until the timing is done.  The
 * winning split count is recorded in the process-wide plan cache, which later
 * tsmm_plan calls for the same (dtype, m, n, k) on a GPU with the same SM count
 * reuse -- and, when no exact entry exists, calls for the same (dtype, n, k)
 * whose m lies in the same quarter octave (2^(b/4) <= m < 2^((b+1)/4)); a new
 * plan with it is returned in *out.  Regime (ii) shapes have no
 * tuned parameter yet and return the default plan.  Errors: as tsmm_plan and
 * tsmm_execute; INVALID_ARG for reps outside 1..1000.
 */
TSMM_API tsmm_status tsmm_autotune(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype,
                                   const void *A_dev, int64_t lda, tsmm_packed_b pb, void *C_dev,
                                   int64_t ldc, tsmm_stream_t stream, int reps, tsmm_plan_t *out);

/*
 * The plan cache (the install-time record of tuned choices).  Text format, one
 * entry per line: `f32|f64 m n k sm_count splits` for an exact m, or
 * `f32q|f64q b n k sm_count splits` for every m of quarter-octave bucket b
 * (b = floor(4 log2 m)); lines starting with '#' are comments.  If the environment variable TSMM_PLAN_CACHE names a file, it is
 * loaded on first use.  load merges a file into the cache (INVALID_ARG if the
 * file is missing or malformed, leaving the cache unchanged); save writes the
 * whole cache; clear empties it; size returns the number of entries (exact
 * and bucket entries together).  The
 * cache is guarded by a mutex and shared by all threads of the process.
 */
TSMM_API tsmm_status tsmm_plan_cache_load(const char *path);
TSMM_API tsmm_status tsmm_plan_cache_save(const char *path);
TSMM_API tsmm_status tsmm_plan_cache_clear(void);
TSMM_API int64_t tsmm_plan_cache_size(void);

/*
 * Serving runtime: a request loop with continuous batching against
 * device-resident packed B matrices (the reuse that pre-packing pays for,
 * Section III).  A scheduler thread owned by the server releases submitted
 * requests once their arrival time (on the tsmm_server_clock clock) has
 * passed, admits them in arrival order while the device memory that admitted,
 * unfinished requests pin -- A (m x k), C (m x n) and the split-K workspace --
 * stays within budget_bytes, and launches every group of admitted requests on
 * one of num_streams lanes as soon as a lane is free: requests admitted while
 * earlier batches run form the next batch and overlap with them on the device.
 * A batch runs cheapest request first, as up to six grouped sub-batches with
 * one completion event each (CUDA events): a new sub-batch starts at a request
 * that alone holds at least the bytes of the current one (and 256 MiB), so a
 * small request completes with its sub-batch, not with a much larger request.  A
 * lane is three high-priority streams and one low-priority stream: the first
 * sub-batch runs as grouped launches, one per kernel class, spread over the
 * high-priority streams; the others run on the low-priority stream.  Every
 * grouped launch has one thread block per work item, so newly launched small
 * work gets SMs as items finish.
 * Each request's plan depends only on its shape, so its result is the same bit
 * for bit alone or in any mix.  The caller owns A, C and the packed B, and must
 * keep them alive until the request's completion has been polled.
 *
 * Ordering contract: the server's streams are not ordered after the caller's
 * streams.  A, C0 (the prior content of C) and the packed B must be complete
 * on the device -- the caller's streams that write them synchronized -- before
 * the request's arrival time (before tsmm_server_submit for a request whose
 * arrival time has already passed).  From submission until the request's
 * completion has been polled the caller must not write A, C or the packed B
 * and must not read C; after the completion is polled, C holds the result and
 * no server work touches A, C or the packed B any more.
 */
typedef struct tsmm_server_s *tsmm_server_t;

typedef struct tsmm_server_config {
    size_t budget_bytes;  /* device memory admitted, unfinished requests may pin (> 0) */
    size_t arena_bytes;   /* split-K workspace arena allocated once (0 = 256 MiB); a request's
                             workspace is capped at a quarter of it */
    int num_streams;      /* lanes (batches that may run concurrently), 1..16 */
    int max_batch;        /* requests per launch group, 1..1024 */
    tsmm_dtype dtype;     /* every request's dtype */
} tsmm_server_config;

typedef struct tsmm_request {
    uint64_t id;          /* caller's tag, returned with the completion */
    tsmm_packed_b pb;     /* packed B (native precision, the server's dtype and device) */
    int64_t m;            /* rows of A and C; k and n come from pb */
    double alpha, beta;
    const void *A_dev;    /* m x k, column-major, lda >= max(1, m) */
    int64_t lda;
    void *C_dev;          /* m x n, column-major, ldc >= max(1, m); C0 on input */
    int64_t ldc;
    double arrival_s;     /* arrival time on tsmm_server_clock(); may be in the future */
} tsmm_request;

typedef struct tsmm_completion {
    uint64_t id;
    double arrival_s, admit_s, launch_s, complete_s; /* tsmm_server_clock() times */
    int status;                                      /* tsmm_status of the request */
} tsmm_completion;

/* Create a server on the current device (allocates its arena, streams, events
   and starts its scheduler thread).  INVALID_ARG for a NULL argument, a dtype
   other than F32/F64, budget_bytes == 0, num_streams outside 1..16 or max_batch
   outside 1..1024; OUT_OF_MEMORY / CUDA if an allocation fails (nothing is
   left allocated).  *out is written only on TSMM_OK; the server owns
   everything it allocates until tsmm_server_destroy. */
TSMM_API tsmm_status tsmm_server_create(const tsmm_server_config *cfg, tsmm_server_t *out);
/* Queue requests (thread-safe).  INVALID_ARG for a request that could never be
   admitted (its bytes exceed the budget) or has bad arguments; none of the
   requests of a failing call is queued. */
TSMM_API tsmm_status tsmm_server_submit(tsmm_server_t s, const tsmm_request *reqs, int count);
/* Wait until every submitted request has completed (TIMEOUT after timeout_s
   seconds, INVALID_ARG for a NULL server).  A request whose kernels gave up
   (a bounded wait ran out) completes with status TSMM_ERR_TIMEOUT. */
TSMM_API tsmm_status tsmm_server_drain(tsmm_server_t s, double timeout_s);
/* Move up to max completions into out (completion order); returns how many
   (0 for a NULL server or out, or max <= 0). */
TSMM_API int64_t tsmm_server_poll(tsmm_server_t s, tsmm_completion *out, int64_t max);
/* Stop the scheduler (requests not yet admitted are dropped), wait for the
   admitted ones, free everything. */
TSMM_API tsmm_status tsmm_server_destroy(tsmm_server_t s);
/* The server's clock: steady, in seconds. */
TSMM_API double tsmm_server_clock(void);

/*
 * tsmm_diag_server_inject_timeout -- diagnostics for the serving failure path
 * (no counterpart in the paper).  The next `units` launch units the server
 * starts finish as if a bounded wait in one of their kernels had run out:
 * after the unit's kernels, on the unit's stream, its status word is set to the
 * timeout record and the split-K arrival counters of its requests are left
 * non-zero (what a block that gave up before taking its ticket leaves behind).
 * The unit's requests then complete with TSMM_ERR_TIMEOUT, and the server
 * must clear those counters before it hands them to later requests.  Nothing
 * faults, traps or hangs.  Errors: INVALID_ARG for a NULL server or units < 0.
 */
TSMM_API tsmm_status tsmm_diag_server_inject_timeout(tsmm_server_t s, int units);

/* Size of the library's built-in device scratch used by tsmm_execute_noalloc. */
#define TSMM_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * tsmm_execute_noalloc -- C = alpha * A * B + beta * C0 for regime (i) shapes
 * (n <= 64) without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * -- code whose device memory is owned and budgeted by a host framework (an
 * inference engine or plug-in host that forbids allocations of its own), and
 * latency-critical loops that cannot afford cudaMalloc's implicit device
 * synchronisation.  Such callers cannot use tsmm_pack_b or tsmm_plan, which
 * allocate.
 *
 * The caller passes the unpacked B (k x n, column-major, ldb) together with A
 * and C exactly as for tsmm_execute.  Every call packs B and runs the same
 * split-K kernel as tsmm_execute, with the packed B, the split-K partial
 * tiles, the arrival counters and the error word all placed in one file-scope
 * device array of TSMM_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading
 * the library holds until the process exits.  The k split is reduced so the
 * partial tiles fit; sizes whose packed B (k rounded up to 32, times n rounded
 * up to one of 1, 2, 4, 8, 16, 24, 32, 48, 64, times the element size) plus one arrival counter per
 * m-slab (256 rows for F32 with n <= 48, 128 for F32 with n > 48, 64 for F64; the plan's bm)
 * do not fit return TSMM_ERR_UNSUPPORTED_SHAPE
 * before any device work, as do shapes with n > 64.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make the first call on
 * a device before any stream capture.  All calls share the one array and it
 * keeps the previous call's contents: each call clears the counters and error
 * word it needs on `stream` first.  Calls whose work can overlap on the GPU
 * (different streams, or different host threads on the same device) race on
 * the array and give wrong results; serialise them.  Device-side timeouts of
 * this entry point are not reported (there is no plan to check); the output
 * tile of a block that gave up is left unwritten.
 *
 * Errors: INVALID_ARG, UNSUPPORTED_SHAPE, MISALIGNED, CUDA, as for
 * tsmm_pack_b and tsmm_execute.  Enqueues up to three operations on `stream`
 * (a memset, the pack, the TSMM kernel) and returns without waiting.
 */
TSMM_API tsmm_status tsmm_execute_noalloc(tsmm_dtype dtype, int64_t m, int64_t n, int64_t k,
                                          double alpha, const void *A_dev, int64_t lda,
                                          const void *B_dev, int64_t ldb, double beta,
                                          void *C_dev, int64_t ldc, tsmm_stream_t stream);

/*
 * tsmm_diag_bounded_wait -- diagnostics for the failure path (no counterpart
 * in the paper).  Every wait on an mbarrier in the library's kernels gives up
 * after one second (or 2^24 polls) and, if the phase never completed, records
 * TSMM_ERR_TIMEOUT in a device status word and lets the kernel return.  This
 * entry point runs that same wait, with at most `polls` polls, against a
 * barrier that nothing completes, in one block of one warp, synchronously.
 * Returns TSMM_ERR_TIMEOUT when the wait ran out (the expected outcome),
 * TSMM_OK if the phase was seen complete, INVALID_ARG for polls == 0, CUDA on
 * an allocation, launch or copy error.  *cycles_out (may be NULL): SM clock
 * cycles the wait took; *seconds_out (may be NULL): the same at the device's
 * maximum SM clock.  Allocates and frees 16 bytes of device memory.
 */
TSMM_API tsmm_status tsmm_diag_bounded_wait(uint32_t polls, uint64_t *cycles_out, double *seconds_out);

/*
 * tsmm_diag_fp_peak -- measures the throughput of one arithmetic pipe of the
 * current GPU, for the roofline denominators of the compute-bound shapes
 * (Eq. 7 rates are judged against it) and for the choice between the FP64
 * FMA and FP64 MMA instructions (the GPU counterpart of the paper's
 * install-time kernel selection, Section IV.B, decided by measurement).
 *
 * pipe: TSMM_DIAG_FFMA (FP32 fma), TSMM_DIAG_FFMA2 (packed FP32x2 fma, the
 * instruction the FP32 kernels use), TSMM_DIAG_DFMA (FP64 fma),
 * TSMM_DIAG_DMMA (FP64 mma.sync m8n8k4).  The kernel runs blocks_per_sm
 * blocks of 256 threads on every SM; each thread runs independent chains of
 * the instruction for `iters` loop trips.  One short untimed launch, then one
 * timed launch between CUDA events on a private stream; synchronous.
 * *flops_out: flops of the timed launch (2 per fma lane, 512 per DMMA warp
 * instruction); *ms_out: its duration; *cycles_out: the longest block's SM
 * clock cycles (cycles / ms gives the SM clock the launch ran at).  Output
 * pointers may be NULL.  Errors: INVALID_ARG (pipe out of range, iters == 0,
 * blocks_per_sm outside 1..8), CUDA.  Allocates and frees a few KB of device
 * memory; changes no device setting.
 */
enum { TSMM_DIAG_FFMA = 0, TSMM_DIAG_FFMA2 = 1, TSMM_DIAG_DFMA = 2, TSMM_DIAG_DMMA = 3 };
TSMM_API tsmm_status tsmm_diag_fp_peak(int pipe, uint32_t iters, int blocks_per_sm, double *flops_out,
                                       double *ms_out, uint64_t *cycles_out);

#ifdef __cplusplus
}
#endif

#endif /* TSMM_H */
