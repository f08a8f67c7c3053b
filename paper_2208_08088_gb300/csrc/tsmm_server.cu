// Serving runtime: a request loop with continuous batching over device-resident
// pre-packed B matrices -- the reuse scenario that motivates pre-packing in the
// paper (Section III: the execution plan and the packed operand are reused by
// many executions, so their cost is amortised).
//
// A scheduler thread owned by the server:
//   * releases submitted requests when their arrival time has passed;
//   * admits them in arrival order (FIFO) while the device memory pinned by
//     admitted, unfinished requests (A + C + split-K workspace) stays within the
//     budget, and while a workspace slice fits in the server's arena;
//   * launches the admitted requests as a batch on a free lane as soon as one
//     is free -- requests admitted while other batches are on the GPU form the
//     next batch, so their work overlaps.  A batch goes out cheapest request
//     first, as a few grouped sub-batches of growing size, each with its own
//     completion event: a small request is done when its sub-batch is, not when
//     the largest request launched with it is.  Each lane has three
//     high-priority streams and one low-priority stream: the first sub-batch
//     runs as grouped launches, one per kernel class, side by side on the
//     high-priority streams; the rest run on the low-priority one.  A grouped
//     launch has one block per work item, so the GPU's block scheduler hands
//     SMs to newly launched small work as items finish;
//   * detects sub-batch completion with CUDA events, records completion times
//     and returns the sub-batch's memory to the budget and the arena.  Each
//     launch unit has its own device status word, so a bounded wait that gave
//     up is charged to the unit whose kernel gave up.  A unit that failed may
//     have left split-K arrival counters part-way (a block that gave up never
//     takes its ticket): its counter slices are cleared on its own stream, and
//     only returned to the arena once that clear has completed.
// Results are deterministic: each request's plan depends only on its shape,
// never on what else is in flight.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "tsmm_device.cuh"
#include "tsmm_internal.h"

using namespace tsmm;

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

// First-fit allocator over one device buffer (offsets aligned to 256 bytes).
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes
    void init(size_t bytes) {
        size = bytes;
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Req {
    tsmm_request r;
    tsmm_plan_s plan;
    size_t ticket_bytes = 0;
    size_t bytes = 0;  // budget charge: A + C + workspace
    size_t ws_off = 0, tk_off = 0;
    double admit_s = 0, launch_s = 0;
};

struct Batch {
    std::vector<Req *> reqs;
    cudaEvent_t ev = nullptr;
    cudaStream_t st = nullptr;  // the stream its kernels (and a clean-up) run on
    int lane = -1;
    int slot = -1;              // its status word
    int fail = TSMM_OK;         // status decided before the event completes
    bool cleaning = false;      // the event now marks the end of the counter clean-up
};

// Status words (mapped, pinned host memory; one per launch unit in flight).
// A launch has at most one unit per kernel class plus kMaxSubBatches - 1, on
// at most 16 lanes: far below this.
constexpr int kStatusSlots = 1024;

// Diagnostics: the effect a kernel that gave up on a bounded wait leaves
// behind -- its status word set -- written by a kernel of its own.
__global__ void diag_flag_timeout_kernel(unsigned *status) { atomicOr(status, kDevErrTimeout); }

// Sub-batches per launch (requests in ascending order of bytes, A + C +
// workspace): a new sub-batch starts at a request that alone holds at least as
// many bytes as the current sub-batch and at least kSubBatchMinBytes, so no
// request waits for one much larger than its whole sub-batch, and their count
// grows with the log of the batch's size spread (at most kMaxSubBatches).
constexpr int kMaxSubBatches = 6;
constexpr size_t kSubBatchMinBytes = size_t(256) << 20;
// Streams of a lane: kHighStreams at high priority, then one at low priority.
constexpr int kHighStreams = 3;
constexpr int kLaneStreams = kHighStreams + 1;

}  // namespace

struct tsmm_server_s {
    tsmm_server_config cfg;
    int dev = 0, sms = 0;
    std::vector<cudaStream_t> streams;    // lane i: kLaneStreams from i * kLaneStreams (high, ..., low)
    std::vector<int> lane_pending;        // launch units in flight per lane (busy while > 0)
    std::vector<cudaEvent_t> events;      // all of them (grown on demand)
    std::vector<cudaEvent_t> free_events;  // not recorded by an in-flight unit
    void *ws_base = nullptr;
    void *tk_base = nullptr;
    unsigned *status_host = nullptr;  // kStatusSlots words, mapped, pinned
    unsigned *status_dev = nullptr;   // their device address
    std::vector<int> free_slots;
    Arena ws_arena, tk_arena;
    std::atomic<int> inject_units{0};  // tsmm_diag_server_inject_timeout

    std::mutex mu;
    std::condition_variable cv_done;
    std::multimap<double, Req *> pending;  // submitted, keyed by arrival time
    std::deque<tsmm_completion> completions;
    int64_t submitted = 0, completed = 0;
    tsmm_status fault = TSMM_OK;

    // scheduler-thread state
    std::deque<Req *> ready;
    std::vector<Req *> forming;
    std::vector<Batch> inflight;
    size_t inflight_bytes = 0;
    std::atomic<bool> stop{false};
    std::thread th;

    void run();
    bool try_admit(Req *q, double t);
    void launch(double t);
    bool poll_batches();
    void finish(Batch &b, int status, double t);
    bool start_cleanup(Batch &b, int status);
};

bool tsmm_server_s::try_admit(Req *q, double t) {
    if (inflight_bytes + q->bytes > cfg.budget_bytes) return false;
    if (q->plan.workspace_bytes && !ws_arena.alloc(q->plan.workspace_bytes, &q->ws_off)) return false;
    if (q->ticket_bytes && !tk_arena.alloc(q->ticket_bytes, &q->tk_off)) {
        if (q->plan.workspace_bytes) ws_arena.release(q->ws_off, q->plan.workspace_bytes);
        return false;
    }
    q->plan.workspace = q->plan.workspace_bytes ? static_cast<char *>(ws_base) + q->ws_off : nullptr;
    q->plan.tickets = q->ticket_bytes
                          ? reinterpret_cast<unsigned *>(static_cast<char *>(tk_base) + q->tk_off)
                          : nullptr;
    q->plan.status = nullptr;  // the launch unit's own word, set in launch()
    q->admit_s = t;
    inflight_bytes += q->bytes;
    return true;
}

void tsmm_server_s::launch(double t) {
    int s = -1;
    for (int i = 0; i < (int)lane_pending.size(); ++i)
        if (lane_pending[i] == 0) {
            s = i;
            break;
        }
    if (s < 0 || forming.empty()) return;
    // cheapest first (stable: arrival order among equals), cut into sub-batches
    std::vector<Req *> reqs;
    reqs.swap(forming);
    std::stable_sort(reqs.begin(), reqs.end(), [](const Req *x, const Req *y) { return x->bytes < y->bytes; });
    std::vector<size_t> cuts;  // end index of each sub-batch
    size_t cur = 0;
    for (size_t i = 0; i < reqs.size(); ++i) {
        const size_t b = reqs[i]->bytes;
        if (cur > 0 && (int)cuts.size() + 1 < kMaxSubBatches && b >= cur && b >= kSubBatchMinBytes) {
            cuts.push_back(i);
            cur = 0;
        }
        cur += b;
        reqs[i]->launch_s = t;
    }
    cuts.push_back(reqs.size());
    // launch units: the first sub-batch split by kernel class (one grouped launch
    // each), spread over the lane's high-priority streams so the classes run side
    // by side; every later sub-batch one unit on the low-priority stream
    struct Unit {
        std::vector<Req *> reqs;
        cudaStream_t st;
    };
    std::vector<Unit> units;
    {
        std::map<int, std::vector<Req *>> by_class;
        for (size_t i = 0; i < cuts[0]; ++i) {
            // kernel class: regime, padded width, whether a tensor map can describe
            // A, and if not the load form of the kernel that reads it
            const tsmm_request &r = reqs[i]->r;
            const tsmm_plan_s &pl = reqs[i]->plan;
            const int64_t es = (int64_t)dtype_size(pl.dtype);
            const bool unaligned = reinterpret_cast<uintptr_t>(r.A_dev) % 16 != 0 || (r.lda * es) % 16 != 0;
            const int form = unaligned ? 1 + (1 + async_load_variant(pl.dtype == TSMM_F32, pl.np, r.A_dev, r.lda)) : 0;
            by_class[pl.regime * 1024 + form * 128 + pl.np].push_back(reqs[i]);
        }
        int h = 0;
        for (auto &kv : by_class)
            units.push_back(Unit{std::move(kv.second), streams[kLaneStreams * s + (h++ % kHighStreams)]});
        for (size_t c = 1; c < cuts.size(); ++c)
            units.push_back(Unit{std::vector<Req *>(reqs.begin() + cuts[c - 1], reqs.begin() + cuts[c]),
                                 streams[kLaneStreams * s + kHighStreams]});
    }
    tsmm_status st = TSMM_OK;
    for (Unit &u : units) {
        Batch b;
        b.reqs = std::move(u.reqs);
        b.st = u.st;
        if (st == TSMM_OK) {
            if (free_events.empty()) {
                cudaEvent_t ev;
                if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
                    events.push_back(ev);
                    free_events.push_back(ev);
                }
            }
            if (free_events.empty() || free_slots.empty()) {
                st = TSMM_ERR_CUDA;  // nothing of this unit was enqueued
            } else {
                b.ev = free_events.back();
                free_events.pop_back();
                b.slot = free_slots.back();
                free_slots.pop_back();
                status_host[b.slot] = 0u;
                std::vector<tsmm_group_item> items(b.reqs.size());
                for (size_t i = 0; i < b.reqs.size(); ++i) {
                    Req *q = b.reqs[i];
                    q->plan.status = status_dev + b.slot;
                    const tsmm_request &r = q->r;
                    items[i] = tsmm_group_item{&q->plan, r.alpha, r.A_dev, r.lda, r.pb, r.beta, r.C_dev, r.ldc};
                }
                st = execute_grouped(items.data(), (int)items.size(), u.st);
                if (st == TSMM_OK && inject_units.load() > 0) {
                    // diagnostics: leave what a block that gave up leaves -- the unit's
                    // status word set and its arrival counters part-way
                    --inject_units;
                    diag_flag_timeout_kernel<<<1, 1, 0, u.st>>>(status_dev + b.slot);
                    for (Req *q : b.reqs)
                        if (q->ticket_bytes) cudaMemsetAsync(q->plan.tickets, 0x01, q->ticket_bytes, u.st);
                    if (cudaGetLastError() != cudaSuccess) st = TSMM_ERR_CUDA;
                }
                // Recorded even when the launch failed: kernels enqueued before the
                // failure may still be running, and the unit's memory stays in use
                // until they are done.
                if (cudaEventRecord(b.ev, u.st) != cudaSuccess) {
                    // wait for what was enqueued, then clear the counters it may have
                    // left part-way before the slices go back to the arena
                    cudaStreamSynchronize(u.st);
                    cudaGetLastError();
                    for (Req *q : b.reqs)
                        if (q->ticket_bytes) cudaMemset(q->plan.tickets, 0, q->ticket_bytes);
                    cudaDeviceSynchronize();
                    cudaGetLastError();
                    if (st == TSMM_OK) st = TSMM_ERR_CUDA;
                    finish(b, st, now_s());
                    continue;
                }
            }
            if (b.ev) {
                b.lane = s;
                b.fail = st;
                ++lane_pending[s];
                inflight.push_back(std::move(b));
                continue;
            }
        }
        finish(b, st, now_s());  // a unit after a failed one: nothing of it was enqueued
    }
}

// A unit finished with an error: its split-K arrival counters may be left
// part-way, which would make the next request given the same slices pick the
// wrong last-arriving block.  Clear them on the unit's stream and keep the
// unit in flight until the clear is done.  Returns false (and waits for the
// stream) if the clear could not be enqueued.
bool tsmm_server_s::start_cleanup(Batch &b, int status) {
    bool any = false;
    cudaError_t e = cudaSuccess;
    for (Req *q : b.reqs)
        if (q->ticket_bytes && e == cudaSuccess) {
            e = cudaMemsetAsync(q->plan.tickets, 0, q->ticket_bytes, b.st);
            any = true;
        }
    if (!any) return false;
    if (e == cudaSuccess) e = cudaEventRecord(b.ev, b.st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (Req *q : b.reqs)
            if (q->ticket_bytes) cudaMemset(q->plan.tickets, 0, q->ticket_bytes);
        cudaDeviceSynchronize();
        cudaGetLastError();
        return false;
    }
    b.cleaning = true;
    b.fail = status;
    return true;
}

void tsmm_server_s::finish(Batch &b, int status, double t) {
    if (b.ev) free_events.push_back(b.ev);
    if (b.slot >= 0) free_slots.push_back(b.slot);
    std::lock_guard<std::mutex> lock(mu);
    for (Req *q : b.reqs) {
        inflight_bytes -= q->bytes;
        if (q->plan.workspace_bytes) ws_arena.release(q->ws_off, q->plan.workspace_bytes);
        if (q->ticket_bytes) tk_arena.release(q->tk_off, q->ticket_bytes);
        completions.push_back(
            tsmm_completion{q->r.id, q->r.arrival_s, q->admit_s, q->launch_s, t, status});
        delete q;
        ++completed;
    }
    if (b.lane >= 0) --lane_pending[b.lane];
    cv_done.notify_all();
}

bool tsmm_server_s::poll_batches() {
    bool progress = false;
    for (size_t i = 0; i < inflight.size();) {
        Batch &ib = inflight[i];
        cudaError_t e = cudaEventQuery(ib.ev);
        if (e == cudaErrorNotReady) {
            ++i;
            continue;
        }
        progress = true;
        int status = ib.fail;
        if (!ib.cleaning) {
            if (e != cudaSuccess) status = TSMM_ERR_CUDA;
            // this unit's give-up record lives in mapped host memory: read it directly
            volatile unsigned *word = status_host + ib.slot;
            if (e == cudaSuccess && *word != 0u) {
                if (status == TSMM_OK) status = TSMM_ERR_TIMEOUT;
                *word = 0u;
            }
            if (status != TSMM_OK && start_cleanup(ib, status)) {
                ++i;  // finished once the clear has completed
                continue;
            }
        }
        Batch b = std::move(ib);
        inflight.erase(inflight.begin() + i);
        finish(b, status, now_s());
    }
    return progress;
}

void tsmm_server_s::run() {
    cudaSetDevice(dev);
    for (;;) {
        bool progress = false;
        const double t = now_s();
        {
            std::lock_guard<std::mutex> lock(mu);
            while (!pending.empty() && pending.begin()->first <= t) {
                ready.push_back(pending.begin()->second);
                pending.erase(pending.begin());
                progress = true;
            }
        }
        // admission in arrival order while memory allows; batch what was admitted
        while (!stop.load() && !ready.empty() && (int)forming.size() < cfg.max_batch) {
            if (!try_admit(ready.front(), t)) break;
            forming.push_back(ready.front());
            ready.pop_front();
            progress = true;
        }
        if (!forming.empty()) {
            const size_t before = inflight.size();
            launch(t);
            progress |= inflight.size() != before;
        }
        progress |= poll_batches();
        // on shutdown, requests not yet admitted are dropped; admitted ones finish
        if (stop.load() && forming.empty() && inflight.empty()) break;
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" {

double tsmm_server_clock(void) { return now_s(); }

tsmm_status tsmm_server_create(const tsmm_server_config *cfg, tsmm_server_t *out) {
    if (!cfg || !out) return TSMM_ERR_INVALID_ARG;
    if ((cfg->dtype != TSMM_F32 && cfg->dtype != TSMM_F64) || cfg->budget_bytes == 0 ||
        cfg->num_streams < 1 || cfg->num_streams > 16 || cfg->max_batch < 1 || cfg->max_batch > 1024)
        return TSMM_ERR_INVALID_ARG;
    tsmm_server_t s = new (std::nothrow) tsmm_server_s();
    if (!s) return TSMM_ERR_OUT_OF_MEMORY;
    s->cfg = *cfg;
    if (s->cfg.arena_bytes == 0) s->cfg.arena_bytes = 256u << 20;
    cudaError_t e = cudaGetDevice(&s->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->dev);
    const size_t tk_bytes = 16u << 20;
    if (e == cudaSuccess) e = cudaMalloc(&s->ws_base, s->cfg.arena_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->tk_base, tk_bytes);
    if (e == cudaSuccess) e = cudaMemset(s->tk_base, 0, tk_bytes);  // arrival counters start at 0
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&s->status_host), kStatusSlots * sizeof(unsigned),
                          cudaHostAllocMapped);
    if (e == cudaSuccess) {
        for (int i = 0; i < kStatusSlots; ++i) s->status_host[i] = 0u;
        e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->status_dev), s->status_host, 0);
    }
    int prio_low = 0, prio_high = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    for (int i = 0; e == cudaSuccess && i < cfg->num_streams; ++i) {
        for (int h = 0; e == cudaSuccess && h < kLaneStreams; ++h) {
            cudaStream_t st;
            e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, h < kHighStreams ? prio_high : prio_low);
            if (e == cudaSuccess) s->streams.push_back(st);
        }
        for (int j = 0; e == cudaSuccess && j < kMaxSubBatches; ++j) {
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) s->events.push_back(ev);
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (auto st : s->streams) cudaStreamDestroy(st);
        for (auto ev : s->events) cudaEventDestroy(ev);
        if (s->ws_base) cudaFree(s->ws_base);
        if (s->tk_base) cudaFree(s->tk_base);
        if (s->status_host) cudaFreeHost(s->status_host);
        delete s;
        return e == cudaErrorMemoryAllocation ? TSMM_ERR_OUT_OF_MEMORY : TSMM_ERR_CUDA;
    }
    s->lane_pending.assign(cfg->num_streams, 0);
    s->free_events = s->events;
    for (int i = kStatusSlots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->ws_arena.init(s->cfg.arena_bytes);
    s->tk_arena.init(tk_bytes);
    s->th = std::thread([s] { s->run(); });
    *out = s;
    return TSMM_OK;
}

tsmm_status tsmm_server_submit(tsmm_server_t s, const tsmm_request *reqs, int count) {
    if (!s || count < 0 || (count > 0 && !reqs)) return TSMM_ERR_INVALID_ARG;
    std::vector<Req *> made;
    made.reserve(count);
    tsmm_status st = TSMM_OK;
    for (int i = 0; i < count && st == TSMM_OK; ++i) {
        const tsmm_request &r = reqs[i];
        tsmm_packed_b pb = r.pb;
        if (!pb || pb->dtype != s->cfg.dtype || pb->precision != TSMM_PREC_NATIVE || r.m < 0 ||
            r.lda < std::max<int64_t>(1, r.m) || r.ldc < std::max<int64_t>(1, r.m) ||
            (r.m > 0 && pb->n > 0 && !r.C_dev) || (r.m > 0 && pb->k > 0 && r.alpha != 0.0 && !r.A_dev)) {
            st = TSMM_ERR_INVALID_ARG;
            break;
        }
        if (pb->device != s->dev) {
            st = TSMM_ERR_MISMATCH;
            break;
        }
        Req *q = new (std::nothrow) Req();
        if (!q) {
            st = TSMM_ERR_OUT_OF_MEMORY;
            break;
        }
        q->r = r;
        const int cached = plan_cache_lookup(s->cfg.dtype, r.m, pb->n, pb->k, s->sms);
        st = plan_layout(r.m, pb->n, pb->k, s->cfg.dtype, cached, TSMM_PREC_NATIVE, s->dev, s->sms,
                         (int64_t)(s->cfg.arena_bytes / 4), &q->plan, &q->ticket_bytes);
        const size_t es = dtype_size(s->cfg.dtype);
        q->bytes = es * (size_t)r.m * (size_t)(pb->k + pb->n) + q->plan.workspace_bytes;
        if (st == TSMM_OK && (q->bytes > s->cfg.budget_bytes || q->ticket_bytes > (16u << 20)))
            st = TSMM_ERR_INVALID_ARG;  // could never be admitted
        if (st != TSMM_OK) {
            delete q;
            break;
        }
        made.push_back(q);
    }
    if (st != TSMM_OK) {
        for (Req *q : made) delete q;
        return st;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    for (Req *q : made) s->pending.emplace(q->r.arrival_s, q);
    s->submitted += (int64_t)made.size();
    return TSMM_OK;
}

int64_t tsmm_server_poll(tsmm_server_t s, tsmm_completion *out, int64_t max) {
    if (!s || !out || max <= 0) return 0;
    std::lock_guard<std::mutex> lock(s->mu);
    int64_t n = 0;
    while (n < max && !s->completions.empty()) {
        out[n++] = s->completions.front();
        s->completions.pop_front();
    }
    return n;
}

tsmm_status tsmm_server_drain(tsmm_server_t s, double timeout_s) {
    if (!s) return TSMM_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                        [s] { return s->completed >= s->submitted; });
    return ok ? TSMM_OK : TSMM_ERR_TIMEOUT;
}

tsmm_status tsmm_diag_server_inject_timeout(tsmm_server_t s, int units) {
    if (!s || units < 0) return TSMM_ERR_INVALID_ARG;
    s->inject_units.store(units);
    return TSMM_OK;
}

tsmm_status tsmm_server_destroy(tsmm_server_t s) {
    if (!s) return TSMM_OK;
    s->stop.store(true);
    if (s->th.joinable()) s->th.join();
    for (auto st : s->streams) cudaStreamSynchronize(st);
    for (auto &kv : s->pending) delete kv.second;
    for (Req *q : s->ready) delete q;
    for (auto st : s->streams) cudaStreamDestroy(st);
    for (auto ev : s->events) cudaEventDestroy(ev);
    cudaFree(s->ws_base);
    cudaFree(s->tk_base);
    cudaFreeHost(s->status_host);
    delete s;
    return TSMM_OK;
}

}  // extern "C"
