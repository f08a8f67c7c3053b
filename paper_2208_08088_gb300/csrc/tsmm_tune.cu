// Autotuner and plan cache: the GPU counterpart of the paper's performance
// evaluator (Section III), which times the candidate blocking / threading
// strategies of the runtime stage and keeps the fastest as the execution plan,
// and of its install-time stage, whose selection is made once per machine and
// reused.  Here the candidates are split-K factors of the regime (i) kernel;
// the winner is remembered in a process-wide cache keyed by (dtype, m, n, k,
// SM count) -- and by (dtype, quarter-octave bucket of m, n, k, SM count), so a
// tuned choice also serves the other m of its bucket -- that tsmm_plan
// consults, and that can be saved to and loaded from a text file
// (TSMM_PLAN_CACHE names one to load on first use).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "tsmm_device.cuh"
#include "tsmm_internal.h"

using namespace tsmm;

namespace {

using Key = std::tuple<int, int64_t, int64_t, int64_t, int>;

std::mutex g_cache_mu;
std::map<Key, int> g_cache;   // exact m
std::map<Key, int> g_bucket;  // m replaced by its bucket
bool g_env_loaded = false;

// quarter-octave bucket of m >= 1: floor(4 log2 m); 2^(b/4) <= m < 2^((b+1)/4)
int64_t m_bucket(int64_t m) {
    return m < 1 ? -1 : (int64_t)std::floor(4.0 * std::log2((double)m) + 1e-9);
}

tsmm_status load_file_locked(const char *path) {
    FILE *f = std::fopen(path, "r");
    if (!f) return TSMM_ERR_INVALID_ARG;
    char line[512];
    std::map<Key, int> parsed, parsed_b;
    bool bad = false;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n' || line[0] == '\0') continue;
        char dt[8] = {0};
        long long m, n, k;
        int sms, splits;
        if (std::sscanf(line, "%7s %lld %lld %lld %d %d", dt, &m, &n, &k, &sms, &splits) != 6 ||
            splits < 1 || m < 0 || n < 0 || k < 0) {
            bad = true;
            break;
        }
        const std::string t(dt);
        const bool bucket = t == "f32q" || t == "f64q";
        int d;
        if (t == "f32" || t == "f32q")
            d = TSMM_F32;
        else if (t == "f64" || t == "f64q")
            d = TSMM_F64;
        else {
            bad = true;
            break;
        }
        (bucket ? parsed_b : parsed)[Key(d, m, n, k, sms)] = splits;
    }
    std::fclose(f);
    if (bad) return TSMM_ERR_INVALID_ARG;
    for (auto &kv : parsed) g_cache[kv.first] = kv.second;
    for (auto &kv : parsed_b) g_bucket[kv.first] = kv.second;
    return TSMM_OK;
}

void load_env_once_locked() {
    if (g_env_loaded) return;
    g_env_loaded = true;
    const char *p = std::getenv("TSMM_PLAN_CACHE");
    if (p && *p) load_file_locked(p);  // a missing or malformed file leaves the cache empty
}

}  // namespace

namespace tsmm {

int plan_cache_lookup(tsmm_dtype dtype, int64_t m, int64_t n, int64_t k, int sms) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    load_env_once_locked();
    auto it = g_cache.find(Key(dtype, m, n, k, sms));
    if (it != g_cache.end()) return it->second;
    auto ib = g_bucket.find(Key(dtype, m_bucket(m), n, k, sms));
    return ib == g_bucket.end() ? 0 : ib->second;
}

void plan_cache_store(tsmm_dtype dtype, int64_t m, int64_t n, int64_t k, int sms, int splits) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    load_env_once_locked();
    g_cache[Key(dtype, m, n, k, sms)] = splits;
    g_bucket[Key(dtype, m_bucket(m), n, k, sms)] = splits;
}

}  // namespace tsmm

extern "C" {

tsmm_status tsmm_plan_cache_load(const char *path) {
    if (!path) return TSMM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_cache_mu);
    load_env_once_locked();
    return load_file_locked(path);
}

tsmm_status tsmm_plan_cache_save(const char *path) {
    if (!path) return TSMM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_cache_mu);
    FILE *f = std::fopen(path, "w");
    if (!f) return TSMM_ERR_INVALID_ARG;
    std::fprintf(f, "# tsmm plan cache v2: dtype m n k sm_count splits (dtype f32q/f64q: m is a "
                    "quarter-octave bucket)\n");
    for (auto &kv : g_cache) {
        std::fprintf(f, "%s %lld %lld %lld %d %d\n", std::get<0>(kv.first) == TSMM_F64 ? "f64" : "f32",
                     (long long)std::get<1>(kv.first), (long long)std::get<2>(kv.first),
                     (long long)std::get<3>(kv.first), std::get<4>(kv.first), kv.second);
    }
    for (auto &kv : g_bucket) {
        std::fprintf(f, "%s %lld %lld %lld %d %d\n", std::get<0>(kv.first) == TSMM_F64 ? "f64q" : "f32q",
                     (long long)std::get<1>(kv.first), (long long)std::get<2>(kv.first),
                     (long long)std::get<3>(kv.first), std::get<4>(kv.first), kv.second);
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? TSMM_OK : TSMM_ERR_INVALID_ARG;
}

tsmm_status tsmm_plan_cache_clear(void) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    g_env_loaded = true;  // an explicit clear also drops the environment's file
    g_cache.clear();
    g_bucket.clear();
    return TSMM_OK;
}

int64_t tsmm_plan_cache_size(void) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    load_env_once_locked();
    return (int64_t)(g_cache.size() + g_bucket.size());
}

tsmm_status tsmm_autotune(int64_t m, int64_t n, int64_t k, tsmm_dtype dtype, const void *A_dev,
                          int64_t lda, tsmm_packed_b pb, void *C_dev, int64_t ldc,
                          tsmm_stream_t stream, int reps, tsmm_plan_t *out) {
    if (!out || reps < 1 || reps > 1000) return TSMM_ERR_INVALID_ARG;
    tsmm_plan_t base = nullptr;
    tsmm_status st = create_plan(m, n, k, dtype, 0, &base);
    if (st != TSMM_OK) return st;
    if (base->regime != 1 || m == 0 || n == 0 || k == 0 || base->kp / kTallBKS <= 1) {
        *out = base;  // nothing to tune: one split is the only choice
        return TSMM_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t kstages = base->kp / kTallBKS;
    const int sms = base->num_sms;
    // candidate split counts: the model's choice for 1..4 resident blocks per
    // SM, its halves and doubles, no split, and counts that fill whole waves
    std::set<int64_t> cand;
    for (int per_sm = 1; per_sm <= 4; ++per_sm)
        cand.insert(choose_splits(base->slabs, kstages, sms, kstages, per_sm));
    const int64_t h = base->splits;
    for (int64_t c : {h, h / 2, 2 * h, (int64_t)1}) cand.insert(c);
    for (int waves = 1; waves <= 4; ++waves) {
        const int64_t want = (int64_t)waves * tall_resident_blocks(dtype == TSMM_F64, base->np) * sms;
        cand.insert(std::max<int64_t>(1, want / std::max<int64_t>(1, base->slabs)));
    }
    std::vector<int64_t> cands;
    for (int64_t c : cand)
        if (c >= 1 && c <= kstages && c <= 65535) cands.push_back(c);

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        tsmm_plan_destroy(base);
        return TSMM_ERR_CUDA;
    }
    tsmm_plan_t best = nullptr;
    float best_ms = -1.f;
    st = TSMM_OK;
    for (int64_t c : cands) {
        tsmm_plan_t p = nullptr;
        if (c == base->splits) {
            p = base;
        } else if (create_plan(m, n, k, dtype, (int)c, &p) != TSMM_OK) {
            continue;  // e.g. the workspace of this candidate does not fit
        }
        // warm-up, then the timed repetitions (beta = 0: C is overwritten)
        st = tsmm_execute(p, 1.0, A_dev, lda, pb, 0.0, C_dev, ldc, stream);
        float ms = -1.f;
        if (st == TSMM_OK) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && st == TSMM_OK; ++r)
                st = tsmm_execute(p, 1.0, A_dev, lda, pb, 0.0, C_dev, ldc, stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                st = TSMM_ERR_CUDA;
        }
        if (st == TSMM_OK) st = tsmm_plan_check(p);
        if (st != TSMM_OK) {
            if (p != base) tsmm_plan_destroy(p);
            break;
        }
        if (best_ms < 0.f || ms < best_ms) {
            if (best && best != base) tsmm_plan_destroy(best);
            best = p;
            best_ms = ms;
        } else if (p != base) {
            tsmm_plan_destroy(p);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TSMM_OK || !best) {
        if (best && best != base) tsmm_plan_destroy(best);
        tsmm_plan_destroy(base);
        return st != TSMM_OK ? st : TSMM_ERR_CUDA;
    }
    if (best != base) tsmm_plan_destroy(base);
    plan_cache_store(dtype, m, n, k, sms, best->splits);
    *out = best;
    return TSMM_OK;
}

}  // extern "C"
