// Launch-shape table and autotuner for the fused product kernels.
//
// The paper picks its implementation variants (loop unrolling, vector
// sizes, thresholds) at compile time through C++ templates (Section 4).
// Here the variants that matter on the GPU -- products per block for the
// one-block sizes, columns per block and rows per block for the two global
// passes -- are runtime launch parameters: a process-wide table keyed by
// (word size, log2 n) holds the chosen shape, defaulting to a heuristic,
// and ntt_autotune() times the candidates on the device and keeps the
// fastest.  The table can be exported to and imported from text.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/gbntt.h"
#include "kernels.h"
#include "ntt_kernels.cuh"
#include "plan.h"

namespace gbntt {

namespace {
std::mutex g_cfg_mu;
std::map<std::pair<unsigned, int>, LaunchCfg> g_cfg;
constexpr size_t kMaxSmem = 200 * 1024;
}  // namespace

size_t col_smem_bytes(unsigned word_bytes, int k2, int logw) {
    return static_cast<size_t>(slab_words(slab_layout(k2, logw))) * word_bytes;
}

size_t tile_smem_bytes(unsigned word_bytes, int logL, int lognvec) {
    return static_cast<size_t>(layout_words(tile_layout(logL, lognvec))) * word_bytes;
}

LaunchCfg default_launch_cfg(unsigned word_bytes, int log2n, int tile_max_log) {
    LaunchCfg c{0, 0, 0};
    if (log2n <= tile_max_log) {
        c.lppc = small_lppc(log2n);
        return c;
    }
    if (log2n >= 2 * kDLog && log2n <= 3 * kDLog) return c;   // logw = 0: the direct kernels
    return generic_global_cfg(word_bytes, log2n);
}

// Columns and rows per block of the generic global passes.
LaunchCfg generic_global_cfg(unsigned word_bytes, int log2n) {
    LaunchCfg c{0, 0, 0};
    const int k2 = log2n / 2, k1 = log2n - k2;
    int logw = (word_bytes == 4) ? 5 : 4;             // 128-byte row segments
    const int min_logw = (word_bytes == 4) ? 3 : 2;   // at least 32-byte sectors
    while (logw > min_logw && col_smem_bytes(word_bytes, k2, logw) > 100 * 1024) --logw;
    c.logw = logw;
    c.lrpc = (k1 <= kMaxLineLog) ? 4 : 0;
    return c;
}

// A shape is usable when its blocks fit in shared memory and its grids are
// not empty.
static bool cfg_valid(unsigned wb, int k, int tile_max_log, const LaunchCfg& c) {
    const size_t cap = 227 * 1024;
    if (k <= tile_max_log) return c.lppc >= 0 && c.lppc <= 6 && tile_smem_bytes(wb, k, c.lppc + 1) <= cap;
    const int k2 = k / 2, k1 = k - k2;
    if (c.logw == 0) return k >= 2 * kDLog && k <= 3 * kDLog;
    return c.logw >= 1 && c.logw <= k1 && col_smem_bytes(wb, k2, c.logw) <= cap && c.lrpc >= 0 &&
           c.lrpc <= k2 && tile_smem_bytes(wb, k1, c.lrpc + 1) <= cap;
}

LaunchCfg launch_cfg(unsigned word_bytes, int log2n, int tile_max_log) {
    {
        std::lock_guard<std::mutex> lock(g_cfg_mu);
        auto it = g_cfg.find({word_bytes, log2n});
        if (it != g_cfg.end() && cfg_valid(word_bytes, log2n, tile_max_log, it->second)) return it->second;
    }
    return default_launch_cfg(word_bytes, log2n, tile_max_log);
}

void set_launch_cfg(unsigned word_bytes, int log2n, LaunchCfg cfg) {
    std::lock_guard<std::mutex> lock(g_cfg_mu);
    g_cfg[{word_bytes, log2n}] = cfg;
}

void clear_launch_cfg(unsigned word_bytes, int log2n) {
    std::lock_guard<std::mutex> lock(g_cfg_mu);
    g_cfg.erase({word_bytes, log2n});
}

}  // namespace gbntt

using namespace gbntt;

namespace {

// Device time of one polymul_mod_p_batch call (median of `reps`).
float time_product(const ntt_plan* P, const void* a, const void* b, void* c, void* ws, size_t wsb,
                   size_t batch, cudaStream_t st, int reps) {
    const size_t n = size_t(1) << P->log2n;
    const size_t na = n / 2, nb = n / 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    polymul_mod_p_batch(P, a, na, b, nb, batch, c, NTT_SCHED_FUSED, ws, wsb, st);   // warm-up
    std::vector<float> t;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, st);
        if (polymul_mod_p_batch(P, a, na, b, nb, batch, c, NTT_SCHED_FUSED, ws, wsb, st) != NTT_OK) {
            t.push_back(1e30f);
            continue;
        }
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

extern "C" int ntt_autotune(const ntt_plan* plan, size_t batch, void* stream, float* best_ms) {
    if (!plan || batch == 0) return NTT_ERR_ARG;
    if (plan->flags & NTT_FLAG_FP64) {        // the shape table is keyed by word size; FP64 plans share it
        gbntt_set_error("ntt_autotune: tune the integer plan of the same word size instead");
        return NTT_ERR_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned wb = plan->word_bytes;
    const int k = static_cast<int>(plan->log2n);
    const size_t n = size_t(1) << k;
    const size_t ws_bytes = std::max<size_t>(256, 2 * n * wb * batch);
    void *a = nullptr, *b = nullptr, *c = nullptr, *ws = nullptr;
    if (cudaMalloc(&a, n / 2 * wb * batch) != cudaSuccess || cudaMalloc(&b, n / 2 * wb * batch) != cudaSuccess ||
        cudaMalloc(&c, n * wb * batch) != cudaSuccess || cudaMalloc(&ws, ws_bytes) != cudaSuccess) {
        cudaFree(a);
        cudaFree(b);
        cudaFree(c);
        cudaFree(ws);
        cudaGetLastError();
        return NTT_ERR_OOM;
    }
    cudaMemsetAsync(a, 0, n / 2 * wb * batch, st);
    cudaMemsetAsync(b, 0, n / 2 * wb * batch, st);
    LaunchCfg best = default_launch_cfg(wb, k, plan->tile_max_log);
    auto try_cfg = [&](LaunchCfg cfg) {
        set_launch_cfg(wb, k, cfg);
        return time_product(plan, a, b, c, ws, ws_bytes, batch, st, 5);
    };
    float best_t = try_cfg(best);
    if (k <= plan->tile_max_log) {
        for (int lppc = 0; lppc <= 5; ++lppc) {
            if (tile_smem_bytes(wb, k, lppc + 1) > kMaxSmem) break;
            LaunchCfg cfg = best;
            cfg.lppc = lppc;
            const float t = try_cfg(cfg);
            if (t < best_t) best_t = t, best = cfg;
        }
    } else {
        // generic shapes: columns per block, then rows per block, from the
        // generic default; the direct kernels (logw = 0, n = 2^16 only)
        // compete with the best of them
        const int k2 = k / 2, k1 = k - k2;
        LaunchCfg g = best;
        float g_t = best_t;
        if (best.logw == 0) {
            g = generic_global_cfg(wb, k);
            g_t = try_cfg(g);
        }
        for (int logw = 1; logw <= 6 && (1 << logw) <= (1 << k1); ++logw) {
            if (col_smem_bytes(wb, k2, logw) > kMaxSmem) break;
            if ((1 << logw) * wb < 16) continue;
            LaunchCfg cfg = g;
            cfg.logw = logw;
            const float t = try_cfg(cfg);
            if (t < g_t) g_t = t, g = cfg;
        }
        for (int lrpc = 0; lrpc <= 6 && lrpc <= k2; ++lrpc) {
            if (tile_smem_bytes(wb, k1, lrpc + 1) > kMaxSmem) break;
            LaunchCfg cfg = g;
            cfg.lrpc = lrpc;
            const float t = try_cfg(cfg);
            if (t < g_t) g_t = t, g = cfg;
        }
        if (g_t < best_t) best_t = g_t, best = g;
        // The direct kernels with TMA input tiles (lppc = 1 at n = 2^16) are
        // not a candidate: a block whose bounded waits both expire returns
        // with its bulk copy possibly still writing the block's shared
        // memory, and no bounded exit avoids that.  They time the same as
        // the per-thread loads and stay available through ntt_tune_import.
    }
    set_launch_cfg(wb, k, best);
    if (best_ms) *best_ms = best_t;
    cudaFree(a);
    cudaFree(b);
    cudaFree(c);
    cudaFree(ws);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gbntt_set_error(std::string("ntt_autotune: ") + cudaGetErrorString(e));
        return NTT_ERR_CUDA;
    }
    return NTT_OK;
}

extern "C" int ntt_tune_get(unsigned word_bytes, unsigned log2n, int* lppc, int* logw, int* lrpc) {
    if (!lppc || !logw || !lrpc || (word_bytes != 4 && word_bytes != 8)) return NTT_ERR_ARG;
    const LaunchCfg c = launch_cfg(word_bytes, static_cast<int>(log2n), word_bytes == 4 ? kTileMaxLog32 : kTileMaxLog64);
    *lppc = c.lppc;
    *logw = c.logw;
    *lrpc = c.lrpc;
    return NTT_OK;
}

extern "C" int ntt_tune_reset(void) {
    std::lock_guard<std::mutex> lock(g_cfg_mu);
    g_cfg.clear();
    return NTT_OK;
}

extern "C" int ntt_tune_export(char* buf, size_t cap, size_t* len) {
    std::ostringstream os;
    {
        std::lock_guard<std::mutex> lock(g_cfg_mu);
        for (const auto& kv : g_cfg)
            os << kv.first.first << ' ' << kv.first.second << ' ' << kv.second.lppc << ' '
               << kv.second.logw << ' ' << kv.second.lrpc << '\n';
    }
    const std::string s = os.str();
    if (len) *len = s.size();
    if (!buf) return NTT_OK;
    if (cap < s.size() + 1) return NTT_ERR_SIZE;
    std::copy(s.begin(), s.end(), buf);
    buf[s.size()] = '\0';
    return NTT_OK;
}

extern "C" int ntt_tune_import(const char* text) {
    if (!text) return NTT_ERR_ARG;
    std::istringstream is(text);
    unsigned wb;
    int k;
    LaunchCfg c;
    while (is >> wb >> k >> c.lppc >> c.logw >> c.lrpc) {
        if ((wb != 4 && wb != 8) || k < 1 || k > 24 || c.lppc < 0 || c.lppc > 6 || c.logw < 0 ||
            c.logw > 6 || c.lrpc < 0 || c.lrpc > 6)
            return NTT_ERR_ARG;
        set_launch_cfg(wb, k, c);
    }
    return NTT_OK;
}
