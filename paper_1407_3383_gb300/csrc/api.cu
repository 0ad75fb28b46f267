// C-ABI entry points: argument checks, then dispatch to the word policy.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gbntt.h"
#include "kernels.h"
#include "plan.h"

using namespace gbntt;

static cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

static bool aligned(const void* ptr, size_t a) { return (reinterpret_cast<uintptr_t>(ptr) % a) == 0; }

// Optional range check (NTT_FLAG_CHECK): copies the operand to the host and
// verifies every word is a residue < p.  Synchronous; meant for debugging.
static int check_range(const ntt_plan* P, const void* d, size_t words, cudaStream_t st) {
    if (!(P->flags & NTT_FLAG_CHECK) || words == 0) return NTT_OK;
    std::vector<uint64_t> h(words);
    if (P->flags & NTT_FLAG_FP64) {                      // doubles: integers in [0, p)
        std::vector<double> hd(words);
        if (cudaMemcpyAsync(hd.data(), d, words * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return NTT_ERR_CUDA;
        for (size_t i = 0; i < words; ++i)
            if (!(hd[i] >= 0.0 && hd[i] < static_cast<double>(P->p)) || hd[i] != static_cast<double>(static_cast<uint64_t>(hd[i]))) {
                gbntt_set_error("input word " + std::to_string(i) + " is not an integer in [0, p)");
                return NTT_ERR_RANGE;
            }
        return NTT_OK;
    }
    if (P->word_bytes == 4) {
        std::vector<uint32_t> h32(words);
        if (cudaMemcpyAsync(h32.data(), d, words * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return NTT_ERR_CUDA;
        for (size_t i = 0; i < words; ++i) h[i] = h32[i];
    } else {
        if (cudaMemcpyAsync(h.data(), d, words * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return NTT_ERR_CUDA;
    }
    for (size_t i = 0; i < words; ++i)
        if (h[i] >= P->p) {
            gbntt_set_error("input word " + std::to_string(i) + " is not below p");
            return NTT_ERR_RANGE;
        }
    return NTT_OK;
}

static int ntt_dir(const ntt_plan* P, void* d_data, size_t batch, void* stream, bool fwd) {
    if (!P || (!d_data && batch)) return NTT_ERR_ARG;
    if (batch == 0) return NTT_OK;
    if (!aligned(d_data, P->word_bytes)) return NTT_ERR_ARG;
    const cudaStream_t st = as_stream(stream);
    const size_t words = batch << P->log2n;
    if (fwd) {
        int rc = check_range(P, d_data, words, st);
        if (rc != NTT_OK) return rc;
    }
    if (P->flags & NTT_FLAG_FP64)
        return launch_ntt<Fma50>(P, P->dpf, static_cast<double*>(d_data), static_cast<long long>(batch), fwd,
                                 P->inv_scalef, st);
    if (P->word_bytes == 4)
        return launch_ntt<Mont32>(P, P->dp32, static_cast<uint32_t*>(d_data),
                                  static_cast<long long>(batch), fwd, P->inv_scale32, st);
    return launch_ntt<Shoup64L>(P, P->dp64, static_cast<uint64_t*>(d_data),
                               static_cast<long long>(batch), fwd, P->inv_scale64, st);
}

extern "C" int ntt_forward(const ntt_plan* plan, void* d_data, size_t batch, void* stream) {
    return ntt_dir(plan, d_data, batch, stream, true);
}

extern "C" int ntt_inverse(const ntt_plan* plan, void* d_data, size_t batch, void* stream) {
    return ntt_dir(plan, d_data, batch, stream, false);
}

extern "C" size_t polymul_workspace_size(const ntt_plan* plan, size_t batch, unsigned schedule) {
    if (!plan || schedule > NTT_SCHED_PLAIN) return 0;
    return polymul_ws_bytes(plan, batch, schedule);
}

extern "C" int polymul_mod_p_batch(const ntt_plan* plan, const void* d_a, size_t na, const void* d_b,
                                   size_t nb, size_t batch, void* d_c, unsigned schedule, void* d_ws,
                                   size_t ws_bytes, void* stream) {
    const ntt_plan* P = plan;
    if (!P || schedule > NTT_SCHED_PLAIN) return NTT_ERR_ARG;
    if (batch == 0) return NTT_OK;
    if (!d_a || !d_b || !d_c || na == 0 || nb == 0) {
        gbntt_set_error("polymul: null operand or empty polynomial");
        return NTT_ERR_ARG;
    }
    if (na + nb - 1 > (size_t(1) << P->log2n)) {
        gbntt_set_error("polymul: na + nb - 1 exceeds the plan's n");
        return NTT_ERR_SIZE;
    }
    if (schedule == NTT_SCHED_PLAIN && !(P->flags & NTT_FLAG_PLAIN)) {
        gbntt_set_error("plain schedule needs a plan created with NTT_FLAG_PLAIN");
        return NTT_ERR_ARG;
    }
    const size_t need = polymul_ws_bytes(P, batch, schedule);
    if (need && (!d_ws || ws_bytes < need || !aligned(d_ws, 256))) {
        gbntt_set_error("polymul: workspace of " + std::to_string(need) +
                        " bytes (256-byte aligned) required");
        return NTT_ERR_WORKSPACE;
    }
    const unsigned wb = P->word_bytes;
    if (!aligned(d_a, wb) || !aligned(d_b, wb) || !aligned(d_c, wb)) return NTT_ERR_ARG;
    const cudaStream_t st = as_stream(stream);
    int rc = check_range(P, d_a, na * batch, st);
    if (rc == NTT_OK) rc = check_range(P, d_b, nb * batch, st);
    if (rc != NTT_OK) return rc;
    const long long lna = static_cast<long long>(na), lnb = static_cast<long long>(nb);
    const long long lb = static_cast<long long>(batch);
    if (P->flags & NTT_FLAG_FP64)                        // fused only (planning refuses PLAIN)
        return launch_polymul_fused<Fma50>(P, P->dpf, static_cast<const double*>(d_a), lna,
                                           static_cast<const double*>(d_b), lnb, lb, static_cast<double*>(d_c),
                                           static_cast<double*>(d_ws), P->inv_scalef, st);
    if (wb == 4) {
        auto a = static_cast<const uint32_t*>(d_a);
        auto b = static_cast<const uint32_t*>(d_b);
        auto c = static_cast<uint32_t*>(d_c);
        auto w = static_cast<uint32_t*>(d_ws);
        return schedule == NTT_SCHED_FUSED
                   ? launch_polymul_fused<Mont32>(P, P->dp32, a, lna, b, lnb, lb, c, w, P->pm_scale32, st)
                   : launch_polymul_plain<Mont32>(P, P->dp32, a, lna, b, lnb, lb, c, w, P->pm_scale32, st);
    }
    auto a = static_cast<const uint64_t*>(d_a);
    auto b = static_cast<const uint64_t*>(d_b);
    auto c = static_cast<uint64_t*>(d_c);
    auto w = static_cast<uint64_t*>(d_ws);
    return schedule == NTT_SCHED_FUSED
               ? launch_polymul_fused<Shoup64L>(P, P->dp64, a, lna, b, lnb, lb, c, w, P->pm_scale64, st)
               : launch_polymul_plain<Shoup64L>(P, P->dp64, a, lna, b, lnb, lb, c, w, P->pm_scale64, st);
}

extern "C" int polymul_mod_p(const ntt_plan* plan, const void* d_a, size_t na, const void* d_b,
                             size_t nb, void* d_c, void* d_ws, size_t ws_bytes, void* stream) {
    return polymul_mod_p_batch(plan, d_a, na, d_b, nb, 1, d_c, NTT_SCHED_FUSED, d_ws, ws_bytes, stream);
}

extern "C" int ntt_modmul_vec(uint64_t p, unsigned kind, unsigned word_bytes, const uint64_t* d_x,
                              const uint64_t* d_y, const uint64_t* d_yc, uint64_t* d_z, size_t n,
                              void* stream) {
    return launch_modmul_vec(p, kind, word_bytes, d_x, d_y, d_yc, d_z, n, as_stream(stream));
}

extern "C" int ntt_modmul_rate(uint64_t p, unsigned kind, unsigned word_bytes, int iters, double* products_per_s) {
    return modmul_rate(p, kind, word_bytes, iters, products_per_s);
}

extern "C" size_t polymat_workspace_size(const ntt_plan* plan, unsigned n) {
    if (!plan || n == 0) return 0;
    return 3ull * n * n * (size_t(1) << plan->log2n) * plan->word_bytes;
}

extern "C" int polymat_mul(const ntt_plan* plan, const void* d_A, const void* d_B, unsigned n, size_t d,
                           void* d_C, void* d_ws, size_t ws_bytes, void* stream) {
    if (!plan || !d_A || !d_B || !d_C || n == 0 || n > 1024 || d == 0) return NTT_ERR_ARG;
    if (plan->flags & NTT_FLAG_FP64) {
        gbntt_set_error("polymat_mul: no FP64 form");
        return NTT_ERR_UNSUPPORTED;
    }
    if (2 * d - 1 > (size_t(1) << plan->log2n)) {
        gbntt_set_error("polymat_mul: 2d - 1 exceeds the plan's n");
        return NTT_ERR_SIZE;
    }
    const size_t need = polymat_workspace_size(plan, n);
    if (!d_ws || ws_bytes < need || !aligned(d_ws, 256)) {
        gbntt_set_error("polymat_mul: workspace of " + std::to_string(need) + " bytes required");
        return NTT_ERR_WORKSPACE;
    }
    const cudaStream_t st = as_stream(stream);
    const long long ld = static_cast<long long>(d);
    if (plan->word_bytes == 4)
        return launch_polymat<Mont32>(plan, plan->dp32, static_cast<const uint32_t*>(d_A),
                                      static_cast<const uint32_t*>(d_B), static_cast<int>(n), ld,
                                      static_cast<uint32_t*>(d_C), static_cast<uint32_t*>(d_ws),
                                      plan->inv_scale32, plan->r32, st);
    return launch_polymat<Shoup64L>(plan, plan->dp64, static_cast<const uint64_t*>(d_A),
                                    static_cast<const uint64_t*>(d_B), static_cast<int>(n), ld,
                                    static_cast<uint64_t*>(d_C), static_cast<uint64_t*>(d_ws),
                                    plan->inv_scale64, plan->r64, st);
}
