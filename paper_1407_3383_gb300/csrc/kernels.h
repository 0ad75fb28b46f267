// Launchers shared between the C-ABI layer and the kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "engine.cuh"

struct ntt_plan;

namespace gbntt {

template <class Ar>
int launch_polymul_fused(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* a,
                         long long na, const typename Ar::word* b, long long nb, long long batch,
                         typename Ar::word* c, typename Ar::word* ws, typename Ar::tw scale,
                         cudaStream_t st);

template <class Ar>
int launch_polymul_plain(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* a,
                         long long na, const typename Ar::word* b, long long nb, long long batch,
                         typename Ar::word* c, typename Ar::word* ws, typename Ar::tw scale,
                         cudaStream_t st);

template <class Ar>
int launch_ntt(const ntt_plan* plan, const DevPlan<Ar>& dp, typename Ar::word* data, long long batch,
               bool fwd, typename Ar::tw scale, cudaStream_t st);

size_t polymul_ws_bytes(const ntt_plan* plan, size_t batch, unsigned schedule);

// Launch profiling hooks (no-ops unless ntt_profile_begin() is active).
void prof_begin_call(cudaStream_t st);
void prof_mark(cudaStream_t st, const char* name);

int launch_modmul_vec(uint64_t p, unsigned kind, unsigned word_bytes, const uint64_t* x,
                      const uint64_t* y, const uint64_t* yc, uint64_t* z, size_t n, cudaStream_t st);

}  // namespace gbntt
