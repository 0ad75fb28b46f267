// Launchers shared between the C-ABI layer and the kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "engine.cuh"
#include "tft.cuh"

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
int launch_batch_small(const DevPlan<Ar>* d_plans, const TftConsts<Ar>* d_tfts, const BatchDesc* d_desc,
                       const void* d_items, unsigned nitems, unsigned* d_ticket, const typename Ar::word* a,
                       const typename Ar::word* b, typename Ar::word* c, size_t smem, int grid,
                       cudaStream_t st);

template <class Ar>
int batch_small_occupancy(size_t smem);

template <class Ar>
int launch_batch_bucket(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* a,
                        const typename Ar::word* b, typename Ar::word* c, const BatchDesc* d_desc,
                        long long count, typename Ar::word* ws, typename Ar::tw scale,
                        cudaStream_t st, long long subs, bool tft);

template <class Ar>
int launch_ntt(const ntt_plan* plan, const DevPlan<Ar>& dp, typename Ar::word* data, long long batch,
               bool fwd, typename Ar::tw scale, cudaStream_t st);

size_t polymul_ws_bytes(const ntt_plan* plan, size_t batch, unsigned schedule);

template <class Ar>
int launch_polymat(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* A,
                   const typename Ar::word* B, int n, long long d, typename Ar::word* C,
                   typename Ar::word* ws, typename Ar::tw inv_scale, typename Ar::tw r, cudaStream_t st);

// Launch shape of the fused product kernels for one (word size, log2 n):
// lppc  log2 of products per block (one-block sizes),
// logw  log2 of columns per block in the column passes,
// lrpc  log2 of rows per block in the row pass.
struct LaunchCfg {
    int lppc, logw, lrpc;
};
LaunchCfg default_launch_cfg(unsigned word_bytes, int log2n, int tile_max_log);
LaunchCfg generic_global_cfg(unsigned word_bytes, int log2n);
LaunchCfg launch_cfg(unsigned word_bytes, int log2n, int tile_max_log);   // tuned or default
void set_launch_cfg(unsigned word_bytes, int log2n, LaunchCfg cfg);
void clear_launch_cfg(unsigned word_bytes, int log2n);
size_t col_smem_bytes(unsigned word_bytes, int k2, int logw);
size_t tile_smem_bytes(unsigned word_bytes, int logL, int lognvec);

// Launch profiling hooks (no-ops unless ntt_profile_begin() is active).
void prof_begin_call(cudaStream_t st);
void prof_mark(cudaStream_t st, const char* name);

int modmul_rate(uint64_t p, unsigned kind, unsigned word_bytes, int iters, double* per_s);

int launch_modmul_vec(uint64_t p, unsigned kind, unsigned word_bytes, const uint64_t* x,
                      const uint64_t* y, const uint64_t* yc, uint64_t* z, size_t n, cudaStream_t st);

}  // namespace gbntt
