// Transform and product kernels instantiated for 32-bit words (Mont32).
#include "ntt_kernels.cuh"

namespace gbntt {

template int launch_polymul_fused<Mont32>(const ntt_plan*, const DevPlan<Mont32>&, const uint32_t*,
                                          long long, const uint32_t*, long long, long long, uint32_t*,
                                          uint32_t*, Tw32, cudaStream_t);
template int launch_polymul_plain<Mont32>(const ntt_plan*, const DevPlan<Mont32>&, const uint32_t*,
                                          long long, const uint32_t*, long long, long long, uint32_t*,
                                          uint32_t*, Tw32, cudaStream_t);
template int launch_batch_small<Mont32>(const DevPlan<Mont32>*, const TftConsts<Mont32>*, const BatchDesc*, const void*, unsigned,
                                         unsigned*, const uint32_t*, const uint32_t*, uint32_t*, size_t, int,
                                         cudaStream_t);
template int launch_batch_bucket<Mont32>(const ntt_plan*, const DevPlan<Mont32>&, const uint32_t*,
                                          const uint32_t*, uint32_t*, const BatchDesc*, long long,
                                          uint32_t*, Tw32, cudaStream_t, long long, bool);
template int batch_small_occupancy<Mont32>(size_t);
template int launch_polymat<Mont32>(const ntt_plan*, const DevPlan<Mont32>&, const uint32_t*, const uint32_t*,
                                    int, long long, uint32_t*, uint32_t*, Tw32, Tw32, cudaStream_t);
template int launch_ntt<Mont32>(const ntt_plan*, const DevPlan<Mont32>&, uint32_t*, long long, bool,
                                Tw32, cudaStream_t);

size_t polymul_ws_bytes(const ntt_plan* plan, size_t batch, unsigned schedule) {
    const size_t N = size_t(1) << plan->log2n;
    if (schedule == NTT_SCHED_FUSED && static_cast<int>(plan->log2n) <= plan->tile_max_log) return 0;
    return 2 * N * plan->word_bytes * batch;
}

}  // namespace gbntt
