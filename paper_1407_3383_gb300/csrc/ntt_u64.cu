// Transform and product kernels instantiated for 64-bit words (Shoup64L, lazy residues).
#include "ntt_kernels.cuh"

namespace gbntt {

template int launch_polymul_fused<Shoup64L>(const ntt_plan*, const DevPlan<Shoup64L>&, const uint64_t*,
                                           long long, const uint64_t*, long long, long long,
                                           uint64_t*, uint64_t*, Tw64, cudaStream_t);
template int launch_polymul_plain<Shoup64L>(const ntt_plan*, const DevPlan<Shoup64L>&, const uint64_t*,
                                           long long, const uint64_t*, long long, long long,
                                           uint64_t*, uint64_t*, Tw64, cudaStream_t);
template int launch_batch_small<Shoup64L>(const DevPlan<Shoup64L>*, const TftConsts<Shoup64L>*, const BatchDesc*, const void*, unsigned,
                                         unsigned*, const uint64_t*, const uint64_t*, uint64_t*, size_t, int,
                                         cudaStream_t);
template int launch_batch_bucket<Shoup64L>(const ntt_plan*, const DevPlan<Shoup64L>&, const uint64_t*,
                                          const uint64_t*, uint64_t*, const BatchDesc*, long long,
                                          uint64_t*, Tw64, cudaStream_t, long long, bool);
template int batch_small_occupancy<Shoup64L>(size_t);
template int launch_polymat<Shoup64L>(const ntt_plan*, const DevPlan<Shoup64L>&, const uint64_t*, const uint64_t*,
                                    int, long long, uint64_t*, uint64_t*, Tw64, Tw64, cudaStream_t);
template int launch_ntt<Shoup64L>(const ntt_plan*, const DevPlan<Shoup64L>&, uint64_t*, long long,
                                 bool, Tw64, cudaStream_t);

}  // namespace gbntt
