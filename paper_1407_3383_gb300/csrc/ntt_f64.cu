// Transform and product kernels instantiated for residues held as doubles
// (Fma50: Function 16 products, p < 2^50) -- plans made with NTT_FLAG_FP64.
#include "ntt_kernels.cuh"

namespace gbntt {

template int launch_polymul_fused<Fma50>(const ntt_plan*, const DevPlan<Fma50>&, const double*, long long,
                                        const double*, long long, long long, double*, double*, TwF,
                                        cudaStream_t);
template int launch_ntt<Fma50>(const ntt_plan*, const DevPlan<Fma50>&, double*, long long, bool, TwF,
                              cudaStream_t);

}  // namespace gbntt
