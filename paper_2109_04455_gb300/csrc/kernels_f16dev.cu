// Kernel instantiations for PrecF16Dev.
#include "lbm_launch_impl.cuh"

namespace lbm {
template cudaError_t launch_adr<PrecF16Dev>(int, int, const AdrArgs &,
                                            cudaStream_t, const AdrOverlap *);
template cudaError_t launch_adr_flux<PrecF16Dev>(int, const void *, const RefT *,
                                                 const uint32_t *, long long,
                                                 int, int, int, double *,
                                                 cudaStream_t);
}  // namespace lbm
