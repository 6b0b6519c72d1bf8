// Kernel instantiations for PrecF32.
#include "lbm_launch_impl.cuh"

namespace lbm {
template cudaError_t launch_adr<PrecF32>(int, int, const AdrArgs &,
                                            cudaStream_t, const AdrOverlap *);
template cudaError_t launch_adr_flux<PrecF32>(int, const void *, const RefT *,
                                                 const uint32_t *, long long,
                                                 int, int, int, double *,
                                                 cudaStream_t);
template cudaError_t launch_flow<PrecF32>(int, const FlowArgs &, dim3,
                                             cudaStream_t);
template cudaError_t launch_adjoint<PrecF32>(int, int, const AdjArgs &,
                                                cudaStream_t);
template cudaError_t launch_adjoint_grad<PrecF32>(
    int, const AdjArgs &, const long long *, long long, const void *, double *,
    double *, const int32_t *, double *, double, double, cudaStream_t);
}  // namespace lbm
