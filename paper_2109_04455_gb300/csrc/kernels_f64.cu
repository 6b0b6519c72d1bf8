// Kernel instantiations for PrecF64.
#include "lbm_launch_impl.cuh"

namespace lbm {
template cudaError_t launch_adr<PrecF64>(int, int, const AdrArgs &,
                                            cudaStream_t, const AdrOverlap *);
template cudaError_t launch_adr_flux<PrecF64>(int, const void *, const RefT *,
                                                 const uint32_t *, long long,
                                                 int, int, int, double *,
                                                 cudaStream_t);
template cudaError_t launch_flow<PrecF64>(int, const FlowArgs &, dim3,
                                             cudaStream_t);
template cudaError_t launch_adjoint<PrecF64>(int, int, const AdjArgs &,
                                                cudaStream_t);
template cudaError_t launch_adjoint_grad<PrecF64>(
    int, const AdjArgs &, const long long *, long long, const void *, double *,
    double *, const int32_t *, double *, double, double, cudaStream_t);

cudaError_t launch_eq_table(const double *u, long long plane, double *etab,
                            cudaStream_t st) {
  const long long blocks = (plane + 255) / 256;
  eq_table_kernel<double><<<static_cast<unsigned>(blocks), 256, 0, st>>>(
      u, plane, etab);
  return cudaGetLastError();
}
}  // namespace lbm
