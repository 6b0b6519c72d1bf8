// Kernel instantiations for PrecF16Dev.
#include "lbm_launch_impl.cuh"

namespace lbm {
// LBM_ADR_QUAD_F16 = 1: plain FP16 steps run the four-nodes-per-thread
// kernel (adr_bulk_quad_kernel; check steps keep the two-node kernel, the
// stored bits are the same).  The choice is made here, by specialising the
// bulk launcher for this precision, so that the other precisions' units
// never see it.
#ifndef LBM_ADR_QUAD_F16
#define LBM_ADR_QUAD_F16 1
#endif
#if LBM_ADR_QUAD_F16 && LBM_ADR_PAIR_F16
#define LBM_QUAD_LAUNCH(NS)                                                   \
  template <>                                                                 \
  void launch_bulk<PrecF16Dev, NS, kAdrStep>(const AdrArgs &a, dim3 bg,       \
                                             cudaStream_t st) {               \
    adr_bulk_quad_kernel<NS><<<bg, dim3(kQuadThreads), 0, st>>>(a);           \
  }
LBM_QUAD_LAUNCH(1)
LBM_QUAD_LAUNCH(2)
LBM_QUAD_LAUNCH(3)
#undef LBM_QUAD_LAUNCH
#endif

template cudaError_t launch_adr<PrecF16Dev>(int, int, const AdrArgs &,
                                            cudaStream_t, const AdrOverlap *);
template cudaError_t launch_adr_flux<PrecF16Dev>(int, const void *, const RefT *,
                                                 const uint32_t *, long long,
                                                 int, int, int, double *,
                                                 cudaStream_t);
}  // namespace lbm
