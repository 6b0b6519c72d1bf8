// Definitions of the kernel launchers declared in lbm_kernels.cuh.  Each
// precision's translation unit includes this file and instantiates them, so
// the kernel variants compile in parallel.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

template <class P>
cudaError_t launch_adr(int ns, int mode, const AdrArgs &a, dim3 grid,
                       cudaStream_t st) {
  const dim3 block(kBlockX);
#define LBM_ADR_CASE(NS, MODE)                              \
  if (ns == NS && mode == MODE) {                           \
    adr_kernel<P, NS, MODE><<<grid, block, 0, st>>>(a);     \
    return cudaGetLastError();                              \
  }
  LBM_ADR_CASE(1, kAdrStep)
  LBM_ADR_CASE(1, kAdrCheck)
  LBM_ADR_CASE(1, kAdrInit)
  LBM_ADR_CASE(2, kAdrStep)
  LBM_ADR_CASE(2, kAdrCheck)
  LBM_ADR_CASE(2, kAdrInit)
  LBM_ADR_CASE(3, kAdrStep)
  LBM_ADR_CASE(3, kAdrCheck)
  LBM_ADR_CASE(3, kAdrInit)
#undef LBM_ADR_CASE
  return cudaErrorInvalidValue;
}

template <class P>
cudaError_t launch_adr_flux(int ns, const void *g, const uint32_t *links,
                            long long plane, int nx_pad, int ny, int xp,
                            const double *cref, double *out, cudaStream_t st) {
  const dim3 block(kReduceThreads);
  if (ns == 1)
    adr_flux_kernel<P, 1><<<1, block, 0, st>>>(g, links, plane, nx_pad, ny, xp,
                                               cref[0], cref[1], cref[2], out);
  else if (ns == 2)
    adr_flux_kernel<P, 2><<<1, block, 0, st>>>(g, links, plane, nx_pad, ny, xp,
                                               cref[0], cref[1], cref[2], out);
  else if (ns == 3)
    adr_flux_kernel<P, 3><<<1, block, 0, st>>>(g, links, plane, nx_pad, ny, xp,
                                               cref[0], cref[1], cref[2], out);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_flow(int mode, const FlowArgs &a, dim3 grid,
                        cudaStream_t st) {
  const dim3 block(kBlockX);
  switch (mode) {
    case kFlowStep: flow_kernel<P, kFlowStep><<<grid, block, 0, st>>>(a); break;
    case kFlowU: flow_kernel<P, kFlowU><<<grid, block, 0, st>>>(a); break;
    case kFlowCheck: flow_kernel<P, kFlowCheck><<<grid, block, 0, st>>>(a); break;
    case kFlowInit: flow_kernel<P, kFlowInit><<<grid, block, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
