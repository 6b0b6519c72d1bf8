// Definitions of the kernel launchers declared in lbm_kernels.cuh.  Each
// precision's translation unit includes this file and instantiates them, so
// the kernel variants compile in parallel.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

template <class P, int NS, int MODE>
static void launch_bulk(const AdrArgs &a, dim3 bg, cudaStream_t st) {
  if constexpr (P::kDev && LBM_ADR_PAIR_F16)
    adr_bulk_pair_kernel<NS, MODE><<<bg, dim3(kPairThreads), 0, st>>>(a);
  else
    adr_bulk_kernel<P, NS, MODE><<<bg, dim3(kBlockX), 0, st>>>(a);
}

template <class P, int NS>
static cudaError_t launch_adr_ns(int mode, const AdrArgs &a, cudaStream_t st,
                                 const AdrOverlap *ov) {
  const dim3 block(kBlockX);
  if (mode == kAdrInit) {
    adr_node_kernel<P, NS, kAdrInit, false>
        <<<adr_node_grid(a.nx_pad, a.ny), block, 0, st>>>(a);
    return cudaGetLastError();
  }
  if (!LBM_ADR_SPLIT) {
    if (mode == kAdrStep)
      adr_node_kernel<P, NS, kAdrStep, false>
          <<<adr_node_grid(a.nx_pad, a.ny), block, 0, st>>>(a);
    else
      adr_node_kernel<P, NS, kAdrCheck, false>
          <<<adr_node_grid(a.nx_pad, a.ny), block, 0, st>>>(a);
    return cudaGetLastError();
  }
  const dim3 bg = adr_bulk_grid(a.nx_pad, a.ny);
  AdrArgs b = a;
  b.part_off = static_cast<long long>(bg.x) * bg.y;
  const unsigned lb = static_cast<unsigned>(adr_list_blocks(a.nbnd));
  // The boundary nodes run on a second stream next to the bulk kernel when
  // one is given: both read only the old populations and write disjoint
  // nodes, so the few boundary blocks hide in the bulk kernel's time.
  cudaStream_t sb = st;
  cudaError_t e = cudaSuccess;
  if (lb && ov && ov->aux) {
    e = cudaEventRecord(ov->fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ov->aux, ov->fork, 0);
    if (e != cudaSuccess) return e;
    sb = ov->aux;
  }
  if (mode == kAdrStep) {
    if (lb) adr_node_kernel<P, NS, kAdrStep, true><<<lb, block, 0, sb>>>(b);
    launch_bulk<P, NS, kAdrStep>(a, bg, st);
  } else {
    if (lb) adr_node_kernel<P, NS, kAdrCheck, true><<<lb, block, 0, sb>>>(b);
    launch_bulk<P, NS, kAdrCheck>(a, bg, st);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess && sb != st) {
    e = cudaEventRecord(ov->join, sb);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ov->join, 0);
  }
  return e;
}

template <class P>
cudaError_t launch_adr(int ns, int mode, const AdrArgs &a, cudaStream_t st,
                       const AdrOverlap *ov) {
  switch (ns) {
    case 1: return launch_adr_ns<P, 1>(mode, a, st, ov);
    case 2: return launch_adr_ns<P, 2>(mode, a, st, ov);
    case 3: return launch_adr_ns<P, 3>(mode, a, st, ov);
    default: return cudaErrorInvalidValue;
  }
}

template <class P>
cudaError_t launch_adr_flux(int ns, const void *g, const RefT *ref,
                            const uint32_t *links, long long plane, int nx_pad,
                            int ny, int xp, double *out, cudaStream_t st) {
  const dim3 block(kReduceThreads);
  if (ns == 1)
    adr_flux_kernel<P, 1><<<1, block, 0, st>>>(g, ref, links, plane, nx_pad, ny, xp, out);
  else if (ns == 2)
    adr_flux_kernel<P, 2><<<1, block, 0, st>>>(g, ref, links, plane, nx_pad, ny, xp, out);
  else if (ns == 3)
    adr_flux_kernel<P, 3><<<1, block, 0, st>>>(g, ref, links, plane, nx_pad, ny, xp, out);
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

template <class P>
cudaError_t launch_adjoint(int ns, int mode, const AdjArgs &a, cudaStream_t st) {
  using T = typename P::T;
  const dim3 block(kBlockX);
  const dim3 grid = adr_node_grid(a.nx_pad, a.ny);
#define LBM_ADJ_CASE(NS)                                                  \
  if (ns == NS) {                                                         \
    if (mode == kAdjCheck) {                                              \
      if (a.periodic)                                                     \
        adj_kernel<T, NS, kAdjCheck, true><<<grid, block, 0, st>>>(a);    \
      else                                                                \
        adj_kernel<T, NS, kAdjCheck, false><<<grid, block, 0, st>>>(a);   \
    } else {                                                              \
      if (a.periodic)                                                     \
        adj_kernel<T, NS, kAdjStep, true><<<grid, block, 0, st>>>(a);     \
      else                                                                \
        adj_kernel<T, NS, kAdjStep, false><<<grid, block, 0, st>>>(a);    \
    }                                                                     \
    return cudaGetLastError();                                            \
  }
  LBM_ADJ_CASE(1)
  LBM_ADJ_CASE(2)
  LBM_ADJ_CASE(3)
#undef LBM_ADJ_CASE
  return cudaErrorInvalidValue;
}

template <class P>
cudaError_t launch_adjoint_grad(int ns, const AdjArgs &a, const long long *bnodes,
                                long long nbnd, const void *conc, double *dkab,
                                double *dkbc, const int32_t *fiber, double *dw,
                                double k1, double k2, cudaStream_t st) {
  using T = typename P::T;
  if (nbnd == 0) return cudaSuccess;
  const dim3 block(kBlockX);
  const unsigned nb = static_cast<unsigned>(adr_list_blocks(nbnd));
  const T *c = static_cast<const T *>(conc);
  switch (ns) {
    case 1: adj_grad_kernel<T, 1><<<nb, block, 0, st>>>(a, bnodes, nbnd, c, dkab, dkbc, fiber, dw, k1, k2); break;
    case 2: adj_grad_kernel<T, 2><<<nb, block, 0, st>>>(a, bnodes, nbnd, c, dkab, dkbc, fiber, dw, k1, k2); break;
    case 3: adj_grad_kernel<T, 3><<<nb, block, 0, st>>>(a, bnodes, nbnd, c, dkab, dkbc, fiber, dw, k1, k2); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
