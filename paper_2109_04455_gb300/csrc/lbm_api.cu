// Host side of the liblbm C ABI (include/lbm.h): argument checks, workspace
// carving, the solve loops and their convergence checks.  All device memory
// is the caller's; this file only launches kernels on the caller's stream.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "lbm_kernels.cuh"
#include "lbm_nvtx.h"

namespace lbm {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

template <int KS, int KM>
static cudaError_t reduce_two_level(const double *partials, long long nb,
                                   double *scratch, double *out,
                                   cudaStream_t st) {
  const dim3 block(kReduceThreads);
  const long long g = nb < kReduceGrid ? (nb > 0 ? nb : 1) : kReduceGrid;
  const long long chunk = (nb + g - 1) / g;
  reduce_partials_kernel<KS, KM><<<static_cast<unsigned>(g), block, 0, st>>>(
      partials, nb, chunk, scratch);
  reduce_partials_kernel<KS, KM><<<1, block, 0, st>>>(scratch, g, g, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(int ks, int km, const double *partials, long long nb,
                          double *scratch, double *out, cudaStream_t st) {
  if (ks == 2 && km == 0) return reduce_two_level<2, 0>(partials, nb, scratch, out, st);
  if (ks == 2 && km == 1) return reduce_two_level<2, 1>(partials, nb, scratch, out, st);
  if (ks == 4 && km == 2) return reduce_two_level<4, 2>(partials, nb, scratch, out, st);
  if (ks == 6 && km == 3) return reduce_two_level<6, 3>(partials, nb, scratch, out, st);
  return cudaErrorInvalidValue;
}

namespace {

inline cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

inline long long plane_of(const lbm_geometry *g) {
  return static_cast<long long>(g->nx_pad) * g->ny;
}

inline dim3 lattice_grid(const lbm_geometry *g) {
  return dim3(static_cast<unsigned>((g->nx_pad + kBlockX - 1) / kBlockX),
              static_cast<unsigned>(g->ny));
}

inline long long grid_blocks(const lbm_geometry *g) {
  const dim3 gr = lattice_grid(g);
  return static_cast<long long>(gr.x) * gr.y;
}

inline bool aligned256(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) & 255u) == 0;
}

lbm_status cuda_fail(const char *where, cudaError_t e) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return LBM_ECUDA;
}

size_t store_bytes(int prec) {
  return prec == LBM_F64 ? 8 : (prec == LBM_F32 ? 4 : 2);
}
size_t compute_bytes(int prec) { return prec == LBM_F64 ? 8 : 4; }

// Make the device that owns `p` current for this thread (the caller's
// buffers decide where the work runs); rejects host memory.
lbm_status bind_device(const void *p, const char *where) {
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) return cuda_fail(where, e);
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
    set_error(std::string(where) + ": buffer is not device memory");
    return LBM_EINVAL;
  }
  int cur = -1;
  e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != at.device) e = cudaSetDevice(at.device);
  if (e != cudaSuccess) return cuda_fail(where, e);
  return LBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" const char *lbm_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// geometry upload
// ---------------------------------------------------------------------------
extern "C" size_t lbm_geometry_ws_bytes(const lbm_geometry *g) {
  if (!g) return 0;
  const size_t p = static_cast<size_t>(plane_of(g));
  return align256(4 * p) + 2 * align256(8 * p) + align256(8 * g->bnodes.size() + 8);
}

extern "C" lbm_status lbm_geometry_upload(lbm_geometry *g, void *dev_ws,
                                          size_t ws_bytes, void *stream) {
  if (!g || !dev_ws) {
    set_error("lbm_geometry_upload: NULL argument");
    return LBM_EINVAL;
  }
  if (!aligned256(dev_ws)) {
    set_error("lbm_geometry_upload: workspace not 256-byte aligned");
    return LBM_EINVAL;
  }
  const size_t need = lbm_geometry_ws_bytes(g);
  if (ws_bytes < need) {
    set_error("lbm_geometry_upload: workspace too small (" +
              std::to_string(ws_bytes) + " < " + std::to_string(need) + ")");
    return LBM_ENOMEM;
  }
  if (lbm_status bs = bind_device(dev_ws, "lbm_geometry_upload")) return bs;
  const size_t p = static_cast<size_t>(plane_of(g));
  char *b = static_cast<char *>(dev_ws);
  uint32_t *d_links = reinterpret_cast<uint32_t *>(b);
  double *d_kab = reinterpret_cast<double *>(b + align256(4 * p));
  double *d_kbc = reinterpret_cast<double *>(b + align256(4 * p) + align256(8 * p));
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(d_links, g->links.data(), 4 * p,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_kab, g->kab.data(), 8 * p, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_kbc, g->kbc.data(), 8 * p, cudaMemcpyHostToDevice, st);
  long long *d_bnodes = reinterpret_cast<long long *>(
      b + align256(4 * p) + 2 * align256(8 * p));
  if (e == cudaSuccess && !g->bnodes.empty())
    e = cudaMemcpyAsync(d_bnodes, g->bnodes.data(), 8 * g->bnodes.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("lbm_geometry_upload", e);
  g->d_links = d_links;
  g->d_kab = d_kab;
  g->d_kbc = d_kbc;
  g->d_bnodes = d_bnodes;
  g->uploaded = true;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// flow
// ---------------------------------------------------------------------------
static int flow_prec(int32_t precision) {
  return precision == LBM_F64 ? LBM_F64 : LBM_F32;
}

extern "C" size_t lbm_flow_ws_bytes(const lbm_geometry *g, int32_t precision) {
  if (!g) return 0;
  const size_t p = static_cast<size_t>(plane_of(g));
  const size_t es = store_bytes(flow_prec(precision));
  return 2 * align256(9 * p * es) +
         align256(static_cast<size_t>(grid_blocks(g)) * 2 * 8) +
         align256(kReduceGrid * 2 * 8) + align256(64 * 8);
}

static cudaError_t flow_launch(int prec, int mode, const FlowArgs &a, dim3 grid,
                               cudaStream_t st) {
  return prec == LBM_F64 ? launch_flow<PrecF64>(mode, a, grid, st)
                         : launch_flow<PrecF32>(mode, a, grid, st);
}

extern "C" lbm_status lbm_flow_solve(const lbm_geometry *g,
                                     const lbm_flow_params *p, void *f_ws,
                                     size_t f_ws_bytes, void *u_out,
                                     void *stream, lbm_solve_info *info) {
  NvtxRange nvtx_range("lbm_flow_solve");
  if (!g || !p || !f_ws || !u_out) {
    set_error("lbm_flow_solve: NULL argument");
    return LBM_EINVAL;
  }
  if (!g->uploaded) {
    set_error("lbm_flow_solve: geometry not uploaded");
    return LBM_EINVAL;
  }
  if (!(p->tau > 0.5) || p->max_steps < 2 || p->check_every < 2 ||
      !std::isfinite(p->u0)) {
    set_error("lbm_flow_solve: need tau > 1/2, max_steps >= 2, check_every >= 2");
    return LBM_EINVAL;
  }
  if (!aligned256(f_ws) || !aligned256(u_out)) {
    set_error("lbm_flow_solve: device buffers must be 256-byte aligned");
    return LBM_EINVAL;
  }
  const int prec = flow_prec(p->precision);
  const size_t need = lbm_flow_ws_bytes(g, p->precision);
  if (f_ws_bytes < need) {
    set_error("lbm_flow_solve: workspace too small");
    return LBM_ENOMEM;
  }
  if (lbm_status bs = bind_device(f_ws, "lbm_flow_solve")) return bs;
  const size_t pl = static_cast<size_t>(plane_of(g));
  const size_t bufb = align256(9 * pl * store_bytes(prec));
  char *b = static_cast<char *>(f_ws);
  void *buf[2] = {b, b + bufb};
  double *partials = reinterpret_cast<double *>(b + 2 * bufb);
  double *scratch = reinterpret_cast<double *>(
      b + 2 * bufb + align256(static_cast<size_t>(grid_blocks(g)) * 16));
  double *result = reinterpret_cast<double *>(
      b + 2 * bufb + align256(static_cast<size_t>(grid_blocks(g)) * 16) +
      align256(kReduceGrid * 2 * 8));
  cudaStream_t st = as_stream(stream);
  const dim3 grid = lattice_grid(g);

  FlowArgs a{};
  a.links = g->d_links;
  a.u = u_out;
  a.partials = partials;
  a.plane = plane_of(g);
  a.nx = g->nx;
  a.ny = g->ny;
  a.nx_pad = g->nx_pad;
  a.omega = 1.0 / p->tau;
  a.u0 = p->u0;
  a.fomega = static_cast<float>(a.omega);
  a.fu0 = static_cast<float>(a.u0);

  cudaError_t e = cudaMemsetAsync(b, 0, 2 * bufb, st);
  if (e != cudaSuccess) return cuda_fail("lbm_flow_solve", e);
  a.src = nullptr;
  a.dst = buf[0];
  e = flow_launch(prec, kFlowInit, a, grid, st);
  if (e != cudaSuccess) return cuda_fail("lbm_flow_solve(init)", e);
  int cur = 0;
  int64_t steps = 0;
  double residual = INFINITY;
  bool converged = false;

  auto step = [&](int mode) -> cudaError_t {
    a.src = buf[cur];
    a.dst = buf[cur ^ 1];
    cur ^= 1;
    ++steps;
    return flow_launch(prec, mode, a, grid, st);
  };
  // n steps, the last two writing u and the residual sums
  auto chunk = [&](int64_t n) -> lbm_status {
    for (int64_t k = 0; k < n - 2; ++k) {
      cudaError_t e2 = step(kFlowStep);
      if (e2 != cudaSuccess) return cuda_fail("lbm_flow_solve(step)", e2);
    }
    cudaError_t e2 = step(kFlowU);
    if (e2 == cudaSuccess) e2 = step(kFlowCheck);
    if (e2 == cudaSuccess)
      e2 = launch_reduce(2, 0, partials, grid_blocks(g), scratch, result, st);
    double h[2] = {0, 0};
    if (e2 == cudaSuccess)
      e2 = cudaMemcpyAsync(h, result, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) return cuda_fail("lbm_flow_solve(check)", e2);
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) {
      residual = NAN;
      set_error("lbm_flow_solve: non-finite velocity");
      return LBM_EUNSTABLE;
    }
    residual = h[1] > 0 ? h[0] / h[1] : 0.0;
    return LBM_OK;
  };

  lbm_status s = LBM_OK;
  if (p->tol <= 0) {
    s = chunk(p->max_steps);
  } else {
    while (s == LBM_OK) {
      const int64_t left = p->max_steps - steps;
      const int64_t n = left < p->check_every ? left : p->check_every;
      s = chunk(n < 2 ? 2 : n);
      if (s != LBM_OK) break;
      if (residual < p->tol) {
        converged = true;
        break;
      }
      if (steps >= p->max_steps) {
        set_error("lbm_flow_solve: not converged within max_steps");
        s = LBM_ENOTCONVERGED;
      }
    }
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->steps = steps;
    info->residual = residual;
    info->converged = converged ? 1 : 0;
  }
  return s;
}

// ---------------------------------------------------------------------------
// ADR
// ---------------------------------------------------------------------------
struct lbm_adr_solver {
  const lbm_geometry *g = nullptr;
  lbm_adr_params p{};
  AdrArgs a{};
  void *buf[2] = {nullptr, nullptr};
  void *cprev = nullptr;
  double *partials = nullptr;
  double *scratch = nullptr;
  double *result = nullptr;
  RefT *rbuf[2] = {nullptr, nullptr};  // reference concentrations (half)
  int cur = 0;
  int64_t steps = 0;
  bool has_check = false;
  long long nb = 0;
  AdrOverlap ov;   // boundary kernel beside the bulk kernel
};

struct AdrLayout {
  size_t buf, cprev, partials, scratch, result, ref, etab, total;
};

static AdrLayout adr_layout(const lbm_geometry *g, const lbm_adr_params *p) {
  const size_t pl = static_cast<size_t>(plane_of(g));
  const size_t ns = static_cast<size_t>(p->nspecies);
  AdrLayout l{};
  l.buf = align256(ns * 9 * pl * store_bytes(p->precision));
  l.cprev = align256(ns * pl * compute_bytes(p->precision));
  l.partials = align256(static_cast<size_t>(adr_partial_rows(
                            g->nx_pad, g->ny,
                            static_cast<long long>(g->bnodes.size()))) *
                        3 * ns * 8);
  l.scratch = align256(kReduceGrid * 3 * ns * 8);
  l.result = align256(kResSlots * 8);
  // half storage: per-node reference concentrations of both buffers
  l.ref = p->precision == LBM_F16DEV ? align256(ns * pl * sizeof(RefT)) : 0;
  // FP64: the equilibrium factors E_i(u) of the frozen velocity [9][plane]
  l.etab = p->precision == LBM_F64 ? align256(9 * pl * sizeof(double)) : 0;
  l.total = 2 * l.buf + l.cprev + l.partials + l.scratch + l.result +
            2 * l.ref + l.etab;
  return l;
}

static bool adr_params_ok(const lbm_adr_params *p) {
  if (p->nspecies < 1 || p->nspecies > 3) return false;
  if (p->precision < LBM_F64 || p->precision > LBM_F16DEV) return false;
  for (int s = 0; s < p->nspecies; ++s)
    if (!(p->tau[s] > 0.5) || !std::isfinite(p->c_in[s])) return false;
  if (p->flags & ~(LBM_ADR_INLET_ABB_ALL | LBM_ADR_NODEWISE)) return false;
  return true;
}

extern "C" size_t lbm_adr_ws_bytes(const lbm_geometry *g,
                                   const lbm_adr_params *p) {
  if (!g || !p || !adr_params_ok(p)) return 0;
  return adr_layout(g, p).total;
}

static cudaError_t adr_launch(int prec, int ns, int mode, const AdrArgs &a,
                              cudaStream_t st, const AdrOverlap *ov = nullptr) {
  switch (prec) {
    case LBM_F64: return launch_adr<PrecF64>(ns, mode, a, st, ov);
    case LBM_F32: return launch_adr<PrecF32>(ns, mode, a, st, ov);
    default: return launch_adr<PrecF16Dev>(ns, mode, a, st, ov);
  }
}

static cudaError_t adr_flux_launch(const lbm_adr_solver *s, cudaStream_t st) {
  const lbm_geometry *g = s->g;
  int xp = s->p.x_plane < 0 ? g->nx - 3 : s->p.x_plane;
  const void *cur = s->buf[s->cur];
  const RefT *ref = s->rbuf[s->cur];
  double *out = s->result + kResFlux;
  const int ns = s->p.nspecies;
  switch (s->p.precision) {
    case LBM_F64:
      return launch_adr_flux<PrecF64>(ns, cur, ref, g->d_links, plane_of(g),
                                      g->nx_pad, g->ny, xp, out, st);
    case LBM_F32:
      return launch_adr_flux<PrecF32>(ns, cur, ref, g->d_links, plane_of(g),
                                      g->nx_pad, g->ny, xp, out, st);
    default:
      return launch_adr_flux<PrecF16Dev>(ns, cur, ref, g->d_links, plane_of(g),
                                         g->nx_pad, g->ny, xp, out, st);
  }
}

extern "C" lbm_status lbm_adr_create(const lbm_geometry *g,
                                     const lbm_adr_params *p, const void *u,
                                     void *ws, size_t ws_bytes,
                                     lbm_adr_solver **out) {
  if (!out) {
    set_error("lbm_adr_create: out is NULL");
    return LBM_EINVAL;
  }
  *out = nullptr;
  if (!g || !p || !u || !ws) {
    set_error("lbm_adr_create: NULL argument");
    return LBM_EINVAL;
  }
  if (!g->uploaded) {
    set_error("lbm_adr_create: geometry not uploaded");
    return LBM_EINVAL;
  }
  if (!adr_params_ok(p)) {
    set_error("lbm_adr_create: need 1..3 species, a known precision, tau > 1/2");
    return LBM_EINVAL;
  }
  const int xp = p->x_plane < 0 ? g->nx - 3 : p->x_plane;
  if (xp < 0 || xp >= g->nx) {
    set_error("lbm_adr_create: flux plane outside the lattice");
    return LBM_EINVAL;
  }
  if (!aligned256(u) || !aligned256(ws)) {
    set_error("lbm_adr_create: device buffers must be 256-byte aligned");
    return LBM_EINVAL;
  }
  const AdrLayout l = adr_layout(g, p);
  if (ws_bytes < l.total) {
    set_error("lbm_adr_create: workspace too small (" + std::to_string(ws_bytes) +
              " < " + std::to_string(l.total) + ")");
    return LBM_ENOMEM;
  }
  if (lbm_status bs = bind_device(ws, "lbm_adr_create")) return bs;
  lbm_adr_solver *s = new (std::nothrow) lbm_adr_solver;
  if (!s) {
    set_error("lbm_adr_create: host allocation failed");
    return LBM_ENOMEM;
  }
  char *b = static_cast<char *>(ws);
  s->g = g;
  s->p = *p;
  s->buf[0] = b;
  s->buf[1] = b + l.buf;
  s->cprev = b + 2 * l.buf;
  s->partials = reinterpret_cast<double *>(b + 2 * l.buf + l.cprev);
  s->scratch = reinterpret_cast<double *>(b + 2 * l.buf + l.cprev + l.partials);
  s->result = reinterpret_cast<double *>(b + 2 * l.buf + l.cprev + l.partials +
                                         l.scratch);
  double *etab = nullptr;
  if (l.etab)
    etab = reinterpret_cast<double *>(b + 2 * l.buf + l.cprev + l.partials +
                                      l.scratch + l.result + 2 * l.ref);
  if (l.ref) {
    char *rb = b + 2 * l.buf + l.cprev + l.partials + l.scratch + l.result;
    s->rbuf[0] = reinterpret_cast<RefT *>(rb);
    s->rbuf[1] = reinterpret_cast<RefT *>(rb + l.ref);
  }
  s->nb = adr_partial_rows(g->nx_pad, g->ny,
                           static_cast<long long>(g->bnodes.size()));
  AdrArgs &a = s->a;
  a.links = g->d_links;
  a.kab = g->d_kab;
  a.kbc = g->d_kbc;
  a.u = u;
  a.etab = etab;
  a.cprev = s->cprev;
  a.partials = s->partials;
  a.bnodes = g->d_bnodes;
  a.nbnd = static_cast<long long>(g->bnodes.size());
  a.part_off = 0;
  a.plane = plane_of(g);
  a.nx = g->nx;
  a.ny = g->ny;
  a.nx_pad = g->nx_pad;
  a.abb_all = (p->flags & LBM_ADR_INLET_ABB_ALL) ? 1 : 0;
  a.nodewise = (p->flags & LBM_ADR_NODEWISE) ? 1 : 0;
  for (int k = 0; k < 3; ++k) {
    const bool on = k < p->nspecies;
    a.omega[k] = on ? 1.0 / p->tau[k] : 0.0;
    a.cin[k] = on ? p->c_in[k] : 0.0;
    a.fomega[k] = static_cast<float>(a.omega[k]);
    a.fcin[k] = static_cast<float>(a.cin[k]);
  }
  // second stream for the boundary-node kernel (no device memory involved)
  if (!g->bnodes.empty()) {
    cudaError_t e = cudaStreamCreateWithFlags(&s->ov.aux, cudaStreamNonBlocking);
    if (e == cudaSuccess)
      e = cudaEventCreateWithFlags(&s->ov.fork, cudaEventDisableTiming);
    if (e == cudaSuccess)
      e = cudaEventCreateWithFlags(&s->ov.join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      lbm_adr_destroy(s);
      return cuda_fail("lbm_adr_create", e);
    }
  }
  *out = s;
  return LBM_OK;
}

extern "C" void lbm_adr_destroy(lbm_adr_solver *s) {
  if (!s) return;
  if (s->ov.fork) cudaEventDestroy(s->ov.fork);
  if (s->ov.join) cudaEventDestroy(s->ov.join);
  if (s->ov.aux) cudaStreamDestroy(s->ov.aux);
  delete s;
}

extern "C" lbm_status lbm_adr_init(lbm_adr_solver *s, void *stream) {
  NvtxRange nvtx_range("lbm_adr_init");
  if (!s) {
    set_error("lbm_adr_init: solver is NULL");
    return LBM_EINVAL;
  }
  if (lbm_status bs = bind_device(s->buf[0], "lbm_adr_init")) return bs;
  cudaStream_t st = as_stream(stream);
  const AdrLayout l = adr_layout(s->g, &s->p);
  cudaError_t e = cudaMemsetAsync(s->buf[0], 0, 2 * l.buf + l.cprev, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->result, 0, kResSlots * sizeof(double), st);
  if (e == cudaSuccess && l.ref) e = cudaMemsetAsync(s->rbuf[0], 0, 2 * l.ref, st);
  if (e == cudaSuccess && s->a.etab)
    e = launch_eq_table(static_cast<const double *>(s->a.u), plane_of(s->g),
                        const_cast<double *>(s->a.etab), st);
  if (e != cudaSuccess) return cuda_fail("lbm_adr_init", e);
  AdrArgs a = s->a;
  a.src = nullptr;
  a.dst = s->buf[0];
  a.rsrc = nullptr;
  a.rdst = s->rbuf[0];
  e = adr_launch(s->p.precision, s->p.nspecies, kAdrInit, a, st);
  if (e != cudaSuccess) return cuda_fail("lbm_adr_init(kernel)", e);
  s->cur = 0;
  s->steps = 0;
  s->has_check = false;
  return LBM_OK;
}

static cudaError_t adr_step(lbm_adr_solver *s, int mode, cudaStream_t st) {
  AdrArgs a = s->a;
  a.src = s->buf[s->cur];
  a.dst = s->buf[s->cur ^ 1];
  a.rsrc = s->rbuf[s->cur];
  a.rdst = s->rbuf[s->cur ^ 1];
  a.step = static_cast<unsigned>(s->steps);
  s->cur ^= 1;
  ++s->steps;
  return adr_launch(s->p.precision, s->p.nspecies, mode, a, st, &s->ov);
}

extern "C" lbm_status lbm_adr_run(lbm_adr_solver *s, int64_t nsteps,
                                  void *stream, lbm_solve_info *info) {
  NvtxRange nvtx_range("lbm_adr_run");
  if (!s || nsteps < 0 || (info && nsteps < 2)) {
    set_error("lbm_adr_run: need a solver, nsteps >= 0 (>= 2 with info)");
    return LBM_EINVAL;
  }
  if (lbm_status bs = bind_device(s->buf[0], "lbm_adr_run")) return bs;
  cudaStream_t st = as_stream(stream);
  const int ns = s->p.nspecies;
  const int64_t plain = info ? nsteps - 2 : nsteps;
  for (int64_t k = 0; k < plain; ++k) {
    cudaError_t e = adr_step(s, kAdrStep, st);
    if (e != cudaSuccess) return cuda_fail("lbm_adr_run(step)", e);
  }
  if (!info) return LBM_OK;
  cudaError_t e = adr_step(s, kAdrCheck, st);
  if (e == cudaSuccess) e = adr_step(s, kAdrCheck, st);
  if (e == cudaSuccess)
    e = launch_reduce(2 * ns, ns, s->partials, s->nb, s->scratch, s->result, st);
  if (e == cudaSuccess) e = adr_flux_launch(s, st);
  double h[kResSlots] = {0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, s->result, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("lbm_adr_run(check)", e);
  s->has_check = true;
  std::memset(info, 0, sizeof(*info));
  info->steps = s->steps;
  bool finite = true;
  double r = 0.0;
  for (int k = 0; k < ns; ++k) {
    const double num = h[2 * k], den = h[2 * k + 1];
    finite = finite && std::isfinite(num) && std::isfinite(den) &&
             std::isfinite(h[kResFlux + k]);
    if (den > 0) r = std::fmax(r, num / den);
    info->flux[k] = h[kResFlux + k];
    info->c_min[k] = h[2 * ns + k];
    info->mass[k] = den;
  }
  info->residual = finite ? r : NAN;
  const bool negative = finite && adr_negative(&s->p, info->c_min);
  info->converged = (finite && !negative && s->p.tol > 0 && r < s->p.tol) ? 1 : 0;
  if (ns >= 2) {
    double eps = 0.0;
    if (lbm_efficiency(info->flux, ns, &eps) == LBM_OK) info->eps = eps;
  }
  if (!finite) {
    set_error("lbm_adr_run: non-finite concentration or flux at step " +
              std::to_string(s->steps));
    return LBM_EUNSTABLE;
  }
  if (negative) {
    double m = 0.0;
    for (int k = 0; k < ns; ++k) m = std::fmin(m, info->c_min[k]);
    set_error("lbm_adr_run: concentration " + std::to_string(m) +
              " below -neg_tol at step " + std::to_string(s->steps) +
              " (the scheme is losing stability: tau near 1/2?)");
    return LBM_EUNSTABLE;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_adr_conc(lbm_adr_solver *s, void *conc_out,
                                   void *stream) {
  if (!s || !conc_out) {
    set_error("lbm_adr_conc: NULL argument");
    return LBM_EINVAL;
  }
  if (!s->has_check) {
    set_error("lbm_adr_conc: no checked step yet (run with info first)");
    return LBM_EINVAL;
  }
  if (lbm_status bs = bind_device(conc_out, "lbm_adr_conc")) return bs;
  const size_t bytes = static_cast<size_t>(s->p.nspecies) *
                       static_cast<size_t>(plane_of(s->g)) *
                       compute_bytes(s->p.precision);
  cudaError_t e = cudaMemcpyAsync(conc_out, s->cprev, bytes,
                                  cudaMemcpyDeviceToDevice, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail("lbm_adr_conc", e);
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// checkpoint / resume: the populations (and, for half storage, the reference
// concentrations) of the current state are the whole state of a run
// ---------------------------------------------------------------------------
namespace {

struct StateHeader {
  uint64_t magic;
  int32_t version, precision, nspecies, nx, ny, nx_pad;
  int64_t steps;
  uint64_t pop_bytes, ref_bytes;
};
constexpr uint64_t kStateMagic = 0x4c424d4144525354ull;  // "LBMADRST"

size_t state_pop_bytes(const lbm_adr_solver *s) {
  return static_cast<size_t>(s->p.nspecies) * 9 *
         static_cast<size_t>(plane_of(s->g)) * store_bytes(s->p.precision);
}
size_t state_ref_bytes(const lbm_adr_solver *s) {
  return s->p.precision == LBM_F16DEV
             ? static_cast<size_t>(s->p.nspecies) *
                   static_cast<size_t>(plane_of(s->g)) * sizeof(RefT)
             : 0;
}

}  // namespace

extern "C" size_t lbm_adr_state_bytes(const lbm_adr_solver *s) {
  if (!s) return 0;
  return sizeof(StateHeader) + state_pop_bytes(s) + state_ref_bytes(s);
}

extern "C" lbm_status lbm_adr_state_save(lbm_adr_solver *s, void *host,
                                         size_t bytes, void *stream) {
  NvtxRange nvtx_range("lbm_adr_state_save");
  if (!s || !host) {
    set_error("lbm_adr_state_save: NULL argument");
    return LBM_EINVAL;
  }
  if (bytes < lbm_adr_state_bytes(s)) {
    set_error("lbm_adr_state_save: host buffer smaller than lbm_adr_state_bytes");
    return LBM_ENOMEM;
  }
  if (lbm_status bs = bind_device(s->buf[0], "lbm_adr_state_save")) return bs;
  StateHeader h{};
  h.magic = kStateMagic;
  h.version = 1;
  h.precision = s->p.precision;
  h.nspecies = s->p.nspecies;
  h.nx = s->g->nx;
  h.ny = s->g->ny;
  h.nx_pad = s->g->nx_pad;
  h.steps = s->steps;
  h.pop_bytes = state_pop_bytes(s);
  h.ref_bytes = state_ref_bytes(s);
  char *out = static_cast<char *>(host);
  std::memcpy(out, &h, sizeof(h));
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(out + sizeof(h), s->buf[s->cur], h.pop_bytes,
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && h.ref_bytes)
    e = cudaMemcpyAsync(out + sizeof(h) + h.pop_bytes, s->rbuf[s->cur],
                        h.ref_bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("lbm_adr_state_save", e);
  return LBM_OK;
}

extern "C" lbm_status lbm_adr_state_load(lbm_adr_solver *s, const void *host,
                                         size_t bytes, void *stream) {
  NvtxRange nvtx_range("lbm_adr_state_load");
  if (!s || !host) {
    set_error("lbm_adr_state_load: NULL argument");
    return LBM_EINVAL;
  }
  StateHeader h{};
  if (bytes < sizeof(h)) {
    set_error("lbm_adr_state_load: buffer too small for a state header");
    return LBM_EINVAL;
  }
  std::memcpy(&h, host, sizeof(h));
  if (h.magic != kStateMagic || h.version != 1 ||
      h.precision != s->p.precision || h.nspecies != s->p.nspecies ||
      h.nx != s->g->nx || h.ny != s->g->ny || h.nx_pad != s->g->nx_pad ||
      h.pop_bytes != state_pop_bytes(s) || h.ref_bytes != state_ref_bytes(s) ||
      h.steps < 0 || bytes < sizeof(h) + h.pop_bytes + h.ref_bytes) {
    set_error("lbm_adr_state_load: state does not match this solver "
              "(lattice, species count or precision) or is truncated");
    return LBM_EINVAL;
  }
  if (lbm_status bs = bind_device(s->buf[0], "lbm_adr_state_load")) return bs;
  const char *in = static_cast<const char *>(host);
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(s->buf[s->cur], in + sizeof(h), h.pop_bytes,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && h.ref_bytes)
    e = cudaMemcpyAsync(s->rbuf[s->cur], in + sizeof(h) + h.pop_bytes,
                        h.ref_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("lbm_adr_state_load", e);
  s->steps = h.steps;
  s->has_check = false;   // no concentrations recorded for this state yet
  return LBM_OK;
}

extern "C" lbm_status lbm_adr_solve(const lbm_geometry *g,
                                    const lbm_adr_params *p, const void *u,
                                    void *ws, size_t ws_bytes, void *conc_out,
                                    void *stream, lbm_solve_info *info) {
  NvtxRange nvtx_range("lbm_adr_solve");
  if (!p || p->max_steps < 2 ||
      ((p->tol > 0 || p->eps_tol > 0) && p->check_every < 2)) {
    set_error("lbm_adr_solve: need max_steps >= 2 and check_every >= 2");
    return LBM_EINVAL;
  }
  lbm_adr_solver *s = nullptr;
  lbm_status st = lbm_adr_create(g, p, u, ws, ws_bytes, &s);
  if (st != LBM_OK) return st;
  st = lbm_adr_init(s, stream);
  lbm_solve_info loc{};
  if (st == LBM_OK) {
    if (p->tol <= 0 && p->eps_tol <= 0) {
      st = lbm_adr_run(s, p->max_steps, stream, &loc);
    } else {
      double hist[3] = {NAN, NAN, NAN};   // efficiency at the last checks
      int nh = 0;
      while (true) {
        const int64_t left = p->max_steps - s->steps;
        const int64_t n = left < p->check_every ? left : p->check_every;
        st = lbm_adr_run(s, n < 2 ? 2 : n, stream, &loc);
        if (st != LBM_OK) break;
        hist[0] = hist[1];
        hist[1] = hist[2];
        hist[2] = loc.eps;
        ++nh;
        bool conv = p->tol <= 0 || loc.residual < p->tol;
        if (conv && p->eps_tol > 0)
          conv = nh >= 3 && eps_distance(hist[0], hist[1], hist[2],
                                         0.1 * p->eps_tol) < p->eps_tol;
        loc.converged = conv ? 1 : 0;
        if (conv) break;
        if (s->steps >= p->max_steps) {
          set_error("lbm_adr_solve: not converged within max_steps");
          st = LBM_ENOTCONVERGED;
          break;
        }
      }
    }
  }
  if ((st == LBM_OK || st == LBM_ENOTCONVERGED) && conc_out) {
    lbm_status c = lbm_adr_conc(s, conc_out, stream);
    if (c == LBM_OK) {
      cudaError_t e = cudaStreamSynchronize(as_stream(stream));
      if (e != cudaSuccess) c = cuda_fail("lbm_adr_solve", e);
    }
    if (c != LBM_OK) st = c;
  }
  if (info) *info = loc;
  lbm_adr_destroy(s);
  return st;
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
struct AdjLayout {
  size_t buf, partials, scratch, result, fiber, total;
};

static AdjLayout adj_layout(const lbm_geometry *g, const lbm_adr_params *p) {
  const size_t pl = static_cast<size_t>(plane_of(g));
  const size_t ns = static_cast<size_t>(p->nspecies);
  const dim3 gr = adr_node_grid(g->nx_pad, g->ny);
  AdjLayout l{};
  l.buf = align256(ns * 9 * pl * compute_bytes(p->precision));
  l.partials = align256(static_cast<size_t>(gr.x) * gr.y * 2 * 8);
  l.scratch = align256(kReduceGrid * 2 * 8);
  l.result = align256(kResSlots * 8);
  l.fiber = align256(4 * pl);
  l.total = 2 * l.buf + l.partials + l.scratch + l.result + l.fiber;
  return l;
}

extern "C" size_t lbm_adr_adjoint_ws_bytes(const lbm_geometry *g,
                                           const lbm_adr_params *p) {
  if (!g || !p || !adr_params_ok(p) || p->precision == LBM_F16DEV) return 0;
  return adj_layout(g, p).total;
}

static cudaError_t adj_launch(int prec, int ns, int mode, const AdjArgs &a,
                              cudaStream_t st) {
  return prec == LBM_F64 ? launch_adjoint<PrecF64>(ns, mode, a, st)
                         : launch_adjoint<PrecF32>(ns, mode, a, st);
}

// d eps / d N_s of Eq. (A-B)
static void efficiency_sensitivity(const double *f, int ns, double *d) {
  d[0] = d[1] = d[2] = 0.0;
  if (ns == 2) {
    const double t = f[0] + f[1];
    d[0] = -f[1] / (t * t);
    d[1] = f[0] / (t * t);
  } else if (ns == 3) {
    const double t = f[0] + f[1] + f[2];
    d[0] = d[1] = -f[2] / (t * t);
    d[2] = (f[0] + f[1]) / (t * t);
  }
}

extern "C" lbm_status lbm_adr_adjoint(lbm_adr_solver *s, int64_t max_steps,
                                      double tol, int32_t check_every, void *ws,
                                      size_t ws_bytes, void *dkab, void *dkbc,
                                      void *dw, void *stream,
                                      lbm_solve_info *info) {
  NvtxRange nvtx_range("lbm_adr_adjoint");
  if (!s || !ws || !dkab || !dkbc) {
    set_error("lbm_adr_adjoint: NULL argument");
    return LBM_EINVAL;
  }
  const lbm_geometry *g = s->g;
  const int ns = s->p.nspecies;
  const int prec = s->p.precision;
  if (ns < 2 || prec == LBM_F16DEV) {
    set_error("lbm_adr_adjoint: needs 2 or 3 species and LBM_F64 / LBM_F32");
    return LBM_EINVAL;
  }
  if (s->p.flags & LBM_ADR_NODEWISE) {
    set_error("lbm_adr_adjoint: the node-wise reaction variant has no adjoint");
    return LBM_EINVAL;
  }
  if (!s->has_check) {
    set_error("lbm_adr_adjoint: run the solver with info first");
    return LBM_EINVAL;
  }
  if (max_steps < 1 || (tol > 0 && check_every < 2)) {
    set_error("lbm_adr_adjoint: need max_steps >= 1 (check_every >= 2 with tol)");
    return LBM_EINVAL;
  }
  if (!aligned256(ws) || !aligned256(dkab) || !aligned256(dkbc)) {
    set_error("lbm_adr_adjoint: device buffers must be 256-byte aligned");
    return LBM_EINVAL;
  }
  const AdjLayout l = adj_layout(g, &s->p);
  if (ws_bytes < l.total) {
    set_error("lbm_adr_adjoint: workspace too small");
    return LBM_ENOMEM;
  }
  if (lbm_status bs = bind_device(ws, "lbm_adr_adjoint")) return bs;
  cudaStream_t st = as_stream(stream);
  char *b = static_cast<char *>(ws);
  void *buf[2] = {b, b + l.buf};
  double *partials = reinterpret_cast<double *>(b + 2 * l.buf);
  double *scratch = reinterpret_cast<double *>(b + 2 * l.buf + l.partials);
  double *result = reinterpret_cast<double *>(b + 2 * l.buf + l.partials + l.scratch);
  int32_t *fiber = reinterpret_cast<int32_t *>(b + 2 * l.buf + l.partials +
                                               l.scratch + l.result);
  const size_t pl = static_cast<size_t>(plane_of(g));
  const dim3 gr = adr_node_grid(g->nx_pad, g->ny);
  const long long rows = static_cast<long long>(gr.x) * gr.y;

  // forward outfluxes of the current state -> d eps / d N_s
  cudaError_t e = adr_flux_launch(s, st);
  double h[kResSlots] = {0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, s->result, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("lbm_adr_adjoint(flux)", e);
  double flux[3] = {h[kResFlux], h[kResFlux + 1], h[kResFlux + 2]};
  double dN[3];
  efficiency_sensitivity(flux, ns, dN);
  if (!std::isfinite(dN[0]) || !std::isfinite(dN[1]) || !std::isfinite(dN[2])) {
    set_error("lbm_adr_adjoint: efficiency undefined (zero outflux)");
    return LBM_EUNSTABLE;
  }

  AdjArgs a{};
  a.links = g->d_links;
  a.kab = g->d_kab;
  a.kbc = g->d_kbc;
  a.u = s->a.u;
  a.etab = s->a.etab;
  a.partials = partials;
  a.plane = plane_of(g);
  a.nx = g->nx;
  a.ny = g->ny;
  a.nx_pad = g->nx_pad;
  a.xp = s->p.x_plane < 0 ? g->nx - 3 : s->p.x_plane;
  a.abb_all = s->a.abb_all;
  a.periodic = g->periodic != 0 ? 1 : 0;
  for (int k = 0; k < 3; ++k) {
    a.omega[k] = s->a.omega[k];
    a.dN[k] = dN[k];
    a.fomega[k] = static_cast<float>(a.omega[k]);
    a.fdN[k] = static_cast<float>(dN[k]);
  }
  e = cudaMemsetAsync(b, 0, 2 * l.buf, st);
  if (e != cudaSuccess) return cuda_fail("lbm_adr_adjoint", e);
  int cur = 0;
  int64_t steps = 0;
  double residual = INFINITY;
  bool converged = false;
  auto iterate = [&](int64_t n) -> lbm_status {
    for (int64_t k = 0; k < n; ++k) {
      a.src = buf[cur];
      a.dst = buf[cur ^ 1];
      const int mode = (k == n - 1) ? kAdjCheck : kAdjStep;
      cudaError_t e2 = adj_launch(prec, ns, mode, a, st);
      if (e2 != cudaSuccess) return cuda_fail("lbm_adr_adjoint(step)", e2);
      cur ^= 1;
      ++steps;
    }
    cudaError_t e2 = launch_reduce(2, 0, partials, rows, scratch, result, st);
    double r[2] = {0, 0};
    if (e2 == cudaSuccess)
      e2 = cudaMemcpyAsync(r, result, sizeof(r), cudaMemcpyDeviceToHost, st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) return cuda_fail("lbm_adr_adjoint(check)", e2);
    if (!std::isfinite(r[0]) || !std::isfinite(r[1])) {
      set_error("lbm_adr_adjoint: non-finite adjoint");
      return LBM_EUNSTABLE;
    }
    residual = r[1] > 0 ? r[0] / r[1] : 0.0;
    return LBM_OK;
  };
  lbm_status stt = LBM_OK;
  if (tol <= 0) {
    stt = iterate(max_steps);
  } else {
    while (stt == LBM_OK) {
      const int64_t left = max_steps - steps;
      stt = iterate(left < check_every ? left : check_every);
      if (stt != LBM_OK) break;
      if (residual < tol) {
        converged = true;
        break;
      }
      if (steps >= max_steps) {
        set_error("lbm_adr_adjoint: not converged within max_steps");
        stt = LBM_ENOTCONVERGED;
      }
    }
  }
  if (stt == LBM_OK || stt == LBM_ENOTCONVERGED) {
    // gradients from the final adjoint and the recorded concentrations
    e = cudaMemsetAsync(dkab, 0, 8 * pl, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dkbc, 0, 8 * pl, st);
    if (e == cudaSuccess && dw && g->nfibers > 0)
      e = cudaMemsetAsync(dw, 0, 8 * static_cast<size_t>(g->nfibers), st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(fiber, g->fiber.data(), 4 * pl, cudaMemcpyHostToDevice, st);
    a.src = buf[cur];
    a.dst = nullptr;
    const long long nbnd = static_cast<long long>(g->bnodes.size());
    if (e == cudaSuccess) {
      e = prec == LBM_F64
              ? launch_adjoint_grad<PrecF64>(ns, a, g->d_bnodes, nbnd, s->cprev,
                                             static_cast<double *>(dkab),
                                             static_cast<double *>(dkbc), fiber,
                                             static_cast<double *>(dw), g->k1,
                                             g->k2, st)
              : launch_adjoint_grad<PrecF32>(ns, a, g->d_bnodes, nbnd, s->cprev,
                                             static_cast<double *>(dkab),
                                             static_cast<double *>(dkbc), fiber,
                                             static_cast<double *>(dw), g->k1,
                                             g->k2, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail("lbm_adr_adjoint(gradient)", e);
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->steps = steps;
    info->residual = residual;
    info->converged = converged ? 1 : 0;
    for (int k = 0; k < 3; ++k) info->flux[k] = flux[k];
    double eps = 0.0;
    if (lbm_efficiency(flux, ns, &eps) == LBM_OK) info->eps = eps;
  }
  return stt;
}

// ---------------------------------------------------------------------------
// outflux without any workspace
//
// For callers that cannot allocate device memory at the point where they
// want the fluxes: e.g. a monitor or plugin running inside an application
// that reserved all device memory for its own pool at start-up (a cudaMalloc
// would fail or fragment that pool), or a time-critical loop that must not
// pay cudaMalloc's implicit device synchronisation.  Instead of a caller
// workspace, the per-block partial sums live in the fixed-size array below,
// which every GPU that loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace lbm {
namespace noalloc {
constexpr int kRowsPerBlock = 256;
constexpr int kMaxRows = 65536;  // a geometry has at most 65535 rows
constexpr int kMaxBlocks = kMaxRows / kRowsPerBlock;
constexpr int kFinal = kMaxBlocks * 3;  // offset of the result
}  // namespace noalloc
}  // namespace lbm

// [kMaxBlocks][3] block partial sums, then the 3 outfluxes (6 KB per GPU)
static __device__ __align__(256) double
    g_noalloc_scratch[lbm::noalloc::kMaxBlocks * 3 + 3];

namespace lbm {
namespace noalloc {

// Rows [b*256, b*256+256) of the plane x = xp: per species the sum over those
// rows of sum_i c_ix g*_{s,i}, written to part[b*3 + s].  Every block writes
// all three slots, so nothing has to start at zero.
template <class P, int NS>
__global__ void __launch_bounds__(kRowsPerBlock)
    outflux_partial_noalloc_kernel(const void *g, const RefT *ref,
                                   const uint32_t *links, long long plane,
                                   int nx_pad, int ny, int xp, double *part) {
  using S = typename P::S;
  const S *src = static_cast<const S *>(g);
  const int y = blockIdx.x * kRowsPerBlock + threadIdx.x;
  double acc[3] = {0.0, 0.0, 0.0};
  if (y < ny) {
    const long long n = (long long)y * nx_pad + xp;
    if (links[n] != kSolidNode) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
          if (cx(i) == 0) continue;
          double gi = double(P::load(src[(long long)(s * 9 + i) * plane + n]));
          if (P::kDev) gi += double(Lattice<float>::w(i)) * double(ref_get(ref, s * plane + n));
          acc[s] += cx(i) > 0 ? gi : -gi;
        }
      }
    }
  }
  block_sum_store<3, double>(acc, part + blockIdx.x * 3);
}

// One block: out[s] = (sum over the nb block partials) / ny.
__global__ void __launch_bounds__(kReduceThreads)
    outflux_final_noalloc_kernel(const double *part, int nb, int ny,
                                 double *out) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
    for (int s = 0; s < 3; ++s) acc[s] += part[b * 3 + s];
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) acc[s] /= double(ny);
  block_sum_store<3, double>(acc, out);
}

template <class P>
cudaError_t outflux_noalloc_launch(int ns, const void *g, const RefT *ref,
                                   const uint32_t *links, long long plane,
                                   int nx_pad, int ny, int xp, double *scratch,
                                   cudaStream_t st) {
  const int nb = (ny + kRowsPerBlock - 1) / kRowsPerBlock;
  const dim3 block(kRowsPerBlock);
  switch (ns) {
    case 1:
      outflux_partial_noalloc_kernel<P, 1><<<nb, block, 0, st>>>(
          g, ref, links, plane, nx_pad, ny, xp, scratch);
      break;
    case 2:
      outflux_partial_noalloc_kernel<P, 2><<<nb, block, 0, st>>>(
          g, ref, links, plane, nx_pad, ny, xp, scratch);
      break;
    default:
      outflux_partial_noalloc_kernel<P, 3><<<nb, block, 0, st>>>(
          g, ref, links, plane, nx_pad, ny, xp, scratch);
      break;
  }
  outflux_final_noalloc_kernel<<<1, dim3(kReduceThreads), 0, st>>>(
      scratch, nb, ny, scratch + kFinal);
  return cudaGetLastError();
}

}  // namespace noalloc
}  // namespace lbm

extern "C" lbm_status lbm_adr_outflux_noalloc(lbm_adr_solver *s,
                                              int32_t x_plane, void *stream,
                                              double *flux_out) {
  if (!s || !flux_out) {
    set_error("lbm_adr_outflux_noalloc: NULL argument");
    return LBM_EINVAL;
  }
  const lbm_geometry *g = s->g;
  const int xp = x_plane < 0 ? g->nx - 3 : x_plane;
  if (xp >= g->nx) {
    set_error("lbm_adr_outflux_noalloc: flux plane outside the lattice");
    return LBM_EINVAL;
  }
  if (g->ny > noalloc::kMaxRows) {
    set_error("lbm_adr_outflux_noalloc: ny = " + std::to_string(g->ny) +
              " exceeds the " + std::to_string(noalloc::kMaxRows) +
              "-row limit of its fixed scratch array");
    return LBM_EINVAL;
  }
  if (lbm_status bs = bind_device(s->buf[0], "lbm_adr_outflux_noalloc")) return bs;
  // The array's name is a host-side stand-in: its device address (on the
  // device the solver's buffers live on, now current) is looked up on every
  // call, so a context torn down and rebuilt (cudaDeviceReset) cannot leave
  // a stale address behind.  The lookup allocates nothing.
  void *sym = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&sym, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail("lbm_adr_outflux_noalloc(address)", e);
  double *scratch = static_cast<double *>(sym);
  cudaStream_t st = as_stream(stream);
  const void *cur = s->buf[s->cur];
  const int ns = s->p.nspecies;
  switch (s->p.precision) {
    case LBM_F64:
      e = noalloc::outflux_noalloc_launch<PrecF64>(ns, cur, s->rbuf[s->cur], g->d_links,
                                                   plane_of(g), g->nx_pad, g->ny, xp,
                                                   scratch, st);
      break;
    case LBM_F32:
      e = noalloc::outflux_noalloc_launch<PrecF32>(ns, cur, s->rbuf[s->cur], g->d_links,
                                                   plane_of(g), g->nx_pad, g->ny, xp,
                                                   scratch, st);
      break;
    default:
      e = noalloc::outflux_noalloc_launch<PrecF16Dev>(ns, cur, s->rbuf[s->cur], g->d_links,
                                                   plane_of(g), g->nx_pad, g->ny, xp,
                                                   scratch, st);
      break;
  }
  double h[3] = {0.0, 0.0, 0.0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, scratch + noalloc::kFinal, sizeof(h),
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("lbm_adr_outflux_noalloc", e);
  for (int k = 0; k < 3; ++k) flux_out[k] = k < ns ? h[k] : 0.0;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// FP64 FMA throughput of the device: the denominator of the FP64 step's
// arithmetic roofline (that step is bound by the double-precision pipe, not
// by HBM).  Sixteen independent FMA chains per thread keep the pipe busy
// whatever its latency; the chains' sum is compared with a value it cannot
// take, so that the compiler keeps every FMA.
// ---------------------------------------------------------------------------
namespace lbm {
namespace peak {
constexpr int kChains = 16;
constexpr int kThreads = 256;
static __device__ double g_sink;

__global__ void __launch_bounds__(kThreads)
    fp64_fma_kernel(int iters, double seed, double mul, double add) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed + 1e-3 * c + 1e-9 * threadIdx.x;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __fma_rn(x[c], mul, add);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) g_sink = s;
}
}  // namespace peak
}  // namespace lbm

extern "C" lbm_status lbm_fp64_fma_tflops(void *stream, double *tflops) {
  if (!tflops) {
    set_error("lbm_fp64_fma_tflops: NULL argument");
    return LBM_EINVAL;
  }
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail("lbm_fp64_fma_tflops", e);
  cudaStream_t st = as_stream(stream);
  const int blocks = 8 * sms, iters = 2048;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first: warm-up
    e = cudaEventRecord(e0, st);
    peak::fp64_fma_kernel<<<blocks, peak::kThreads, 0, st>>>(iters, 0.5,
                                                             0.9999999, 1e-8);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail("lbm_fp64_fma_tflops", e);
  const double flops = 2.0 * peak::kChains * static_cast<double>(iters) *
                       blocks * peak::kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return LBM_OK;
}
