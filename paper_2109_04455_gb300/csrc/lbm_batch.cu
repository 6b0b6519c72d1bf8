// Batched ADR solves: many lattices of uneven size (a Pe x Da sweep) advanced
// together, one persistent launch per time step, replayed from a CUDA graph
// between convergence checks; the launch shape is picked by a small
// autotuner that times the candidates on the batch itself.
//
// Work list: every active instance contributes its interior row tiles (BX
// consecutive nodes of one row) and its boundary-node chunks (BX entries of
// its boundary list).  Items are stored instance by instance, so each
// instance's check-step partial sums occupy a contiguous row range.  A
// persistent grid of blocks walks the list; per item the instance's
// arguments are staged in shared memory and the same per-node updates as the
// single-lattice kernels run (adr_interior_node / adr_general_node), so a
// batched solve gives the same populations as lbm_adr_solve on each lattice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_kernels.cuh"
#include "lbm_nvtx.h"

namespace lbm {
namespace batch {

constexpr unsigned long long kChunkBit = 1ull << 63;

__host__ __device__ inline unsigned long long tile_item(int inst, long long y,
                                                         long long xb) {
  return (static_cast<unsigned long long>(inst) << 48) |
         (static_cast<unsigned long long>(y) << 24) |
         static_cast<unsigned long long>(xb);
}
__host__ __device__ inline unsigned long long chunk_item(int inst,
                                                          long long start) {
  return kChunkBit | (static_cast<unsigned long long>(inst) << 48) |
         static_cast<unsigned long long>(start);
}

// stepc[parity]: steps every active instance has done before this one (all
// start together); the launch passes it to the per-node updates as
// AdrArgs::step (the rounding seed of half storage) and leaves the next
// count in stepc[parity ^ 1] for the next launch.
template <class P, int NS, int MODE, int BX>
__global__ void __launch_bounds__(BX)
    batch_step_kernel(const AdrArgs *__restrict__ table, int parity,
                      const unsigned long long *__restrict__ work,
                      long long nwork, double *partials, unsigned *stepc) {
  using T = typename P::T;
  __shared__ AdrArgs sa;
  constexpr int kWords = sizeof(AdrArgs) / sizeof(unsigned long long);
  static_assert(sizeof(AdrArgs) % sizeof(unsigned long long) == 0,
                "AdrArgs is copied as 8-byte words");
  constexpr int kStepWord = static_cast<int>(offsetof(AdrArgs, step) / 8);
  constexpr int kStepShift = static_cast<int>(offsetof(AdrArgs, step) % 8) * 8;
  const unsigned step = stepc[parity];
  if (blockIdx.x == 0 && threadIdx.x == 0) stepc[parity ^ 1] = step + 1u;
  for (long long w = blockIdx.x; w < nwork; w += gridDim.x) {
    const unsigned long long item = work[w];
    const int inst = static_cast<int>((item >> 48) & 0x7fff);
    __syncthreads();  // the previous item is done with sa
    {
      const unsigned long long *srcw =
          reinterpret_cast<const unsigned long long *>(table + 2 * inst + parity);
      unsigned long long *dstw = reinterpret_cast<unsigned long long *>(&sa);
      for (int k = threadIdx.x; k < kWords; k += BX) {
        unsigned long long v = srcw[k];
        if (k == kStepWord)
          v = (v & ~(0xFFFFFFFFull << kStepShift)) |
              (static_cast<unsigned long long>(step) << kStepShift);
        dstw[k] = v;
      }
    }
    __syncthreads();
    T acc[1][3 * NS];
#pragma unroll
    for (int k = 0; k < 3 * NS; ++k) acc[0][k] = T(0);
    if (!(item & kChunkBit)) {
      const long long y = static_cast<long long>((item >> 24) & 0xffffff);
      const long long xb = static_cast<long long>(item & 0xffffff);
      const int x = static_cast<int>(xb * BX + threadIdx.x);
      const long long n = y * sa.nx_pad + x;
      const uint32_t lw = (x < sa.nx_pad) ? sa.links[n] : kSolidNode;
      if (lw == 0u) adr_interior_node<P, NS, MODE>(sa, n, acc[0]);
    } else {
      const long long t =
          static_cast<long long>(item & ((1ull << 48) - 1)) + threadIdx.x;
      if (t < sa.nbnd) {
        const long long n = sa.bnodes[t];
        adr_general_node<P, NS, MODE>(sa, n, static_cast<int>(n % sa.nx_pad),
                                      sa.links[n], acc[0]);
      }
    }
    if constexpr (MODE == kAdrCheck)
      block_partials_store<2 * NS, NS, 1, BX, T>(acc, partials + w * (3 * NS));
  }
}

// out[i*K + k] = fold of partial rows [rows[2i], rows[2i+1]) (one block per
// instance, fixed order): sums of the first 2 NS components, minima of the
// last NS.
template <int NS>
__global__ void __launch_bounds__(kReduceThreads)
    batch_reduce_kernel(const double *partials, const long long *rows,
                        double *out) {
  constexpr int K = 3 * NS;
  const long long lo = rows[2 * blockIdx.x], hi = rows[2 * blockIdx.x + 1];
  double acc[1][K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[0][k] = 0.0;
  for (long long b = lo + threadIdx.x; b < hi; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      acc[0][k] = k < 2 * NS ? acc[0][k] + partials[b * K + k]
                             : fmin(acc[0][k], partials[b * K + k]);
  }
  block_partials_store<2 * NS, NS, 1, kReduceThreads, double>(
      acc, out + (long long)blockIdx.x * K);
}

// Outflux of every instance on its plane (one block per instance), from the
// populations the last step wrote (table[2i + parity].dst).
template <class P, int NS>
__global__ void __launch_bounds__(kReduceThreads)
    batch_flux_kernel(const AdrArgs *table, int parity, double *out) {
  using S = typename P::S;
  const AdrArgs &a = table[2 * blockIdx.x + parity];
  const S *src = static_cast<const S *>(a.dst);
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  for (int y = threadIdx.x; y < a.ny; y += blockDim.x) {
    const long long n = (long long)y * a.nx_pad + a.xp;
    if (a.links[n] == kSolidNode) continue;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double v = 0.0;
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        if (cx(i) == 0) continue;
        double gi = double(P::load(src[(long long)(s * 9 + i) * a.plane + n]));
        if (P::kDev) gi += double(Lattice<float>::w(i)) * double(ref_get(a.rdst, s * a.plane + n));
        v += cx(i) > 0 ? gi : -gi;
      }
      acc[s] += v;
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] /= double(a.ny);
  block_sum_store<NS, double>(acc, out + (long long)blockIdx.x * 3);
}

template <class P, int NS>
cudaError_t launch_step(int mode, int bx, const AdrArgs *table, int parity,
                        const unsigned long long *work, long long nwork,
                        double *partials, unsigned *stepc, unsigned grid,
                        cudaStream_t st) {
  if (bx == 128) {
    if (mode == kAdrCheck)
      batch_step_kernel<P, NS, kAdrCheck, 128><<<grid, 128, 0, st>>>(table, parity, work, nwork, partials, stepc);
    else
      batch_step_kernel<P, NS, kAdrStep, 128><<<grid, 128, 0, st>>>(table, parity, work, nwork, partials, stepc);
  } else {
    if (mode == kAdrCheck)
      batch_step_kernel<P, NS, kAdrCheck, 256><<<grid, 256, 0, st>>>(table, parity, work, nwork, partials, stepc);
    else
      batch_step_kernel<P, NS, kAdrStep, 256><<<grid, 256, 0, st>>>(table, parity, work, nwork, partials, stepc);
  }
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_step_p(int ns, int mode, int bx, const AdrArgs *table,
                          int parity, const unsigned long long *work,
                          long long nwork, double *partials, unsigned *stepc,
                          unsigned grid, cudaStream_t st) {
  return ns == 2 ? launch_step<P, 2>(mode, bx, table, parity, work, nwork,
                                     partials, stepc, grid, st)
                 : launch_step<P, 3>(mode, bx, table, parity, work, nwork,
                                     partials, stepc, grid, st);
}

template <class P>
cudaError_t launch_flux_p(int ns, int count, const AdrArgs *table, int parity,
                          double *out, cudaStream_t st) {
  if (ns == 2)
    batch_flux_kernel<P, 2><<<count, kReduceThreads, 0, st>>>(table, parity, out);
  else
    batch_flux_kernel<P, 3><<<count, kReduceThreads, 0, st>>>(table, parity, out);
  return cudaGetLastError();
}

template <class P>
int occupancy(int ns, int bx) {
  int nb = 0;
  if (bx == 128)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, ns == 2 ? batch_step_kernel<P, 2, kAdrStep, 128>
                     : batch_step_kernel<P, 3, kAdrStep, 128>, 128, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, ns == 2 ? batch_step_kernel<P, 2, kAdrStep, 256>
                     : batch_step_kernel<P, 3, kAdrStep, 256>, 256, 0);
  return nb > 0 ? nb : 1;
}

inline size_t a256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace batch
}  // namespace lbm

using namespace lbm;
using namespace lbm::batch;

struct lbm_batch {
  int count = 0, ns = 0, prec = 0;
  std::vector<const lbm_geometry *> geoms;
  std::vector<lbm_adr_params> params;
  std::vector<AdrArgs> table;           // 2 per instance (parity 0 / 1)
  std::vector<const void *> u;
  // device regions
  AdrArgs *d_table = nullptr;
  unsigned long long *d_work = nullptr;
  double *d_partials = nullptr;
  long long *d_rows = nullptr;
  double *d_sums = nullptr;             // [count][3*ns]: sums, minima
  double *d_flux = nullptr;             // [count][3]
  unsigned *d_step = nullptr;           // [2] step count, ping-pong
  long long max_items = 0;
  // state
  int parity = 0;
  std::vector<char> active;
  std::vector<int64_t> steps;
  std::vector<double> eps_hist;         // [count][3] efficiency at the checks
  std::vector<int> nhist;
  int check_every = 100;
  // launch shape (autotuned)
  int bx = 256;
  unsigned grid = 0;
  bool tuned = false;
  float tune_ms[8] = {0};
  // work list of the current active set
  long long nwork = 0;
  std::vector<unsigned long long> work;
  std::vector<long long> rows;
  // captured chunk
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  bool solved = false;                  // a solve has recorded concentrations
};

namespace {

lbm_status bfail(const char *where, cudaError_t e) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return LBM_ECUDA;
}

long long items_of(const lbm_geometry *g, int bx) {
  const long long tiles = static_cast<long long>((g->nx_pad + bx - 1) / bx) * g->ny;
  const long long nb = static_cast<long long>(g->bnodes.size());
  return tiles + (nb + bx - 1) / bx;
}

size_t store_b(int prec) { return prec == LBM_F64 ? 8 : (prec == LBM_F32 ? 4 : 2); }
size_t comp_b(int prec) { return prec == LBM_F64 ? 8 : 4; }

struct BatchLayout {
  size_t table, work, partials, rows, sums, flux, step, head, total;
  std::vector<size_t> inst_off;  // start of each instance's buffers
  std::vector<size_t> buf;       // bytes of one population buffer
  std::vector<size_t> cprev;
  std::vector<size_t> ref;       // bytes of one reference buffer (half only)
};

BatchLayout batch_layout(int count, const lbm_geometry *const *geoms,
                         const lbm_adr_params *p) {
  BatchLayout l{};
  const int ns = p[0].nspecies;
  long long items = 0;
  for (int i = 0; i < count; ++i) items += items_of(geoms[i], 128);
  l.table = a256(sizeof(AdrArgs) * 2 * count);
  l.work = a256(8 * items);
  l.partials = a256(8 * 3 * ns * items);
  l.rows = a256(8 * 2 * count);
  l.sums = a256(8 * 3 * ns * count);
  l.flux = a256(8 * 3 * count);
  l.step = a256(2 * sizeof(unsigned));
  l.head = l.table + l.work + l.partials + l.rows + l.sums + l.flux + l.step;
  size_t off = l.head;
  for (int i = 0; i < count; ++i) {
    const size_t pl = static_cast<size_t>(geoms[i]->nx_pad) * geoms[i]->ny;
    const size_t b = a256(ns * 9 * pl * store_b(p[0].precision));
    const size_t c = a256(ns * pl * comp_b(p[0].precision));
    const size_t r = p[0].precision == LBM_F16DEV ? a256(ns * pl * sizeof(RefT)) : 0;
    l.inst_off.push_back(off);
    l.buf.push_back(b);
    l.cprev.push_back(c);
    l.ref.push_back(r);
    off += 2 * b + c + 2 * r;
  }
  l.total = off;
  return l;
}

bool batch_args_ok(int count, const lbm_geometry *const *geoms,
                   const lbm_adr_params *p) {
  if (count < 1 || count > 32767 || !geoms || !p) return false;
  for (int i = 0; i < count; ++i) {
    if (!geoms[i] || !geoms[i]->uploaded) return false;
    if (p[i].nspecies != p[0].nspecies || p[i].precision != p[0].precision)
      return false;
    if (p[i].nspecies < 2 || p[i].nspecies > 3) return false;
    if (p[i].precision < LBM_F64 || p[i].precision > LBM_F16DEV) return false;
    for (int s = 0; s < p[i].nspecies; ++s)
      if (!(p[i].tau[s] > 0.5)) return false;
    if (geoms[i]->ny >= (1 << 24) || geoms[i]->nx_pad / 128 >= (1 << 24))
      return false;
  }
  return true;
}

cudaError_t step_launch(lbm_batch *b, int mode, int parity, cudaStream_t st) {
  switch (b->prec) {
    case LBM_F64:
      return launch_step_p<PrecF64>(b->ns, mode, b->bx, b->d_table, parity,
                                    b->d_work, b->nwork, b->d_partials, b->d_step, b->grid, st);
    case LBM_F32:
      return launch_step_p<PrecF32>(b->ns, mode, b->bx, b->d_table, parity,
                                    b->d_work, b->nwork, b->d_partials, b->d_step, b->grid, st);
    default:
      return launch_step_p<PrecF16Dev>(b->ns, mode, b->bx, b->d_table, parity,
                                       b->d_work, b->nwork, b->d_partials, b->d_step, b->grid, st);
  }
}

cudaError_t flux_launch(lbm_batch *b, int parity, cudaStream_t st) {
  switch (b->prec) {
    case LBM_F64: return launch_flux_p<PrecF64>(b->ns, b->count, b->d_table, parity, b->d_flux, st);
    case LBM_F32: return launch_flux_p<PrecF32>(b->ns, b->count, b->d_table, parity, b->d_flux, st);
    default: return launch_flux_p<PrecF16Dev>(b->ns, b->count, b->d_table, parity, b->d_flux, st);
  }
}

cudaError_t reduce_launch(lbm_batch *b, cudaStream_t st) {
  if (b->ns == 2)
    batch_reduce_kernel<2><<<b->count, kReduceThreads, 0, st>>>(b->d_partials, b->d_rows, b->d_sums);
  else
    batch_reduce_kernel<3><<<b->count, kReduceThreads, 0, st>>>(b->d_partials, b->d_rows, b->d_sums);
  return cudaGetLastError();
}

int occupancy_of(lbm_batch *b, int bx) {
  switch (b->prec) {
    case LBM_F64: return occupancy<PrecF64>(b->ns, bx);
    case LBM_F32: return occupancy<PrecF32>(b->ns, bx);
    default: return occupancy<PrecF16Dev>(b->ns, bx);
  }
}

// Work list of the active instances for tile width bx; uploads it.
cudaError_t build_work(lbm_batch *b, cudaStream_t st) {
  b->work.clear();
  b->rows.assign(2 * b->count, 0);
  for (int i = 0; i < b->count; ++i) {
    const long long lo = static_cast<long long>(b->work.size());
    if (b->active[i]) {
      const lbm_geometry *g = b->geoms[i];
      const long long nxb = (g->nx_pad + b->bx - 1) / b->bx;
      for (long long y = 0; y < g->ny; ++y)
        for (long long xb = 0; xb < nxb; ++xb) b->work.push_back(tile_item(i, y, xb));
      const long long nb = static_cast<long long>(g->bnodes.size());
      for (long long t = 0; t < nb; t += b->bx) b->work.push_back(chunk_item(i, t));
    }
    b->rows[2 * i] = lo;
    b->rows[2 * i + 1] = static_cast<long long>(b->work.size());
  }
  b->nwork = static_cast<long long>(b->work.size());
  cudaError_t e = cudaSuccess;
  if (b->nwork)
    e = cudaMemcpyAsync(b->d_work, b->work.data(), 8 * b->work.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_rows, b->rows.data(), 8 * b->rows.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

void drop_graph(lbm_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
}

// Capture one check interval: check_every - 2 plain steps, two check steps,
// the per-instance sums and the outfluxes.  check_every is even, so the
// parity is the same at the start of every interval.
cudaError_t capture_chunk(lbm_batch *b) {
  drop_graph(b);
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  int par = b->parity;
  for (int k = 0; k < b->check_every && e == cudaSuccess; ++k) {
    const int mode = (k >= b->check_every - 2) ? kAdrCheck : kAdrStep;
    e = step_launch(b, mode, par, b->cap);
    par ^= 1;
  }
  if (e == cudaSuccess) e = reduce_launch(b, b->cap);
  // the last step ran with parity par ^ 1 and wrote table[.., par ^ 1].dst
  if (e == cudaSuccess) e = flux_launch(b, par ^ 1, b->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return e;
}

lbm_status init_states(lbm_batch *b, cudaStream_t st) {
  for (int i = 0; i < b->count; ++i) {
    AdrArgs a = b->table[2 * i];
    // both population buffers and the concentration scratch (contiguous)
    const size_t bytes = static_cast<size_t>(reinterpret_cast<char *>(a.cprev) -
                                             static_cast<const char *>(a.src)) +
                         static_cast<size_t>(b->ns) * a.plane * comp_b(b->prec);
    cudaError_t e = cudaMemsetAsync(const_cast<void *>(a.src), 0, bytes, st);
    if (e == cudaSuccess) {
      a.src = nullptr;
      a.dst = const_cast<void *>(b->table[2 * i].src);  // initial state: buffer 0
      a.rsrc = nullptr;
      a.rdst = const_cast<RefT *>(b->table[2 * i].rsrc);
      switch (b->prec) {
        case LBM_F64: e = launch_adr<PrecF64>(b->ns, kAdrInit, a, st); break;
        case LBM_F32: e = launch_adr<PrecF32>(b->ns, kAdrInit, a, st); break;
        default: e = launch_adr<PrecF16Dev>(b->ns, kAdrInit, a, st); break;
      }
    }
    if (e != cudaSuccess) return bfail("lbm_batch(init)", e);
    b->steps[i] = 0;
  }
  cudaError_t e = cudaMemsetAsync(b->d_step, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return bfail("lbm_batch(init)", e);
  b->parity = 0;
  return LBM_OK;
}

}  // namespace

extern "C" size_t lbm_batch_ws_bytes(int32_t count,
                                     const lbm_geometry *const *geoms,
                                     const lbm_adr_params *params) {
  if (!batch_args_ok(count, geoms, params)) return 0;
  return batch_layout(count, geoms, params).total;
}

extern "C" lbm_status lbm_batch_create(int32_t count,
                                       const lbm_geometry *const *geoms,
                                       const lbm_adr_params *params,
                                       const void *const *u, void *ws,
                                       size_t ws_bytes, lbm_batch **out) {
  if (!out) {
    set_error("lbm_batch_create: out is NULL");
    return LBM_EINVAL;
  }
  *out = nullptr;
  if (!batch_args_ok(count, geoms, params) || !u || !ws) {
    set_error("lbm_batch_create: need 1..32767 uploaded geometries, one "
              "species count (2 or 3) and precision for all, tau > 1/2");
    return LBM_EINVAL;
  }
  for (int i = 0; i < count; ++i) {
    const int xp = params[i].x_plane < 0 ? geoms[i]->nx - 3 : params[i].x_plane;
    if (!u[i] || xp < 0 || xp >= geoms[i]->nx) {
      set_error("lbm_batch_create: missing velocity or flux plane outside");
      return LBM_EINVAL;
    }
  }
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) {
    set_error("lbm_batch_create: workspace must be 256-byte aligned");
    return LBM_EINVAL;
  }
  const BatchLayout l = batch_layout(count, geoms, params);
  if (ws_bytes < l.total) {
    set_error("lbm_batch_create: workspace too small");
    return LBM_ENOMEM;
  }
  lbm_batch *b = new (std::nothrow) lbm_batch;
  if (!b) {
    set_error("lbm_batch_create: host allocation failed");
    return LBM_ENOMEM;
  }
  char *base = static_cast<char *>(ws);
  b->count = count;
  b->ns = params[0].nspecies;
  b->prec = params[0].precision;
  b->geoms.assign(geoms, geoms + count);
  b->params.assign(params, params + count);
  b->u.assign(u, u + count);
  b->d_table = reinterpret_cast<AdrArgs *>(base);
  b->d_work = reinterpret_cast<unsigned long long *>(base + l.table);
  b->d_partials = reinterpret_cast<double *>(base + l.table + l.work);
  b->d_rows = reinterpret_cast<long long *>(base + l.table + l.work + l.partials);
  b->d_sums = reinterpret_cast<double *>(base + l.table + l.work + l.partials + l.rows);
  b->d_flux = reinterpret_cast<double *>(base + l.table + l.work + l.partials +
                                         l.rows + l.sums);
  b->d_step = reinterpret_cast<unsigned *>(base + l.table + l.work + l.partials +
                                           l.rows + l.sums + l.flux);
  b->active.assign(count, 1);
  b->steps.assign(count, 0);
  int ce = params[0].check_every < 2 ? 100 : params[0].check_every;
  b->check_every = ce + (ce & 1);
  b->table.resize(2 * count);
  for (int i = 0; i < count; ++i) {
    const lbm_geometry *g = geoms[i];
    const lbm_adr_params &p = params[i];
    AdrArgs a{};
    void *buf0 = base + l.inst_off[i];
    void *buf1 = base + l.inst_off[i] + l.buf[i];
    a.links = g->d_links;
    a.kab = g->d_kab;
    a.kbc = g->d_kbc;
    a.u = u[i];
    a.cprev = base + l.inst_off[i] + 2 * l.buf[i];
    a.partials = nullptr;
    a.bnodes = g->d_bnodes;
    a.nbnd = static_cast<long long>(g->bnodes.size());
    a.part_off = 0;
    a.plane = static_cast<long long>(g->nx_pad) * g->ny;
    a.nx = g->nx;
    a.ny = g->ny;
    a.nx_pad = g->nx_pad;
    a.abb_all = (p.flags & LBM_ADR_INLET_ABB_ALL) ? 1 : 0;
    a.nodewise = (p.flags & LBM_ADR_NODEWISE) ? 1 : 0;
    a.xp = p.x_plane < 0 ? g->nx - 3 : p.x_plane;
    for (int k = 0; k < 3; ++k) {
      const bool on = k < p.nspecies;
      a.omega[k] = on ? 1.0 / p.tau[k] : 0.0;
      a.cin[k] = on ? p.c_in[k] : 0.0;
      a.fomega[k] = static_cast<float>(a.omega[k]);
      a.fcin[k] = static_cast<float>(a.cin[k]);
    }
    RefT *ref0 = nullptr, *ref1 = nullptr;
    if (l.ref[i]) {
      char *rb = base + l.inst_off[i] + 2 * l.buf[i] + l.cprev[i];
      ref0 = reinterpret_cast<RefT *>(rb);
      ref1 = reinterpret_cast<RefT *>(rb + l.ref[i]);
    }
    a.src = buf0;
    a.dst = buf1;
    a.rsrc = ref0;
    a.rdst = ref1;
    b->table[2 * i] = a;
    a.src = buf1;
    a.dst = buf0;
    a.rsrc = ref1;
    a.rdst = ref0;
    b->table[2 * i + 1] = a;
  }
  cudaError_t e = cudaMemcpy(b->d_table, b->table.data(),
                             sizeof(AdrArgs) * b->table.size(),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return bfail("lbm_batch_create", e);
  }
  *out = b;
  return LBM_OK;
}

extern "C" void lbm_batch_destroy(lbm_batch *b) {
  if (!b) return;
  drop_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

extern "C" lbm_status lbm_batch_tune(lbm_batch *b, void *stream,
                                     int32_t *tile, int32_t *grid) {
  NvtxRange nvtx_range("lbm_batch_tune");
  if (!b) {
    set_error("lbm_batch_tune: batch is NULL");
    return LBM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  lbm_status s = init_states(b, st);
  if (s != LBM_OK) return s;
  std::fill(b->active.begin(), b->active.end(), 1);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_bx = 256;
  unsigned best_grid = 0;
  int k = 0;
  const int bxs[2] = {128, 256};
  const int mults[4] = {1, 2, 4, 8};
  for (int bx : bxs) {
    b->bx = bx;
    cudaError_t e = build_work(b, st);
    if (e != cudaSuccess) return bfail("lbm_batch_tune", e);
    const int occ = occupancy_of(b, bx);
    for (int m : mults) {
      const long long g = std::min<long long>(b->nwork,
                                              static_cast<long long>(occ) * sms * m);
      b->grid = static_cast<unsigned>(std::max<long long>(g, 1));
      // two warm-up steps, then four timed steps
      for (int r = 0; r < 2; ++r) step_launch(b, kAdrStep, r & 1, st);
      cudaEventRecord(e0, st);
      for (int r = 0; r < 4; ++r) step_launch(b, kAdrStep, r & 1, st);
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return bfail("lbm_batch_tune", e);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (k < 8) b->tune_ms[k] = ms / 4;
      ++k;
      if (ms < best) {
        best = ms;
        best_bx = bx;
        best_grid = b->grid;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->bx = best_bx;
  b->grid = best_grid;
  b->tuned = true;
  drop_graph(b);
  if (tile) *tile = best_bx;
  if (grid) *grid = static_cast<int32_t>(best_grid);
  // the timing runs advanced the states: start over
  return init_states(b, st);
}

extern "C" lbm_status lbm_batch_solve(lbm_batch *b, void *stream,
                                      lbm_solve_info *infos) {
  NvtxRange nvtx_range("lbm_batch_solve");
  if (!b || !infos) {
    set_error("lbm_batch_solve: NULL argument");
    return LBM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!b->tuned) {
    lbm_status s = lbm_batch_tune(b, stream, nullptr, nullptr);
    if (s != LBM_OK) return s;
  }
  lbm_status s = init_states(b, st);
  if (s != LBM_OK) return s;
  b->solved = true;
  std::fill(b->active.begin(), b->active.end(), 1);
  b->eps_hist.assign(3 * b->count, NAN);
  b->nhist.assign(b->count, 0);
  std::memset(infos, 0, sizeof(lbm_solve_info) * b->count);
  const int ns = b->ns;
  std::vector<double> sums(3 * ns * b->count), flux(3 * b->count);
  bool rebuild = true;
  lbm_status result = LBM_OK;
  while (true) {
    int nact = 0;
    for (char a : b->active) nact += a;
    if (nact == 0) break;
    if (rebuild) {
      cudaError_t e = build_work(b, st);
      if (e == cudaSuccess) e = capture_chunk(b);
      if (e != cudaSuccess) return bfail("lbm_batch_solve(capture)", e);
      rebuild = false;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sums.data(), b->d_sums, 8 * sums.size(),
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(flux.data(), b->d_flux, 8 * flux.size(),
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bfail("lbm_batch_solve", e);
    // check_every is even: the parity at the start of the next chunk is
    // unchanged
    for (int i = 0; i < b->count; ++i) {
      if (!b->active[i]) continue;
      b->steps[i] += b->check_every;
      lbm_solve_info &inf = infos[i];
      inf.steps = b->steps[i];
      const lbm_adr_params &p = b->params[i];
      const double *row = &sums[(size_t)i * 3 * ns];
      double r = 0.0;
      bool finite = true;
      for (int k = 0; k < ns; ++k) {
        const double num = row[2 * k], den = row[2 * k + 1];
        finite = finite && std::isfinite(num) && std::isfinite(den);
        if (den > 0) r = std::fmax(r, num / den);
        inf.flux[k] = flux[(size_t)i * 3 + k];
        finite = finite && std::isfinite(inf.flux[k]);
        inf.c_min[k] = row[2 * ns + k];
        inf.mass[k] = den;
      }
      inf.residual = finite ? r : NAN;
      double eps = 0.0;
      if (lbm_efficiency(inf.flux, ns, &eps) == LBM_OK) inf.eps = eps;
      const bool negative = finite && adr_negative(&p, inf.c_min);
      double *eh = &b->eps_hist[3 * (size_t)i];
      eh[0] = eh[1];
      eh[1] = eh[2];
      eh[2] = inf.eps;
      ++b->nhist[i];
      bool conv = finite && !negative && (p.tol > 0 || p.eps_tol > 0) &&
                  (p.tol <= 0 || r < p.tol);
      if (conv && p.eps_tol > 0)
        conv = b->nhist[i] >= 3 &&
               eps_distance(eh[0], eh[1], eh[2], 0.1 * p.eps_tol) < p.eps_tol;
      inf.converged = conv ? 1 : 0;
      if (!finite) {
        result = LBM_EUNSTABLE;
        set_error("lbm_batch_solve: non-finite sums in instance " + std::to_string(i));
      } else if (negative) {
        result = LBM_EUNSTABLE;
        set_error("lbm_batch_solve: instance " + std::to_string(i) +
                  " has a concentration below -neg_tol at step " +
                  std::to_string(b->steps[i]));
      }
      if (conv || !finite || negative || b->steps[i] >= p.max_steps) {
        b->active[i] = 0;
        rebuild = true;
        if (!conv && finite && !negative && (p.tol > 0 || p.eps_tol > 0) &&
            result == LBM_OK)
          result = LBM_ENOTCONVERGED;
      }
    }
  }
  return result;
}

extern "C" lbm_status lbm_batch_tuning(const lbm_batch *b, int32_t *tile,
                                       int32_t *grid, float *ms_per_step) {
  if (!b) {
    set_error("lbm_batch_tuning: batch is NULL");
    return LBM_EINVAL;
  }
  if (tile) *tile = b->bx;
  if (grid) *grid = static_cast<int32_t>(b->grid);
  if (ms_per_step)
    for (int k = 0; k < 8; ++k) ms_per_step[k] = b->tune_ms[k];
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_conc(const lbm_batch *b, int32_t index,
                                     void *conc_out, void *stream) {
  if (!b || !conc_out || index < 0 || index >= b->count) {
    set_error("lbm_batch_conc: NULL argument or index outside the batch");
    return LBM_EINVAL;
  }
  if (!b->solved) {
    set_error("lbm_batch_conc: no solve has run on this batch");
    return LBM_EINVAL;
  }
  const AdrArgs &a = b->table[2 * index];
  const size_t bytes = static_cast<size_t>(b->ns) * static_cast<size_t>(a.plane) *
                       comp_b(b->prec);
  cudaError_t e = cudaMemcpyAsync(conc_out, a.cprev, bytes, cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return bfail("lbm_batch_conc", e);
  return LBM_OK;
}
