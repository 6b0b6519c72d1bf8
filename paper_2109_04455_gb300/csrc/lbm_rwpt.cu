// Random walk particle tracking (RWPT) of the paper's Sec. III.B: the second,
// independent method for the reaction efficiency of a 2D cross-section.
//
// Each particle (species A, B or C) moves per time step dt by
//   advection  x += dt u(x), u bilinear in the LBM velocity field,
//   diffusion  x += sqrt(4 D dt) (cos t, sin t), t uniform,
// reflects elastically off the channel walls and the fibers, reacts with
// probability k dt per step while within a reactive shell of width delta
// around a catalytic fiber (A -> B at rate k_AB, B -> C at rate k_BC), and
// is counted per species when it leaves through the outlet.  The entrance
// strip x in [-1/2, 1/2) is held at a fixed density of A: every step the A
// particles that ended there are removed and the strip is seeded anew.
//
// Random numbers: draw k of particle `id` at step t is the (64 t + k + 1)-th
// output of the particle's SplitMix64 stream (Steele, Lea and Flood, OOPSLA
// 2014), whose seed is output id + 1 of the stream of the run's seed.  A
// particle's path thus depends only on (seed, id), not on where it is
// stored.  The direction is drawn by rejection from the unit disc, and every
// floating-point step is an IEEE operation with one rounding (explicit
// round-to-nearest intrinsics, no contraction), so a plain CPU restatement
// of the same steps reproduces every position bit for bit.
//
// Storage: structure of arrays in two buffers (ping-pong); a step compacts
// the survivors of one buffer into the other (warp ballots, one atomic per
// warp) and appends the new entrance particles.  Counts live on the device,
// so steps need no host synchronisation.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"
#include "lbm_nvtx.h"

namespace lbm {
namespace rwpt {

constexpr unsigned long long kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kDraws = 64;       // draws reserved per particle and step
constexpr int kTries = 16;       // direction candidates (2 draws each)
constexpr int kReactDraw = 40;   // draw index of the reaction test
constexpr int kSpawnDraw = 48;   // draws of a new particle's position
constexpr int kReflections = 4;  // reflection passes per step
constexpr int kThreads = 256;

__host__ __device__ inline unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ inline unsigned long long particle_seed(unsigned long long seed,
                                                   unsigned long long id) {
  return mix64(seed + (id + 1ull) * kGamma);
}
// uniform double in [0, 1): the top 53 bits of the draw
__device__ inline double draw(unsigned long long ps, long long t, int k) {
  const unsigned long long c =
      static_cast<unsigned long long>(t) * kDraws + static_cast<unsigned>(k) + 1ull;
  return static_cast<double>(mix64(ps + c * kGamma) >> 11) * 0x1.0p-53;
}

// a fiber as the particles see it
struct Fiber {
  double cx, cy;
  double rp;      // reflecting radius
  double kab, kbc;
  double nx, ny;  // side-by-side fiber: A -> B where (p - c).n >= 0
  int split;      // 1: side-by-side (rates by side), 0: rates everywhere
  int pad;
};

struct Args {
  int nx, ny, nx_pad, nfib;
  int nspecies;
  int periodic;      // box periodic in x and y: no inlet, outlet or walls
  int homogeneous;   // every particle reacts, wherever it is
  int pad;
  double dt, len, delta;   // time step, diffusion step length, shell width
  double hk1, hk2;         // homogeneous rates (A -> B, B -> C)
  unsigned long long seed;
  const double *u;         // [2][ny][nx_pad]
  const Fiber *fib;
};

struct Buf {
  double *x, *y;
  unsigned long long *id;
  int *s;
};

// Counters (device, unsigned long long): the particle count of each buffer,
// the outflow of each species since the last reset, the overflow flag.  A
// buffer's count can pass the capacity when particles are dropped for lack
// of room (the appends count them, the slots refuse them), so every reader
// takes min(count, capacity).
enum { kCount0 = 0, kCount1 = 1, kOut = 2, kOverflow = 5, kCounters = 8 };

__device__ inline double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ inline double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ inline double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ inline double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// u at (px, py): bilinear in the four nodes around the point (node indices
// clamped to the lattice)
__device__ inline void velocity(const Args &a, double px, double py,
                                double &ux, double &uy) {
  const double fx0 = floor(px), fy0 = floor(py);
  const double fx = dsub(px, fx0), fy = dsub(py, fy0);
  int i0 = static_cast<int>(fx0), j0 = static_cast<int>(fy0);
  int i1 = i0 + 1, j1 = j0 + 1;
  i0 = min(max(i0, 0), a.nx - 1);
  i1 = min(max(i1, 0), a.nx - 1);
  j0 = min(max(j0, 0), a.ny - 1);
  j1 = min(max(j1, 0), a.ny - 1);
  const double gx = dsub(1.0, fx), gy = dsub(1.0, fy);
  const double w00 = dmul(gx, gy), w10 = dmul(fx, gy);
  const double w01 = dmul(gx, fy), w11 = dmul(fx, fy);
  const long long plane = static_cast<long long>(a.nx_pad) * a.ny;
  const long long n00 = static_cast<long long>(j0) * a.nx_pad + i0;
  const long long n10 = static_cast<long long>(j0) * a.nx_pad + i1;
  const long long n01 = static_cast<long long>(j1) * a.nx_pad + i0;
  const long long n11 = static_cast<long long>(j1) * a.nx_pad + i1;
  ux = dadd(dadd(dadd(dmul(w00, a.u[n00]), dmul(w10, a.u[n10])),
                 dmul(w01, a.u[n01])), dmul(w11, a.u[n11]));
  uy = dadd(dadd(dadd(dmul(w00, a.u[plane + n00]), dmul(w10, a.u[plane + n10])),
                 dmul(w01, a.u[plane + n01])), dmul(w11, a.u[plane + n11]));
}

// Mirror p at the circle of radius rp about c if p is inside it:
// the distance to the centre d becomes 2 rp - d along the same ray.
__device__ inline bool reflect_fiber(const Fiber &f, double &px, double &py) {
  const double dx = dsub(px, f.cx), dy = dsub(py, f.cy);
  const double d2 = dadd(dmul(dx, dx), dmul(dy, dy));
  const double r2 = dmul(f.rp, f.rp);
  if (!(d2 < r2)) return false;
  if (d2 == 0.0) {   // at the centre: out along +x
    px = dadd(f.cx, f.rp);
    return true;
  }
  const double d = __dsqrt_rn(d2);
  const double q = ddiv(dsub(dmul(2.0, f.rp), d), d);
  px = dadd(f.cx, dmul(q, dx));
  py = dadd(f.cy, dmul(q, dy));
  return true;
}

__device__ inline double wrap(double v, double lo, double span) {
  // v in [lo - span, lo + 2 span): back into [lo, lo + span)
  if (v < lo) return dadd(v, span);
  if (!(v < dadd(lo, span))) return dsub(v, span);
  return v;
}

// The rate that applies to a particle of species s at (px, py), or 0: the
// first fiber (list order) whose shell rp <= d < rp + delta holds the point
// and whose catalyst acts on s.
__device__ inline double shell_rate(const Args &a, int s, double px,
                                    double py) {
  if (a.homogeneous) return s == 0 ? a.hk1 : (s == 1 ? a.hk2 : 0.0);
  for (int j = 0; j < a.nfib; ++j) {
    const Fiber &f = a.fib[j];
    const double dx = dsub(px, f.cx), dy = dsub(py, f.cy);
    const double d2 = dadd(dmul(dx, dx), dmul(dy, dy));
    const double ro = dadd(f.rp, a.delta);
    if (!(d2 >= dmul(f.rp, f.rp)) || !(d2 < dmul(ro, ro))) continue;
    double kab = f.kab, kbc = f.kbc;
    if (f.split) {
      const bool first = dadd(dmul(dx, f.nx), dmul(dy, f.ny)) >= 0.0;
      kab = first ? f.kab : 0.0;
      kbc = first ? 0.0 : f.kbc;
    }
    const double k = s == 0 ? kab : (s == 1 ? kbc : 0.0);
    if (k > 0.0) return k;
  }
  return 0.0;
}

// Append the kept lanes of a warp to `out` (count in *cnt): one atomic per
// warp.  Returns this lane's slot (or -1), -2 if the buffer is full.
__device__ inline long long warp_slot(bool keep, unsigned long long *cnt,
                                      long long cap, unsigned long long *overflow) {
  const unsigned mask = __ballot_sync(0xffffffffu, keep);
  const int lane = threadIdx.x & 31;
  const int leader = mask ? __ffs(mask) - 1 : 0;
  unsigned long long base = 0;
  if (mask && lane == leader) base = atomicAdd(cnt, static_cast<unsigned long long>(__popc(mask)));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (!keep) return -1;
  const long long slot =
      static_cast<long long>(base) + __popc(mask & ((1u << lane) - 1u));
  if (slot >= cap) {
    atomicExch(overflow, 1ull);
    return -2;
  }
  return slot;
}

// One time step of every particle of `in` (count in cnt[kin]); survivors go
// to `out` (count in cnt[kout], zero on entry).
__global__ void __launch_bounds__(kThreads)
    rwpt_step_kernel(const Args a, Buf in, Buf out, unsigned long long *cnt,
                     int kin, int kout, long long cap, long long t) {
  const long long n = min(static_cast<long long>(cnt[kin]), cap);
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x; base < n;
       base += stride) {
    const long long i = base + threadIdx.x;
    bool keep = i < n;
    int outflow = -1;
    double px = 0.0, py = 0.0;
    int s = 0;
    unsigned long long id = 0;
    if (keep) {
      px = in.x[i];
      py = in.y[i];
      s = in.s[i];
      id = in.id[i];
      const unsigned long long ps = particle_seed(a.seed, id);
      // advection (Euler)
      if (a.u != nullptr) {
        double ux, uy;
        velocity(a, px, py, ux, uy);
        px = dadd(px, dmul(a.dt, ux));
        py = dadd(py, dmul(a.dt, uy));
      }
      // diffusion: a step of length sqrt(4 D dt) in a uniform direction
      if (a.len > 0.0) {
        double v1 = 1.0, v2 = 0.0, q = 1.0;
        for (int k = 0; k < kTries; ++k) {
          const double c1 = dsub(dmul(2.0, draw(ps, t, 2 * k)), 1.0);
          const double c2 = dsub(dmul(2.0, draw(ps, t, 2 * k + 1)), 1.0);
          const double q2 = dadd(dmul(c1, c1), dmul(c2, c2));
          if (q2 > 0.0 && q2 <= 1.0) {
            v1 = c1;
            v2 = c2;
            q = q2;
            break;
          }
        }
        const double r = __dsqrt_rn(q);
        px = dadd(px, ddiv(dmul(a.len, v1), r));
        py = dadd(py, ddiv(dmul(a.len, v2), r));
      }
      // elastic reflections: walls y = -1/2, ny - 1/2 and the fibers
      const double ytop = dsub(static_cast<double>(a.ny), 0.5);
      for (int pass = 0; pass < kReflections; ++pass) {
        bool hit = false;
        if (a.periodic) {
          px = wrap(px, -0.5, static_cast<double>(a.nx));
          py = wrap(py, -0.5, static_cast<double>(a.ny));
        } else {
          if (py < -0.5) {
            py = dsub(-1.0, py);
            hit = true;
          } else if (py > ytop) {
            py = dsub(dmul(2.0, ytop), py);
            hit = true;
          }
        }
        for (int k = 0; k < a.nfib; ++k) hit = reflect_fiber(a.fib[k], px, py) || hit;
        if (!hit) break;
      }
      // reaction with probability k dt
      if (s < a.nspecies - 1) {
        const double k = shell_rate(a, s, px, py);
        if (k > 0.0 && draw(ps, t, kReactDraw) < dmul(k, a.dt)) s += 1;
      }
      // inlet and outlet
      if (!a.periodic) {
        const double xout = dsub(static_cast<double>(a.nx), 0.5);
        if (!(px < xout)) {
          outflow = s;
          keep = false;
        } else if (px < -0.5) {
          if (s == 0)
            keep = false;          // back into the reservoir of A
          else
            px = dsub(-1.0, px);   // B and C: the entrance reflects
        }
        if (keep && s == 0 && px < 0.5) keep = false;  // strip: re-seeded
      }
    }
    // outflow counts (one atomic per warp and species)
#pragma unroll
    for (int sp = 0; sp < 3; ++sp) {
      const unsigned m = __ballot_sync(0xffffffffu, outflow == sp);
      if (m && (threadIdx.x & 31) == __ffs(m) - 1)
        atomicAdd(cnt + kOut + sp, static_cast<unsigned long long>(__popc(m)));
    }
    const long long slot = warp_slot(keep, cnt + kout, cap, cnt + kOverflow);
    if (slot >= 0) {
      out.x[slot] = px;
      out.y[slot] = py;
      out.s[slot] = s;
      out.id[slot] = id;
    }
  }
}

// New particles of species A with ids id0 .. id0 + m - 1, uniform in the
// rectangle [x0, x0 + wx) x [-1/2, ny - 1/2), those inside a fiber dropped,
// appended to `out`.
__global__ void __launch_bounds__(kThreads)
    rwpt_spawn_kernel(const Args a, Buf out, unsigned long long *cnt, int kout,
                      long long cap, long long t, unsigned long long id0,
                      long long m, double x0, double wx) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x; base < m;
       base += stride) {
    const long long j = base + threadIdx.x;
    bool keep = j < m;
    double px = 0.0, py = 0.0;
    const unsigned long long id = id0 + static_cast<unsigned long long>(j);
    if (keep) {
      const unsigned long long ps = particle_seed(a.seed, id);
      px = dadd(x0, dmul(wx, draw(ps, t, kSpawnDraw)));
      py = dadd(-0.5, dmul(static_cast<double>(a.ny), draw(ps, t, kSpawnDraw + 1)));
      for (int k = 0; k < a.nfib && keep; ++k) {
        const Fiber &f = a.fib[k];
        const double dx = dsub(px, f.cx), dy = dsub(py, f.cy);
        if (dadd(dmul(dx, dx), dmul(dy, dy)) < dmul(f.rp, f.rp)) keep = false;
      }
    }
    const long long slot = warp_slot(keep, cnt + kout, cap, cnt + kOverflow);
    if (slot >= 0) {
      out.x[slot] = px;
      out.y[slot] = py;
      out.s[slot] = 0;
      out.id[slot] = id;
    }
  }
}

inline size_t a256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace rwpt
}  // namespace lbm

using namespace lbm;
using namespace lbm::rwpt;

struct lbm_rwpt {
  Args a{};
  lbm_rwpt_params p{};
  int nx = 0, ny = 0;
  long long cap = 0;
  Buf buf[2];
  unsigned long long *cnt = nullptr;
  int cur = 0;                 // buffer holding the current particles
  long long steps = 0, window = 0;
  unsigned long long next_id = 0;
  long long seed_count = 0;    // entrance particles per step
  int grid = 0;
  bool started = false;
};

namespace {

struct RwptLayout {
  size_t xy, id, s, fib, cnt, total;
};
RwptLayout rwpt_layout(long long cap, int nfib) {
  RwptLayout l{};
  l.xy = a256(8 * static_cast<size_t>(cap));
  l.id = a256(8 * static_cast<size_t>(cap));
  l.s = a256(4 * static_cast<size_t>(cap));
  l.fib = a256(sizeof(Fiber) * static_cast<size_t>(nfib > 0 ? nfib : 1));
  l.cnt = a256(8 * kCounters);
  l.total = 2 * (2 * l.xy + l.id + l.s) + l.fib + l.cnt;
  return l;
}

lbm_status rfail(const char *where, cudaError_t e) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return LBM_ECUDA;
}

}  // namespace

extern "C" size_t lbm_rwpt_ws_bytes(int64_t capacity, int32_t nfibers) {
  if (capacity < 1 || nfibers < 0) return 0;
  return rwpt_layout(capacity, nfibers).total;
}

extern "C" lbm_status lbm_rwpt_create(int32_t nx, int32_t ny,
                                      const double *fibers, int32_t nfibers,
                                      double k1, double k2,
                                      const lbm_rwpt_params *p, const void *u,
                                      int64_t capacity, void *ws,
                                      size_t ws_bytes, lbm_rwpt **out) {
  if (!out) {
    set_error("lbm_rwpt_create: out is NULL");
    return LBM_EINVAL;
  }
  *out = nullptr;
  if (!p || !ws || nx < 2 || ny < 1 || nfibers < 0 || (nfibers > 0 && !fibers) ||
      capacity < 1) {
    set_error("lbm_rwpt_create: NULL argument, nx < 2, ny < 1 or capacity < 1");
    return LBM_EINVAL;
  }
  const bool periodic = (p->flags & LBM_RWPT_PERIODIC) != 0;
  if (!(p->dt > 0.0) || !(p->D >= 0.0) || !(p->delta >= 0.0) ||
      !(p->density >= 0.0) || p->nspecies < 1 || p->nspecies > 3 ||
      !(k1 >= 0.0) || !(k2 >= 0.0) || k1 * p->dt > 1.0 || k2 * p->dt > 1.0 ||
      (p->flags & ~(LBM_RWPT_PERIODIC | LBM_RWPT_HOMOGENEOUS))) {
    set_error("lbm_rwpt_create: need dt > 0, D, delta, density >= 0, 1..3 "
              "species, 0 <= k dt <= 1, known flags");
    return LBM_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0 ||
      (u && (reinterpret_cast<uintptr_t>(u) & 7u) != 0)) {
    set_error("lbm_rwpt_create: workspace not 256-byte aligned");
    return LBM_EINVAL;
  }
  const RwptLayout l = rwpt_layout(capacity, nfibers);
  if (ws_bytes < l.total) {
    set_error("lbm_rwpt_create: workspace too small");
    return LBM_ENOMEM;
  }
  std::vector<Fiber> fib(static_cast<size_t>(nfibers));
  for (int f = 0; f < nfibers; ++f) {
    const double *r = fibers + 6 * static_cast<int64_t>(f);
    const int cat = static_cast<int>(r[3]);
    if (!(r[2] >= 0.0) || cat < 0 || cat > 3) {
      set_error("lbm_rwpt_create: bad fiber row " + std::to_string(f));
      return LBM_EINVAL;
    }
    Fiber &q = fib[f];
    q.cx = r[0];
    q.cy = r[1];
    q.rp = r[2] + p->radius_offset;
    q.split = 0;
    q.kab = q.kbc = 0.0;
    if (cat != 0 && r[5] >= 0.0) {
      q.kab = r[5] * k1;
      q.kbc = (1.0 - r[5]) * k2;
    } else if (cat == 1) {
      q.kab = k1;
    } else if (cat == 2) {
      q.kbc = k2;
    } else if (cat == 3) {
      q.kab = k1;
      q.kbc = k2;
      q.split = 1;
      q.nx = std::cos(r[4]);
      q.ny = std::sin(r[4]);
    }
  }
  lbm_rwpt *r = new (std::nothrow) lbm_rwpt;
  if (!r) {
    set_error("lbm_rwpt_create: host allocation failed");
    return LBM_ENOMEM;
  }
  char *b = static_cast<char *>(ws);
  for (int k = 0; k < 2; ++k) {
    char *o = b + k * (2 * l.xy + l.id + l.s);
    r->buf[k].x = reinterpret_cast<double *>(o);
    r->buf[k].y = reinterpret_cast<double *>(o + l.xy);
    r->buf[k].id = reinterpret_cast<unsigned long long *>(o + 2 * l.xy);
    r->buf[k].s = reinterpret_cast<int *>(o + 2 * l.xy + l.id);
  }
  Fiber *d_fib = reinterpret_cast<Fiber *>(b + 2 * (2 * l.xy + l.id + l.s));
  r->cnt = reinterpret_cast<unsigned long long *>(b + 2 * (2 * l.xy + l.id + l.s) + l.fib);
  r->p = *p;
  r->nx = nx;
  r->ny = ny;
  r->cap = capacity;
  Args &a = r->a;
  a.nx = nx;
  a.ny = ny;
  a.nx_pad = static_cast<int>(pad32(nx));
  a.nfib = nfibers;
  a.nspecies = p->nspecies;
  a.periodic = periodic ? 1 : 0;
  a.homogeneous = (p->flags & LBM_RWPT_HOMOGENEOUS) ? 1 : 0;
  a.dt = p->dt;
  a.len = std::sqrt(4.0 * p->D * p->dt);
  a.delta = p->delta;
  a.hk1 = k1;
  a.hk2 = k2;
  a.seed = p->seed;
  a.u = static_cast<const double *>(u);
  a.fib = d_fib;
  r->seed_count = periodic ? 0 : static_cast<long long>(std::llround(p->density * ny));
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  r->grid = 8 * sms;
  cudaError_t e = cudaSuccess;
  if (nfibers > 0)
    e = cudaMemcpy(d_fib, fib.data(), sizeof(Fiber) * fib.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete r;
    return rfail("lbm_rwpt_create", e);
  }
  *out = r;
  return LBM_OK;
}

extern "C" void lbm_rwpt_destroy(lbm_rwpt *r) { delete r; }

extern "C" lbm_status lbm_rwpt_init(lbm_rwpt *r, void *stream) {
  NvtxRange nvtx_range("lbm_rwpt_init");
  if (!r) {
    set_error("lbm_rwpt_init: NULL argument");
    return LBM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(r->cnt, 0, 8 * kCounters, st);
  r->cur = 0;
  r->steps = 0;
  r->window = 0;
  r->next_id = 0;
  // the start: A at the density over the whole box (the fluid part of it)
  const long long m = std::llround(r->p.density * static_cast<double>(r->nx) * r->ny);
  if (e == cudaSuccess && m > 0) {
    rwpt_spawn_kernel<<<r->grid, kThreads, 0, st>>>(
        r->a, r->buf[0], r->cnt, kCount0, r->cap, -1, 0ull, m, -0.5,
        static_cast<double>(r->nx));
    e = cudaGetLastError();
  }
  r->next_id = static_cast<unsigned long long>(m);
  if (e != cudaSuccess) return rfail("lbm_rwpt_init", e);
  r->started = true;
  return LBM_OK;
}

extern "C" lbm_status lbm_rwpt_run(lbm_rwpt *r, int64_t nsteps, void *stream,
                                   lbm_rwpt_info *info) {
  NvtxRange nvtx_range("lbm_rwpt_run");
  if (!r || nsteps < 0 || !r->started) {
    set_error("lbm_rwpt_run: NULL solver, nsteps < 0 or not initialised");
    return LBM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
    const int kin = kCount0 + r->cur, kout = kCount0 + (r->cur ^ 1);
    e = cudaMemsetAsync(r->cnt + kout, 0, 8, st);
    if (e != cudaSuccess) break;
    rwpt_step_kernel<<<r->grid, kThreads, 0, st>>>(r->a, r->buf[r->cur],
                                                   r->buf[r->cur ^ 1], r->cnt,
                                                   kin, kout, r->cap, r->steps);
    if (r->seed_count > 0)
      rwpt_spawn_kernel<<<r->grid, kThreads, 0, st>>>(
          r->a, r->buf[r->cur ^ 1], r->cnt, kout, r->cap, r->steps, r->next_id,
          r->seed_count, -0.5, 1.0);
    e = cudaGetLastError();
    r->next_id += static_cast<unsigned long long>(r->seed_count);
    r->cur ^= 1;
    ++r->steps;
    ++r->window;
  }
  if (e != cudaSuccess) return rfail("lbm_rwpt_run", e);
  if (!info) return LBM_OK;
  unsigned long long h[kCounters] = {0};
  e = cudaMemcpyAsync(h, r->cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rfail("lbm_rwpt_run", e);
  std::memset(info, 0, sizeof(*info));
  info->steps = r->steps;
  info->window_steps = r->window;
  info->alive = static_cast<int64_t>(h[kCount0 + r->cur]) < r->cap
                    ? static_cast<int64_t>(h[kCount0 + r->cur])
                    : r->cap;
  for (int s = 0; s < 3; ++s) info->out[s] = static_cast<int64_t>(h[kOut + s]);
  info->overflow = h[kOverflow] ? 1 : 0;
  const int ns = r->p.nspecies;
  double f[3] = {double(h[kOut]), double(h[kOut + 1]), double(h[kOut + 2])};
  if (ns >= 2) {
    double eps = 0.0;
    if (lbm_efficiency(f, ns, &eps) == LBM_OK) info->eps = eps;
  }
  if (info->overflow) {
    set_error("lbm_rwpt_run: particle capacity exceeded (particles were lost)");
    return LBM_ENOMEM;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_rwpt_reset_counts(lbm_rwpt *r, void *stream) {
  if (!r) {
    set_error("lbm_rwpt_reset_counts: NULL argument");
    return LBM_EINVAL;
  }
  cudaError_t e = cudaMemsetAsync(r->cnt + kOut, 0, 8 * 3,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return rfail("lbm_rwpt_reset_counts", e);
  r->window = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_rwpt_particles(lbm_rwpt *r, void *stream,
                                         int64_t max_count, int64_t *count,
                                         double *x, double *y, int32_t *species,
                                         uint64_t *id) {
  if (!r || !count || !x || !y || !species || !id) {
    set_error("lbm_rwpt_particles: NULL argument");
    return LBM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long n = 0;
  cudaError_t e = cudaMemcpyAsync(&n, r->cnt + kCount0 + r->cur, 8,
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rfail("lbm_rwpt_particles", e);
  if (static_cast<long long>(n) > r->cap) n = static_cast<unsigned long long>(r->cap);
  *count = static_cast<int64_t>(n);
  if (static_cast<long long>(n) > max_count) {
    set_error("lbm_rwpt_particles: host arrays shorter than the particle count");
    return LBM_ENOMEM;
  }
  const Buf &b = r->buf[r->cur];
  e = cudaMemcpyAsync(x, b.x, 8 * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(y, b.y, 8 * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(species, b.s, 4 * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(id, b.id, 8 * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rfail("lbm_rwpt_particles", e);
  return LBM_OK;
}
