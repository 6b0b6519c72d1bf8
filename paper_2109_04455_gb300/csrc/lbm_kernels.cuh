// sm_103a kernels of liblbm: fused pull stream-collide for the flow lattice
// and for all ADR species at once, plus the outflux and residual reductions.
//
// Data layout in HBM (structure of arrays, x contiguous):
//   populations  [species][q][ny][nx_pad]   (two buffers, ping-pong)
//   link words   [ny][nx_pad]  uint32, nibble j-1 = type of neighbour x+c_j
//   rates        k_AB, k_BC [ny][nx_pad] double (read on catalytic links only)
//   velocity     [2][ny][nx_pad]
// One thread owns one node; a block covers kBlockX consecutive nodes of one
// row, so every population plane is read and written with coalesced
// accesses (the pull of a plane is a pure shift: each element of the source
// plane is read exactly once per step).
//
// The path is bandwidth bound (about 1 flop per byte in float), so there are
// no tensor-core contractions here; what matters is bytes per node update.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm_internal.h"

namespace lbm {

constexpr int kBlockX = 128;      // threads per block (one row segment)
constexpr int kReduceThreads = 256;

// ---------------------------------------------------------------------------
// precision traits: storage type S, compute type T
// ---------------------------------------------------------------------------
struct PrecF64 {
  using S = double;
  using T = double;
  static constexpr bool kDev = false;
  static __device__ __forceinline__ T load(S v) { return v; }
  static __device__ __forceinline__ S store(T v) { return v; }
};
struct PrecF32 {
  using S = float;
  using T = float;
  static constexpr bool kDev = false;
  static __device__ __forceinline__ T load(S v) { return v; }
  static __device__ __forceinline__ S store(T v) { return v; }
};
// half storage of the deviation g - w_i c_ref (round to nearest even)
struct PrecF16Dev {
  using S = __half;
  using T = float;
  static constexpr bool kDev = true;
  static __device__ __forceinline__ T load(S v) { return __half2float(v); }
  static __device__ __forceinline__ S store(T v) { return __float2half_rn(v); }
};

template <typename T>
struct Lattice {
  static __device__ __forceinline__ T w(int i) {
    return i == 0 ? T(4) / T(9) : (i < 5 ? T(1) / T(9) : T(1) / T(36));
  }
};

__device__ __forceinline__ constexpr int cx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ constexpr int cy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4 + 1) : ((i - 5 + 2) % 4 + 5));
}
__device__ __forceinline__ uint32_t nib(uint32_t word, int j) {
  return (word >> (4 * (j - 1))) & 0xFu;
}

// ---------------------------------------------------------------------------
// deterministic block reduction of K doubles (fixed order for a fixed block
// size); result valid in thread 0
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double red[32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w][k];
      v[k] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// ADR
// ---------------------------------------------------------------------------
struct AdrArgs {
  const void *src;          // S [ns][9][plane]  post-collision at time t
  void *dst;                // S [ns][9][plane]  post-collision at time t+1
  const uint32_t *links;    // [plane]
  const double *kab, *kbc;  // [plane]
  const void *u;            // T [2][plane]
  void *cprev;              // T [ns][plane]     (check steps)
  double *partials;         // [nblocks][2*ns]   (check steps)
  long long plane;          // ny * nx_pad
  int nx, ny, nx_pad;
  int abb_all;              // anti-bounce-back inlet for every species
  double omega[3];          // 1/tau per species
  double cin[3];            // inlet concentration per species
  double cref[3];           // reference concentration of the stored deviation
};

enum AdrMode { kAdrStep = 0, kAdrCheck = 1, kAdrInit = 2 };

template <class P, int NS, int MODE>
__global__ void __launch_bounds__(kBlockX) adr_kernel(const AdrArgs a) {
  using S = typename P::S;
  using T = typename P::T;
  const int x = blockIdx.x * kBlockX + threadIdx.x;
  const int y = blockIdx.y;
  const long long n = (long long)y * a.nx_pad + x;
  const long long plane = a.plane;
  const uint32_t lw = (x < a.nx_pad) ? a.links[n] : kSolidNode;
  double acc[2 * NS];
#pragma unroll
  for (int k = 0; k < 2 * NS; ++k) acc[k] = 0.0;

  if (lw != kSolidNode) {
    const S *__restrict__ src = static_cast<const S *>(a.src);
    S *__restrict__ dst = static_cast<S *>(a.dst);
    const T *__restrict__ U = static_cast<const T *>(a.u);
    const T ux = U[n], uy = U[plane + n];
    const long long np = (long long)a.nx_pad;

    // shift of the stored deviation
    auto shift = [&](int s, int i) -> T {
      return P::kDev ? Lattice<T>::w(i) * T(a.cref[s]) : T(0);
    };
    auto ld = [&](int s, int i, long long m) -> T {
      return P::load(src[(long long)(s * 9 + i) * plane + m]) + shift(s, i);
    };

    // equilibrium factors E_i(u), shared by every species:
    // g_i^eq = C * E_i, E_i = w_i (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u)
    T E[9];
    {
      const T uu = ux * ux + uy * uy;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const T cu = T(cx(i)) * ux + T(cy(i)) * uy;
        E[i] = Lattice<T>::w(i) *
               (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
      }
    }

    T g[NS][9];
    if (MODE == kAdrInit) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const T c0 = (s == 0) ? T(1) : T(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) g[s][i] = c0 * E[i];
      }
    } else if (lw == 0u) {
      // interior node: every population streams from a fluid neighbour
#pragma unroll
      for (int s = 0; s < NS; ++s) {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[s][i] = ld(s, i, n - (cy(i) * np + cx(i)));
      }
    } else {
      // boundary node: pull or apply the rule of the source's link type
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        T cb = T(0);
        if (x == a.nx - 1) {
#pragma unroll
          for (int j = 0; j < 9; ++j) cb += ld(s, j, n);
        }
        g[s][0] = ld(s, 0, n);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
          const uint32_t t = nib(lw, opp(i));
          if (t == kFluid) {
            g[s][i] = ld(s, i, n - (cy(i) * np + cx(i)));
          } else if (t == kInlet) {
            const T back = ld(s, opp(i), n);
            g[s][i] = (s == 0 || a.abb_all)
                          ? -back + T(2) * Lattice<T>::w(i) * T(a.cin[s])
                          : back;
          } else if (t == kOutlet) {
            g[s][i] = -ld(s, opp(i), n) + T(2) * Lattice<T>::w(i) * cb;
          } else {  // wall, inert or catalytic fiber: bounce-back
            g[s][i] = ld(s, opp(i), n);
          }
        }
      }
    }

    // concentrations and BGK collision
    T C[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      T c = T(0);
#pragma unroll
      for (int i = 0; i < 9; ++i) c += g[s][i];
      C[s] = c;
      const T om = T(a.omega[s]);
#pragma unroll
      for (int i = 0; i < 9; ++i) g[s][i] = g[s][i] + om * (c * E[i] - g[s][i]);
    }

    // Dawson source on links into catalytic fiber nodes
    if (lw != 0u) {
#pragma unroll
      for (int j = 1; j < 9; ++j) {
        if (nib(lw, j) == kCat) {
          const long long m = n + cy(j) * np + cx(j);
          const T wj = Lattice<T>::w(j);
          const T ra = T(a.kab[m]) * wj * C[0];
          const T rb = (NS >= 3) ? T(a.kbc[m]) * wj * C[NS >= 2 ? 1 : 0] : T(0);
          g[0][j] -= ra;
          if (NS >= 2) g[NS >= 2 ? 1 : 0][j] += ra - rb;
          if (NS >= 3) g[NS >= 3 ? 2 : 0][j] += rb;
        }
      }
    }

#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int i = 0; i < 9; ++i)
        dst[(long long)(s * 9 + i) * plane + n] = P::store(g[s][i] - shift(s, i));
    }

    if (MODE == kAdrCheck) {
      T *cp = static_cast<T *>(a.cprev);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const T prev = cp[s * plane + n];
        acc[2 * s] = fabs(double(C[s]) - double(prev));
        acc[2 * s + 1] = fabs(double(C[s]));
        cp[s * plane + n] = C[s];
      }
    }
  }

  if (MODE == kAdrCheck) {
    block_sum<2 * NS>(acc);
    if (threadIdx.x == 0) {
      const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
      for (int k = 0; k < 2 * NS; ++k) a.partials[b * (2 * NS) + k] = acc[k];
    }
  }
}

// Outflux on the plane x = xp from the stored post-collision populations:
// out[s] = (1/ny) sum_y sum_i c_ix g*_{s,i}(xp, y).  One block.
template <class P, int NS>
__global__ void __launch_bounds__(kReduceThreads)
    adr_flux_kernel(const void *g, const uint32_t *links, long long plane,
                    int nx_pad, int ny, int xp, double cref0, double cref1,
                    double cref2, double *out) {
  using S = typename P::S;
  const S *src = static_cast<const S *>(g);
  const double cref[3] = {cref0, cref1, cref2};
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  for (int y = threadIdx.x; y < ny; y += blockDim.x) {
    const long long n = (long long)y * nx_pad + xp;
    if (links[n] == kSolidNode) continue;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double v = 0.0;
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        if (cx(i) == 0) continue;
        double gi = double(P::load(src[(long long)(s * 9 + i) * plane + n]));
        if (P::kDev) gi += double(Lattice<float>::w(i)) * cref[s];
        v += cx(i) > 0 ? gi : -gi;
      }
      acc[s] += v;
    }
  }
  block_sum<NS>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) out[s] = acc[s] / double(ny);
  }
}

// Sum nb rows of K partials in a fixed order into out[0..K).  One block.
template <int K>
__global__ void __launch_bounds__(kReduceThreads)
    reduce_partials_kernel(const double *partials, long long nb, double *out) {
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (long long b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += partials[b * K + k];
  }
  block_sum<K>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = acc[k];
  }
}

// ---------------------------------------------------------------------------
// flow
// ---------------------------------------------------------------------------
struct FlowArgs {
  const void *src;        // S [9][plane]
  void *dst;              // S [9][plane]
  const uint32_t *links;  // [plane]
  void *u;                // T [2][plane]  (written on u / check steps)
  double *partials;       // [nblocks][2]  (check steps)
  long long plane;
  int nx, ny, nx_pad;
  double omega;           // 1/tau
  double u0;              // inflow centreline velocity
};

enum FlowMode { kFlowStep = 0, kFlowU = 1, kFlowCheck = 2, kFlowInit = 3 };

template <class P, int MODE>
__global__ void __launch_bounds__(kBlockX) flow_kernel(const FlowArgs a) {
  using S = typename P::S;
  using T = typename P::T;
  const int x = blockIdx.x * kBlockX + threadIdx.x;
  const int y = blockIdx.y;
  const long long n = (long long)y * a.nx_pad + x;
  const long long plane = a.plane;
  const uint32_t lw = (x < a.nx_pad) ? a.links[n] : kSolidNode;
  double acc[2] = {0.0, 0.0};
  T *U = static_cast<T *>(a.u);

  if (lw != kSolidNode) {
    const S *__restrict__ src = static_cast<const S *>(a.src);
    S *__restrict__ dst = static_cast<S *>(a.dst);
    const long long np = (long long)a.nx_pad;
    auto ld = [&](int i, long long m) -> T {
      return P::load(src[(long long)i * plane + m]);
    };
    // inflow parabola at this row, zeros half a node outside the walls
    const T yy = T(y);
    const T uin = T(4) * T(a.u0) * (yy + T(0.5)) * (T(a.ny) - T(0.5) - yy) /
                  (T(a.ny) * T(a.ny));

    T f[9];
    if (MODE == kFlowInit) {
      const T uu = uin * uin;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const T cu = T(cx(i)) * uin;
        f[i] = Lattice<T>::w(i) *
               (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
      }
    } else if (lw == 0u) {
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = ld(i, n - (cy(i) * np + cx(i)));
    } else {
      // velocity of the boundary node at time t (outlet rule only)
      T uwx = T(0), uwy = T(0);
      if (x == a.nx - 1) {
        T r = T(0), jx = T(0), jy = T(0);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          const T v = ld(j, n);
          r += v;
          jx += T(cx(j)) * v;
          jy += T(cy(j)) * v;
        }
        uwx = jx / r;
        uwy = jy / r;
      }
      f[0] = ld(0, n);
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const uint32_t t = nib(lw, opp(i));
        if (t == kFluid) {
          f[i] = ld(i, n - (cy(i) * np + cx(i)));
        } else if (t == kInlet) {
          // velocity bounce-back, rho_w = 1, u_w = (u_in(y), 0)
          f[i] = ld(opp(i), n) + T(6) * Lattice<T>::w(i) * T(cx(i)) * uin;
        } else if (t == kOutlet) {
          // pressure anti-bounce-back, rho_w = 1, u_w = u(x_b, t)
          const T cu = T(cx(i)) * uwx + T(cy(i)) * uwy;
          const T uu = uwx * uwx + uwy * uwy;
          f[i] = -ld(opp(i), n) +
                 T(2) * Lattice<T>::w(i) * (T(1) + T(4.5) * cu * cu - T(1.5) * uu);
        } else {
          f[i] = ld(opp(i), n);
        }
      }
    }

    T rho = T(0), jx = T(0), jy = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      rho += f[i];
      jx += T(cx(i)) * f[i];
      jy += T(cy(i)) * f[i];
    }
    const T ux = jx / rho, uy = jy / rho;
    const T uu = ux * ux + uy * uy;
    const T om = T(a.omega);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const T cu = T(cx(i)) * ux + T(cy(i)) * uy;
      const T feq = Lattice<T>::w(i) * rho *
                    (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
      dst[(long long)i * plane + n] = P::store(f[i] + om * (feq - f[i]));
    }
    if (MODE == kFlowU || MODE == kFlowCheck) {
      if (MODE == kFlowCheck) {
        acc[0] = fabs(double(ux) - double(U[n])) + fabs(double(uy) - double(U[plane + n]));
        acc[1] = fabs(double(ux)) + fabs(double(uy));
      }
      U[n] = ux;
      U[plane + n] = uy;
    }
  } else if ((MODE == kFlowU || MODE == kFlowCheck) && x < a.nx_pad) {
    U[n] = T(0);
    U[plane + n] = T(0);
  }

  if (MODE == kFlowCheck) {
    block_sum<2>(acc);
    if (threadIdx.x == 0) {
      const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
      a.partials[b * 2] = acc[0];
      a.partials[b * 2 + 1] = acc[1];
    }
  }
}

// ---------------------------------------------------------------------------
// launchers (one translation unit per precision instantiates them)
// ---------------------------------------------------------------------------
template <class P>
cudaError_t launch_adr(int ns, int mode, const AdrArgs &a, dim3 grid,
                       cudaStream_t st);
template <class P>
cudaError_t launch_adr_flux(int ns, const void *g, const uint32_t *links,
                            long long plane, int nx_pad, int ny, int xp,
                            const double *cref, double *out, cudaStream_t st);
template <class P>
cudaError_t launch_flow(int mode, const FlowArgs &a, dim3 grid, cudaStream_t st);

cudaError_t launch_reduce(int k, const double *partials, long long nb,
                          double *out, cudaStream_t st);

}  // namespace lbm
