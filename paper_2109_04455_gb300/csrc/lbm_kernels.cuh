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
#include <type_traits>

#include "lbm_internal.h"

namespace lbm {

// Launch shape of the lattice kernels (compile-time tuning knobs):
//   LBM_BLOCK_X        threads per block = nodes of one row segment
//   LBM_ADR_MIN_BLOCKS if defined, resident blocks per SM asked of the
//                      register allocator for every precision (otherwise
//                      each precision's kMinBlocks below)
#ifndef LBM_BLOCK_X
#define LBM_BLOCK_X 256
#endif
//   LBM_ADR_PAIR_F16   1: the FP16 bulk step updates two nodes per thread
//                      (adr_bulk_pair_kernel); 0: one node per thread
#ifndef LBM_ADR_PAIR_F16
#define LBM_ADR_PAIR_F16 1
#endif
//   LBM_PAIR_MIN_BLOCKS resident blocks per SM asked of the register
//                      allocator for adr_bulk_pair_kernel (6: 80 registers
//                      with per-species loads)
#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 6
#endif
constexpr int kBlockX = LBM_BLOCK_X;
#ifdef LBM_ADR_MIN_BLOCKS
#define LBM_MIN_BLOCKS(P) LBM_ADR_MIN_BLOCKS
#else
#define LBM_MIN_BLOCKS(P) P::kMinBlocks
#endif
constexpr int kReduceThreads = 256;

// ---------------------------------------------------------------------------
// precision traits: storage type S, compute type T
// ---------------------------------------------------------------------------
struct PrecF64 {
  using S = double;
  using T = double;
  static constexpr bool kDev = false;
  static constexpr int kMinBlocks = 1;
  static __device__ __forceinline__ T load(S v) { return v; }
  static __device__ __forceinline__ S store(T v) { return v; }
};
struct PrecF32 {
  using S = float;
  using T = float;
  static constexpr bool kDev = false;
  static constexpr int kMinBlocks = 1;
  static __device__ __forceinline__ T load(S v) { return v; }
  static __device__ __forceinline__ S store(T v) { return v; }
};
// half storage of the deviation g - w_i R from a per-node reference R (the
// node's concentration when the value was stored, kept in half beside the
// populations), scaled by 2^14 (exact) so that the deviations of dilute
// species stay in half's normal range (|value| <= 0.45 * 2^14 < 65504);
// rounded to nearest even.  The deviation is the advective and
// non-equilibrium part of g, a few percent of it, so half's 11 bits resolve
// g to ~1e-5 instead of ~5e-4.
struct PrecF16Dev {
  using S = __half;
  using T = float;
  static constexpr bool kDev = true;
  static constexpr int kMinBlocks = 5;   // <= 51 registers, 40 warps per SM
  static __device__ __forceinline__ T load(S v) {
    return __half2float(v) * (1.0f / 16384.0f);
  }
  static __device__ __forceinline__ S store(T v) {
    return __float2half_rn(v * 16384.0f);
  }
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
// Index of the neighbour x + c_j of the node (x, y) (plane index
// y * np + x), wrapped around a periodic edge; for a neighbour inside the
// lattice it is the plain shift.  Used on boundary nodes only (kPeriodic
// pulls, rates of catalytic links).
__device__ __forceinline__ long long neighbour(int x, int y, int j, int nx,
                                               int ny, long long np) {
  int tx = x + cx(j), ty = y + cy(j);
  tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
  ty = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
  return (long long)ty * np + tx;
}

__device__ __forceinline__ float absT(float x) { return fabsf(x); }
__device__ __forceinline__ double absT(double x) { return fabs(x); }

// ---------------------------------------------------------------------------
// deterministic block sum of K values in the value type A, stored by threads
// 0..K-1 (one component each) to dst[0..K): used in double for the outflux
// and for the adjoint's convergence measure.  (The forward check steps use
// block_partials_store below, which sums in double whatever the precision.)
// ---------------------------------------------------------------------------
template <int K, typename A>
__device__ __forceinline__ void block_sum_store(const A (&v)[K], double *dst) {
  __shared__ A red[32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  A w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    w[k] = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w[k] += __shfl_down_sync(0xffffffffu, w[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp][k] = w[k];
  }
  __syncthreads();
  if (threadIdx.x < K) {
    const int nw = (blockDim.x + 31) >> 5;
    A s = A(0);
    for (int i = 0; i < nw; ++i) s += red[i][threadIdx.x];
    dst[threadIdx.x] = double(s);
  }
}

// Check-step partials of one block, accumulated in double.  Each of the BX
// threads passes the values of NPER nodes, v[NPER][KS + KM] (zeros for a
// thread or node without a fluid node): the first KS components are summed,
// the last KM reduced by minimum (a minimum starts at 0, so it is that of
// min(value, 0)).  The values are staged in shared memory, one row per
// component; warp w then reduces components w, w + BX/32, ...: its lanes add
// the component's values at a stride of 32 in double, and the 32 lane sums
// are folded by double shuffles.  Every per-node value enters a double sum,
// so a block partial carries no single-precision rounding; the fixed order
// makes it deterministic.
template <int KS, int KM, int NPER, int BX, typename A>
__device__ __forceinline__ void block_partials_store(const A (&v)[NPER][KS + KM],
                                                     double *dst) {
  constexpr int K = KS + KM;
  constexpr int NV = BX * NPER;
  static_assert(BX % 32 == 0, "whole warps");
  __shared__ A stage[K][NV];
  const int t = threadIdx.x;
#pragma unroll
  for (int p = 0; p < NPER; ++p) {
#pragma unroll
    for (int k = 0; k < K; ++k) stage[k][p * BX + t] = v[p][k];
  }
  __syncthreads();
  const int lane = t & 31, warp = t >> 5;
  for (int k = warp; k < K; k += BX / 32) {
    double r = 0.0;
    if (k < KS) {
#pragma unroll 4
      for (int j = lane; j < NV; j += 32) r += double(stage[k][j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    } else {
      A m = A(0);
#pragma unroll 4
      for (int j = lane; j < NV; j += 32) m = stage[k][j] < m ? stage[k][j] : m;
      r = double(m);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r = fmin(r, __shfl_down_sync(0xffffffffu, r, o));
    }
    if (lane == 0) dst[k] = r;
  }
}

// Per-node contribution of species s to a check step's partials (layout
// [2 NS sums | NS minima]): |C(t) - C(t-1)|, |C(t)|, and C(t) for the most
// negative concentration.
template <int NS, typename T>
__device__ __forceinline__ void check_add(T (&acc)[3 * NS], int s, T c, T prev) {
  acc[2 * s] += absT(c - prev);
  acc[2 * s + 1] += absT(c);
  acc[2 * NS + s] = c < acc[2 * NS + s] ? c : acc[2 * NS + s];
}

// two-wide vector of a storage / compute type
template <typename S> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<__half> { using type = __half2; };

template <typename S>
__device__ __forceinline__ S zero_of() { return S(0); }
template <>
__device__ __forceinline__ __half zero_of<__half>() { return __float2half_rn(0.0f); }


// Reference concentrations of the half path are themselves stored in half:
// any reference works as long as the writer and every reader use the same
// value, so the writer subtracts the rounded reference it stores.
using RefT = __half;
__device__ __forceinline__ float ref_get(const RefT *r, long long k) {
  return __half2float(r[k]);
}
__device__ __forceinline__ float ref_round(float c) {
  return __half2float(__float2half_rn(c));
}

// Kernel parameters come in double and in float; the float paths read the
// float copy, so no thread converts a double (this part's FP64 pipe is
// narrow enough for per-thread conversions to show up in a step's time).
template <typename T>
__device__ __forceinline__ T pick(double d, float f);
template <>
__device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pick<float>(double, float f) { return f; }


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
  double *partials;         // [rows][3*ns]      (check steps)
  const long long *bnodes;  // boundary fluid nodes (link word != 0)
  long long nbnd;           // number of boundary nodes
  long long part_off;       // first partial row of the boundary kernel
  long long plane;          // ny * nx_pad
  int nx, ny, nx_pad;
  int abb_all;              // anti-bounce-back inlet for every species
  int nodewise;             // every population of a reactive node reacts
  unsigned step;            // steps done before this one (rounding seed)
  int xp;                   // flux plane
  double omega[3];          // 1/tau per species
  double cin[3];            // inlet concentration per species
  float fomega[3], fcin[3]; // the same in float
  // half storage: reference concentrations [ns][plane] of the src and dst
  // populations (the stored value is g - w_i R of its node)
  const RefT *rsrc;
  RefT *rdst;
  // FP64: equilibrium factors E_i(u) [9][plane] of the frozen velocity,
  // filled once by eq_table_kernel (nullptr: computed per node and step;
  // the FP64 step is bound by this part's FP64 pipe, and the table takes
  // about a third of its double operations away)
  const double *etab;
};

enum AdrMode { kAdrStep = 0, kAdrCheck = 1, kAdrInit = 2 };


// value added back to the stored population (s, i) of node m (half storage
// only: w_i times the node's reference concentration)
template <class P>
__device__ __forceinline__ typename P::T adr_ref(const AdrArgs &a, int s, int i,
                                                 long long m) {
  using T = typename P::T;
  if constexpr (P::kDev)
    return Lattice<T>::w(i) * T(ref_get(a.rsrc, s * a.plane + m));
  else
    return T(0);
}
// value removed before storing population i of a node whose reference is c
template <class P>
__device__ __forceinline__ typename P::T adr_unref(int i, typename P::T c) {
  using T = typename P::T;
  if constexpr (P::kDev)
    return Lattice<T>::w(i) * c;
  else
    return T(0);
}

template <class P>
__device__ __forceinline__ typename P::T adr_ld(const AdrArgs &a, int s, int i,
                                                long long m) {
  const typename P::S *src = static_cast<const typename P::S *>(a.src);
  return P::load(src[(long long)(s * 9 + i) * a.plane + m]) + adr_ref<P>(a, s, i, m);
}

// equilibrium factors E_i(u), shared by every species:
// g_i^eq = C * E_i, E_i = w_i (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u)
template <typename T>
__device__ __forceinline__ void eq_factors(T ux, T uy, T (&E)[9]) {
  const T uu = ux * ux + uy * uy;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T cu = T(cx(i)) * ux + T(cy(i)) * uy;
    E[i] = Lattice<T>::w(i) * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
  }
}
// The double version is written with explicit roundings: the FP64 step reads
// E from a table that eq_table_kernel fills once per solver, while boundary
// nodes and the batch kernel compute it in place, and all of them must get
// the same bits.
template <>
__device__ __forceinline__ void eq_factors<double>(double ux, double uy,
                                                   double (&E)[9]) {
  const double base = __fma_rn(-1.5, __fma_rn(ux, ux, __dmul_rn(uy, uy)), 1.0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double cu = __dadd_rn(double(cx(i)) * ux, double(cy(i)) * uy);
    E[i] = __dmul_rn(Lattice<double>::w(i),
                     __fma_rn(__dmul_rn(4.5, cu), cu, __fma_rn(3.0, cu, base)));
  }
}

// equilibrium factors of node n: from the FP64 table when there is one
template <class P>
__device__ __forceinline__ void adr_eq(const AdrArgs &a, long long n,
                                       typename P::T (&E)[9]) {
  using T = typename P::T;
  if constexpr (sizeof(T) == 8) {
    if (a.etab != nullptr) {
#pragma unroll
      for (int i = 0; i < 9; ++i) E[i] = a.etab[(long long)i * a.plane + n];
      return;
    }
  }
  const T *__restrict__ U = static_cast<const T *>(a.u);
  eq_factors<T>(U[n], U[a.plane + n], E);
}

// E_i(u) of every node of the lattice into etab [9][plane] (FP64 only)
template <typename T>
__global__ void __launch_bounds__(256)
    eq_table_kernel(const T *u, long long plane, T *etab) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= plane) return;
  T E[9];
  eq_factors<T>(u[n], u[plane + n], E);
#pragma unroll
  for (int i = 0; i < 9; ++i) etab[(long long)i * plane + n] = E[i];
}

// The species are updated one after the other (A, then B, then C): the
// sources are triangular (A's depends on C_A, B's on C_A and C_B, C's on
// C_B), so every source term is known when its species is collided, and only
// one species' nine populations need to be live at a time.

// Boundary node x (link word lw != 0), species s: replace every population
// whose pull source is not a fluid node by the rule of that source's link
// type (Eq. BC and bounce-back), reading the node's own post-collision values.
template <class P>
__device__ __forceinline__ void adr_boundary(const AdrArgs &a, int s,
                                             uint32_t lw, long long n, int x,
                                             typename P::T (&g)[9]) {
  using T = typename P::T;
  T cb = T(0);
  if (x == a.nx - 1) {
#pragma unroll
    for (int j = 0; j < 9; ++j) cb += adr_ld<P>(a, s, j, n);
  }
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const uint32_t t = nib(lw, opp(i));
    if (t == kFluid || t == kPeriodic) continue;   // pulled already
    const T back = adr_ld<P>(a, s, opp(i), n);
    if (t == kInlet) {
      g[i] = (s == 0 || a.abb_all)
                 ? -back + T(2) * Lattice<T>::w(i) * pick<T>(a.cin[s], a.fcin[s])
                                   : back;
    } else if (t == kOutlet) {
      g[i] = -back + T(2) * Lattice<T>::w(i) * cb;
    } else {  // wall, inert or catalytic fiber: bounce-back
      g[i] = back;
    }
  }
}

// BGK collision of species s towards C E_i, then its Dawson source on links
// into catalytic fiber nodes (Eq. source_lbm):
//   Q_A = -k_AB w C_A,  Q_B = +k_AB w C_A - k_BC w C_B,  Q_C = +k_BC w C_B.
// With a.nodewise, a node with catalytic links reacts on all nine
// populations instead, with the mean rates of those links.
// C[] holds the pre-collision concentrations of species 0..s; returns C_s.
template <class P, int NS>
__device__ __forceinline__ typename P::T adr_collide(const AdrArgs &a, int s,
                                                     uint32_t lw, long long n,
                                                     int x, int y,
                                                     const typename P::T (&E)[9],
                                                     typename P::T (&g)[9],
                                                     typename P::T (&C)[NS]) {
  using T = typename P::T;
  T c = T(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) c += g[i];
  C[s] = c;
  const T om = pick<T>(a.omega[s], a.fomega[s]);
#pragma unroll
  for (int i = 0; i < 9; ++i) g[i] = g[i] + om * (c * E[i] - g[i]);
  if (lw != 0u && a.nodewise) {
    const long long np = a.nx_pad;
    T sa = T(0), sb = T(0);
    int ncat = 0;
#pragma unroll
    for (int j = 1; j < 9; ++j) {
      if (nib(lw, j) != kCat) continue;
      const long long m = neighbour(x, y, j, a.nx, a.ny, np);
      sa += T(a.kab[m]);
      sb += T(a.kbc[m]);
      ++ncat;
    }
    if (ncat > 0) {
      const T ka = sa / T(ncat), kb = sb / T(ncat);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const T wi = Lattice<T>::w(i);
        if (s == 0) {
          g[i] -= ka * wi * C[0];
        } else if (s == 1) {
          const T ra = ka * wi * C[0];
          const T rb = (NS >= 3) ? kb * wi * C[NS >= 2 ? 1 : 0] : T(0);
          g[i] += ra - rb;
        } else {
          g[i] += kb * wi * C[NS >= 2 ? 1 : 0];
        }
      }
    }
  } else if (lw != 0u) {
    const long long np = a.nx_pad;
#pragma unroll
    for (int j = 1; j < 9; ++j) {
      if (nib(lw, j) != kCat) continue;
      const long long m = neighbour(x, y, j, a.nx, a.ny, np);
      const T wj = Lattice<T>::w(j);
      if (s == 0) {
        g[j] -= T(a.kab[m]) * wj * C[0];
      } else if (s == 1) {
        const T ra = T(a.kab[m]) * wj * C[0];
        const T rb = (NS >= 3) ? T(a.kbc[m]) * wj * C[NS >= 2 ? 1 : 0] : T(0);
        g[j] += ra - rb;
      } else {
        g[j] += T(a.kbc[m]) * wj * C[NS >= 2 ? 1 : 0];
      }
    }
  }
  return c;
}

// Update of one fluid node x = n % nx_pad with every link rule in place (or
// its initial state): the species one after the other.
template <class P, int NS, int MODE>
__device__ __forceinline__ void adr_general_node(const AdrArgs &a, long long n,
                                                 int x, uint32_t lw,
                                                 typename P::T (&acc)[3 * NS]) {
  using S = typename P::S;
  using T = typename P::T;
  const long long plane = a.plane;
  S *__restrict__ dst = static_cast<S *>(a.dst);
  const long long np = (long long)a.nx_pad;
  const int y = lw != 0u ? static_cast<int>(n / np) : 0;
  T E[9];
  adr_eq<P>(a, n, E);
  T C[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    T g[9];
    if (MODE == kAdrInit) {
      const T c0 = (s == 0) ? T(1) : T(0);
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = c0 * E[i];
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        // pull from x - c_i when that node is fluid (always for lw == 0),
        // from the wrapped node across a periodic edge
        const uint32_t t = (i == 0 || lw == 0u) ? (uint32_t)kFluid : nib(lw, opp(i));
        if (t == kFluid)
          g[i] = adr_ld<P>(a, s, i, n - (cy(i) * np + cx(i)));
        else if (t == kPeriodic)
          g[i] = adr_ld<P>(a, s, i, neighbour(x, y, opp(i), a.nx, a.ny, np));
      }
      if (lw != 0u) adr_boundary<P>(a, s, lw, n, x, g);
    }
    const T c = adr_collide<P, NS>(a, s, lw, n, x, y, E, g, C);
    T cq = c;   // the reference stored with the populations (half path)
    if constexpr (P::kDev) {
      cq = ref_round(c);
      a.rdst[s * plane + n] = __float2half_rn(c);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i)
      dst[(long long)(s * 9 + i) * plane + n] = P::store(g[i] - adr_unref<P>(i, cq));
    if (MODE == kAdrCheck) {
      T *cp = static_cast<T *>(a.cprev);
      check_add<NS, T>(acc, s, c, cp[s * plane + n]);
      cp[s * plane + n] = c;
    }
  }
}

// L2 prefetch ahead of the bulk stencil.  With D = LBM_PREFETCH_ROWS_* > 0
// each block of the bulk step asks L2 for the row segments that the block D
// rows further down will read: one bulk prefetch per plane (the 9 NS
// population rows y + D - c_iy, for FP16 storage the NS reference rows, u
// and the link words of row y + D).  Blocks start in row order, so those
// lines are on their way from HBM about D rows of blocks before their loads
// are issued, and they are in flight without holding registers.
#ifndef LBM_PREFETCH_ROWS_F16
#define LBM_PREFETCH_ROWS_F16 6
#endif
#ifndef LBM_PREFETCH_ROWS_F32
#define LBM_PREFETCH_ROWS_F32 0
#endif
// [p, p + bytes) into L2, nothing to wait for; p 16-byte aligned and bytes
// a multiple of 16
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
               :: "l"(p), "r"(bytes) : "memory");
}
// S: stored population type, U: velocity type, REF: reference planes
// (FP16 storage).  Rows outside the lattice are skipped.
template <typename S, typename U, int NS, bool REF>
__device__ __forceinline__ void bulk_prefetch_rows(const AdrArgs &a, int yp) {
  constexpr int kPop = 9 * NS, kRef = REF ? NS : 0;
  const int t = threadIdx.x;
  if (t >= kPop + kRef + 3 || yp >= a.ny) return;
  const long long np = a.nx_pad, plane = a.plane;
  const int xb = blockIdx.x * kBlockX;
  // nx_pad is a multiple of 32 and xb of kBlockX, so every segment starts
  // 64-byte aligned (buffers are 256-byte aligned) and is a multiple of 64
  // bytes long
  const unsigned cnt = static_cast<unsigned>(min(kBlockX, a.nx_pad - xb));
  if (t < kPop) {
    const int i = t % 9, row = yp - cy(i);
    if (row < 0 || row >= a.ny) return;
    prefetch_l2(static_cast<const S *>(a.src) + (long long)t * plane +
                    (long long)row * np + xb,
                static_cast<unsigned>(sizeof(S)) * cnt);
  } else if (t < kPop + kRef) {
    prefetch_l2(a.rsrc + (long long)(t - kPop) * plane + (long long)yp * np + xb,
                static_cast<unsigned>(sizeof(RefT)) * cnt);
  } else if (t < kPop + kRef + 2) {
    prefetch_l2(static_cast<const U *>(a.u) + (long long)(t - kPop - kRef) * plane +
                    (long long)yp * np + xb,
                static_cast<unsigned>(sizeof(U)) * cnt);
  } else {
    prefetch_l2(a.links + (long long)yp * np + xb, 4u * cnt);
  }
}


}  // namespace lbm
// FP16-deviation storage: interior update (one and two nodes per thread)
#include "lbm_f16.cuh"
namespace lbm {

// Update of one interior node (link word 0: every neighbour is fluid): the
// interior formula (pull from x - c_i, BGK, no source).  All populations of
// all species are loaded before any arithmetic, so a thread keeps NS*9
// independent loads in flight.
template <class P, int NS, int MODE>
__device__ __forceinline__ void adr_interior_node(const AdrArgs &a, long long n,
                                                  typename P::T (&acc)[3 * NS]) {
  using S = typename P::S;
  using T = typename P::T;
  if constexpr (P::kDev) {
    adr_interior_node_f16<NS, MODE>(a, n, acc);
    return;
  }
  const long long np = a.nx_pad, plane = a.plane;
  const S *__restrict__ src = static_cast<const S *>(a.src);
  S *__restrict__ dst = static_cast<S *>(a.dst);
  T g[NS][9];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const long long m = n - (cy(i) * np + cx(i));
      g[s][i] = P::load(src[(long long)(s * 9 + i) * plane + m]);
    }
  }
  // the previous concentrations are loaded with the populations, so the
  // check step waits on memory once, like the plain step
  T *__restrict__ cp = static_cast<T *>(a.cprev);
  T prev[NS];
  if (MODE == kAdrCheck) {
#pragma unroll
    for (int s = 0; s < NS; ++s) prev[s] = cp[s * plane + n];
  }
  T E[9];
  adr_eq<P>(a, n, E);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    T c = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) c += g[s][i];
    const T om = pick<T>(a.omega[s], a.fomega[s]);
#pragma unroll
    for (int i = 0; i < 9; ++i)
      dst[(long long)(s * 9 + i) * plane + n] =
          P::store(g[s][i] + om * (c * E[i] - g[s][i]));
    if (MODE == kAdrCheck) {
      check_add<NS, T>(acc, s, c, prev[s]);
      cp[s * plane + n] = c;
    }
  }
}

// One node per thread, every link rule handled in place.  LIST = false: the
// whole lattice (initial state; also the plain one-kernel step).  LIST = true:
// only the boundary nodes of a.bnodes, after the bulk kernel (below) has
// updated the interior nodes; its partial sums go to rows a.part_off + block.
template <class P, int NS, int MODE, bool LIST>
__global__ void __launch_bounds__(kBlockX, LBM_MIN_BLOCKS(P))
    adr_node_kernel(const AdrArgs a) {
  using T = typename P::T;
  long long n;
  int x;
  uint32_t lw;
  if (LIST) {
    const long long t = (long long)blockIdx.x * kBlockX + threadIdx.x;
    n = t < a.nbnd ? a.bnodes[t] : 0;
    x = static_cast<int>(n % a.nx_pad);
    lw = t < a.nbnd ? a.links[n] : kSolidNode;
  } else {
    x = blockIdx.x * kBlockX + threadIdx.x;
    n = (long long)blockIdx.y * a.nx_pad + x;
    lw = (x < a.nx_pad) ? a.links[n] : kSolidNode;
  }
  T acc[1][3 * NS];
#pragma unroll
  for (int k = 0; k < 3 * NS; ++k) acc[0][k] = T(0);
  if (lw != kSolidNode) adr_general_node<P, NS, MODE>(a, n, x, lw, acc[0]);
  if constexpr (MODE == kAdrCheck) {
    const long long b = LIST ? a.part_off + blockIdx.x
                             : (long long)blockIdx.y * gridDim.x + blockIdx.x;
    block_partials_store<2 * NS, NS, 1, kBlockX, T>(acc, a.partials + b * (3 * NS));
  }
}

// Bulk step, one node per thread: the interior formula for the nodes whose
// eight neighbours are all fluid (link word 0); every other node is left to
// adr_node_kernel<..., LIST = true>, which runs beside it.
template <class P, int NS, int MODE>
__global__ void __launch_bounds__(kBlockX, LBM_MIN_BLOCKS(P))
    adr_bulk_kernel(const AdrArgs a) {
  using T = typename P::T;
  if constexpr (std::is_same<typename P::S, float>::value && LBM_PREFETCH_ROWS_F32 > 0)
    bulk_prefetch_rows<float, float, NS, false>(a, blockIdx.y + LBM_PREFETCH_ROWS_F32);
  const int x = blockIdx.x * kBlockX + threadIdx.x;
  const long long n = (long long)blockIdx.y * a.nx_pad + x;
  const uint32_t lw = (x < a.nx_pad) ? a.links[n] : kSolidNode;
  T acc[1][3 * NS];
#pragma unroll
  for (int k = 0; k < 3 * NS; ++k) acc[0][k] = T(0);
  // (half storage: the references of the nine source nodes are read next
  // to the populations; gathering them with warp shuffles instead measured
  // slower, the shuffles keep the population loads from being issued early)
  if (lw == 0u) adr_interior_node<P, NS, MODE>(a, n, acc[0]);
  if constexpr (MODE == kAdrCheck) {
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    block_partials_store<2 * NS, NS, 1, kBlockX, T>(acc, a.partials + b * (3 * NS));
  }
}

// Outflux on the plane x = xp from the stored post-collision populations:
// out[s] = (1/ny) sum_y sum_i c_ix g*_{s,i}(xp, y).  One block.
template <class P, int NS>
__global__ void __launch_bounds__(kReduceThreads)
    adr_flux_kernel(const void *g, const RefT *ref, const uint32_t *links,
                    long long plane, int nx_pad, int ny, int xp, double *out) {
  using S = typename P::S;
  const S *src = static_cast<const S *>(g);
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
        if (P::kDev) gi += double(Lattice<float>::w(i)) * double(ref_get(ref, s * plane + n));
        v += cx(i) > 0 ? gi : -gi;
      }
      acc[s] += v;
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] /= double(ny);
  block_sum_store<NS, double>(acc, out);
}

// Fold rows of KS + KM partials in a fixed order (sums of the first KS
// components, minima of the last KM).  Block b of the grid folds the rows
// [b*chunk, (b+1)*chunk) into out[b*K + k]; a second launch with one block
// folds those.  Deterministic for a fixed grid.
template <int KS, int KM>
__global__ void __launch_bounds__(kReduceThreads)
    reduce_partials_kernel(const double *partials, long long nb, long long chunk,
                           double *out) {
  constexpr int K = KS + KM;
  double acc[1][K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[0][k] = 0.0;
  const long long lo = (long long)blockIdx.x * chunk;
  long long hi = lo + chunk;
  if (hi > nb) hi = nb;
  for (long long b = lo + threadIdx.x; b < hi; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      acc[0][k] = k < KS ? acc[0][k] + partials[b * K + k]
                         : fmin(acc[0][k], partials[b * K + k]);
  }
  block_partials_store<KS, KM, 1, kReduceThreads, double>(
      acc, out + (long long)blockIdx.x * K);
}

}  // namespace lbm
// discrete adjoint of the ADR step: arguments and kernels
#include "lbm_adjoint.cuh"
namespace lbm {

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
  float fomega, fu0;      // the same in float
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
  T acc[1][2] = {{T(0), T(0)}};
  T *U = static_cast<T *>(a.u);

  if (lw != kSolidNode) {
    const S *__restrict__ src = static_cast<const S *>(a.src);
    S *__restrict__ dst = static_cast<S *>(a.dst);
    const long long np = (long long)a.nx_pad;
    auto ld = [&](int i, long long m) -> T {
      return P::load(src[(long long)i * plane + m]);
    };
    // inflow parabola at this row, zeros half a node outside the walls
    // (evaluated only where it is used: the initial state and inlet links;
    // its division is a sizeable share of an FP64 node update)
    auto inflow = [&]() -> T {
      const T yy = T(y);
      return T(4) * pick<T>(a.u0, a.fu0) * (yy + T(0.5)) * (T(a.ny) - T(0.5) - yy) /
             (T(a.ny) * T(a.ny));
    };

    T f[9];
    if (MODE == kFlowInit) {
      const T uin = inflow();
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
        } else if (t == kPeriodic) {
          f[i] = ld(i, neighbour(x, y, opp(i), a.nx, a.ny, np));
        } else if (t == kInlet) {
          // velocity bounce-back, rho_w = 1, u_w = (u_in(y), 0)
          f[i] = ld(opp(i), n) + T(6) * Lattice<T>::w(i) * T(cx(i)) * inflow();
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
    const T om = pick<T>(a.omega, a.fomega);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const T cu = T(cx(i)) * ux + T(cy(i)) * uy;
      const T feq = Lattice<T>::w(i) * rho *
                    (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
      dst[(long long)i * plane + n] = P::store(f[i] + om * (feq - f[i]));
    }
    if (MODE == kFlowU || MODE == kFlowCheck) {
      if (MODE == kFlowCheck) {
        acc[0][0] = absT(ux - U[n]) + absT(uy - U[plane + n]);
        acc[0][1] = absT(ux) + absT(uy);
      }
      U[n] = ux;
      U[plane + n] = uy;
    }
  } else if ((MODE == kFlowU || MODE == kFlowCheck) && x < a.nx_pad) {
    U[n] = T(0);
    U[plane + n] = T(0);
  }

  if constexpr (MODE == kFlowCheck) {
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    block_partials_store<2, 0, 1, kBlockX, T>(acc, a.partials + b * 2);
  }
}

// ---------------------------------------------------------------------------
// launchers (one translation unit per precision instantiates them)
// ---------------------------------------------------------------------------
// A time step is the bulk kernel (two nodes per thread, interior formula)
// followed by the boundary kernel over the boundary-node list; with
// LBM_ADR_SPLIT=0 it is the one-node kernel over the whole lattice instead.
#ifndef LBM_ADR_SPLIT
#define LBM_ADR_SPLIT 1
#endif
inline dim3 adr_bulk_grid(int nx_pad, int ny) {
  const int per = kBlockX;
  return dim3(static_cast<unsigned>((nx_pad + per - 1) / per),
              static_cast<unsigned>(ny));
}
inline dim3 adr_node_grid(int nx_pad, int ny) {
  return dim3(static_cast<unsigned>((nx_pad + kBlockX - 1) / kBlockX),
              static_cast<unsigned>(ny));
}
inline long long adr_list_blocks(long long nbnd) {
  return (nbnd + kBlockX - 1) / kBlockX;
}
// partial-sum rows written by one check step
inline long long adr_partial_rows(int nx_pad, int ny, long long nbnd) {
  if (!LBM_ADR_SPLIT) {
    const dim3 g = adr_node_grid(nx_pad, ny);
    return static_cast<long long>(g.x) * g.y;
  }
  const dim3 g = adr_bulk_grid(nx_pad, ny);
  return static_cast<long long>(g.x) * g.y + adr_list_blocks(nbnd);
}

// second stream and fork / join events for running the boundary-node kernel
// beside the bulk kernel (aux == nullptr: one stream)
struct AdrOverlap {
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
template <class P>
cudaError_t launch_adr(int ns, int mode, const AdrArgs &a, cudaStream_t st,
                       const AdrOverlap *ov = nullptr);
template <class P>
cudaError_t launch_adr_flux(int ns, const void *g, const RefT *ref,
                            const uint32_t *links, long long plane, int nx_pad,
                            int ny, int xp, double *out, cudaStream_t st);
template <class P>
cudaError_t launch_flow(int mode, const FlowArgs &a, dim3 grid, cudaStream_t st);
template <class P>
cudaError_t launch_adjoint(int ns, int mode, const AdjArgs &a, cudaStream_t st);
// FP64 equilibrium-factor table of a velocity field (defined with the FP64
// kernels)
cudaError_t launch_eq_table(const double *u, long long plane, double *etab,
                            cudaStream_t st);
template <class P>
cudaError_t launch_adjoint_grad(int ns, const AdjArgs &a, const long long *bnodes,
                                long long nbnd, const void *conc, double *dkab,
                                double *dkbc, const int32_t *fiber, double *dw,
                                double k1, double k2, cudaStream_t st);

// Two-level deterministic fold of nb rows of ks + km partials (ks sums, km
// minima) into out[0..ks+km); scratch holds kReduceGrid * (ks + km)
// doubles.  (ks, km) is (2, 0) (flow and adjoint residuals) or
// (2 ns, ns) (ADR check steps).
constexpr int kReduceGrid = 256;
cudaError_t launch_reduce(int ks, int km, const double *partials, long long nb,
                          double *scratch, double *out, cudaStream_t st);

// Slots of a solver's result buffer: the folded check partials
// [2 ns sums | ns minima] from 0, the outfluxes from kResFlux.
constexpr int kResFlux = 16;
constexpr int kResSlots = 24;

}  // namespace lbm
