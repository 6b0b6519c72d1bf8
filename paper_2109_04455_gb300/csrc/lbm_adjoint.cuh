// Discrete adjoint of the ADR step: its arguments and kernels.  Included by
// lbm_kernels.cuh after the forward step's helpers (eq_factors, block sums,
// link words), which it reuses.
#pragma once

namespace lbm {

// ---------------------------------------------------------------------------
// discrete adjoint of the ADR step (frozen u)
//
// The step is affine in the stored state: g*(t+1) = K (P g*(t) + b), with P
// the pull and its link rules, K the per-node collision + source.  The
// efficiency depends on g* on the flux plane through N_s (dN[s] = d eps/dN_s).
// The adjoint of the pre-collision populations solves
//   nu = K^T (P^T nu + l),   l_{s,i}(x) = dN[s] c_ix / ny on the plane,
// iterated from nu = 0.  P^T is a gather in the opposite direction of the
// forward pull: the value pulled by neighbour x + c_i is read back from it,
// a bounced population from the node's own opposite direction.  K^T is
// local and cheap: nu'_{s,m} = (1 - w_s) mu_{s,m} + w_s sum_i E_i mu_{s,i}
// + R_s, with R_A = sum_j w_j k_AB (mu_B - mu_A)_j and
// R_B = sum_j w_j k_BC (mu_C - mu_B)_j over the catalytic links j.
// ---------------------------------------------------------------------------
struct AdjArgs {
  const void *src;          // T [ns][9][plane]  nu at iteration t
  void *dst;                // T [ns][9][plane]  nu at iteration t+1
  const uint32_t *links;
  const double *kab, *kbc;
  const void *u;            // T [2][plane]
  const double *etab;       // FP64: E_i(u) [9][plane] of the forward solver
  double *partials;         // [rows][2]  (check iterations)
  long long plane;
  int nx, ny, nx_pad, xp;
  int abb_all;
  int periodic;             // the geometry has periodic edges (kPeriodic links)
  double omega[3];
  double dN[3];             // d eps / d N_s
  float fomega[3], fdN[3];  // the same in float
};

enum AdjMode { kAdjStep = 0, kAdjCheck = 1 };

// mu = P^T nu + l of species s at fluid node n = y nx_pad + x (link word lw).
// PER: the geometry may have periodic links (wrapped neighbours); without
// them the gather keeps the plain shifts and fewer registers.
template <typename T, bool PER>
__device__ __forceinline__ void adj_gather(const AdjArgs &a, int s, uint32_t lw,
                                           long long n, int x, int y, T (&mu)[9]) {
  const T *nu = static_cast<const T *>(a.src) + (long long)s * 9 * a.plane;
  const long long np = a.nx_pad, plane = a.plane;
  mu[0] = nu[n];
  T outlet = T(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const uint32_t t = lw == 0u ? (uint32_t)kFluid : nib(lw, i);
    if (t == kFluid) {
      mu[i] = nu[(long long)i * plane + n + cy(i) * np + cx(i)];
    } else if (PER && t == kPeriodic) {
      mu[i] = nu[(long long)i * plane + neighbour(x, y, i, a.nx, a.ny, np)];
    } else {
      const T back = nu[(long long)opp(i) * plane + n];
      if (t == kInlet) {
        mu[i] = (s == 0 || a.abb_all) ? -back : back;
      } else if (t == kOutlet) {
        mu[i] = -back;
        outlet += T(2) * Lattice<T>::w(opp(i)) * back;
      } else {
        mu[i] = back;
      }
    }
  }
  if (outlet != T(0)) {
#pragma unroll
    for (int i = 0; i < 9; ++i) mu[i] += outlet;
  }
  if (x == a.xp) {
    const T d = pick<T>(a.dN[s], a.fdN[s]) / T(a.ny);
#pragma unroll
    for (int i = 0; i < 9; ++i) mu[i] += T(cx(i)) * d;
  }
}

// nu' = K^T mu of one node: lam_s = om sum_i E_i mu_i + R_s, then
// nu'_m = (1 - om) mu_m + lam_s, stored (check iterations also sum |dnu|)
template <typename T, int NS, int MODE>
__device__ __forceinline__ void adj_update(const AdjArgs &a, long long n,
                                           const T (&E)[9], const T (&mu)[NS][9],
                                           const T (&R)[NS], T (&acc)[2]) {
  const long long plane = a.plane;
  T *dst = static_cast<T *>(a.dst);
  const T *src = static_cast<const T *>(a.src);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const T om = pick<T>(a.omega[s], a.fomega[s]);
    T lam = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) lam += E[i] * mu[s][i];
    lam = om * lam + R[s];
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      const T v = (T(1) - om) * mu[s][m] + lam;
      const long long idx = (long long)(s * 9 + m) * plane + n;
      if (MODE == kAdjCheck) {
        acc[0] += absT(v - src[idx]);
        acc[1] += absT(v);
      }
      dst[idx] = v;
    }
  }
}

template <typename T>
__device__ __forceinline__ void adj_eq(const AdjArgs &a, long long n, T (&E)[9]) {
  if (sizeof(T) == 8 && a.etab != nullptr) {
#pragma unroll
    for (int i = 0; i < 9; ++i) E[i] = T(a.etab[(long long)i * a.plane + n]);
  } else {
    const T *U = static_cast<const T *>(a.u);
    eq_factors<T>(U[n], U[a.plane + n], E);
  }
}

// One adjoint iteration.  Interior nodes (link word 0: every neighbour is
// fluid, no source, no inlet or outlet) take a branch-free path that issues
// all NS*9 gathered loads before any arithmetic; boundary nodes go through
// adj_gather's link rules.  Both give the same values for an interior node.
template <typename T, int NS, int MODE, bool PER>
__global__ void __launch_bounds__(kBlockX) adj_kernel(const AdjArgs a) {
  const int x = blockIdx.x * kBlockX + threadIdx.x;
  const int y = blockIdx.y;
  const long long n = (long long)y * a.nx_pad + x;
  const long long plane = a.plane;
  const uint32_t lw = (x < a.nx_pad) ? a.links[n] : kSolidNode;
  T acc[2] = {T(0), T(0)};
  if (lw == 0u) {
    const long long np = a.nx_pad;
    const T *nu = static_cast<const T *>(a.src);
    T mu[NS][9];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int i = 0; i < 9; ++i)
        mu[s][i] = nu[(long long)(s * 9 + i) * plane + n + cy(i) * np + cx(i)];
    }
    T E[9];
    adj_eq<T>(a, n, E);
    if (x == a.xp) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const T d = pick<T>(a.dN[s], a.fdN[s]) / T(a.ny);
#pragma unroll
        for (int i = 0; i < 9; ++i) mu[s][i] += T(cx(i)) * d;
      }
    }
    T R[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) R[s] = T(0);
    adj_update<T, NS, MODE>(a, n, E, mu, R, acc);
  } else if (lw != kSolidNode) {
    T E[9];
    adj_eq<T>(a, n, E);
    T mu[NS][9];
#pragma unroll
    for (int s = 0; s < NS; ++s) adj_gather<T, PER>(a, s, lw, n, x, y, mu[s]);
    T R[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) R[s] = T(0);
    const long long np = a.nx_pad;
#pragma unroll
    for (int j = 1; j < 9; ++j) {
      if (nib(lw, j) != kCat) continue;
      const long long m = PER ? neighbour(x, y, j, a.nx, a.ny, np)
                              : n + cy(j) * np + cx(j);
      const T wj = Lattice<T>::w(j);
      const T ka = T(a.kab[m]) * wj;
      R[0] += ka * ((NS >= 2 ? mu[NS >= 2 ? 1 : 0][j] : T(0)) - mu[0][j]);
      if (NS >= 3) {
        const T kb = T(a.kbc[m]) * wj;
        R[NS >= 3 ? 1 : 0] += kb * (mu[NS >= 3 ? 2 : 0][j] - mu[NS >= 3 ? 1 : 0][j]);
      }
    }
    adj_update<T, NS, MODE>(a, n, E, mu, R, acc);
  }
  if (MODE == kAdjCheck) {
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    block_sum_store<2, T>(acc, a.partials + b * 2);
  }
}

// Rate gradients from the adjoint (a.src = nu) and the pre-collision
// concentrations C (the forward solver's last checked step), over the
// boundary nodes; each link x -> n into a fiber node adds
//   d eps/dk_AB(n) += w_j C_A(x) (mu_B - mu_A)_j,
//   d eps/dk_BC(n) += w_j C_B(x) (mu_C - mu_B)_j,
// and, when fiber ids are given, d eps/dw_f += k1 (first) - k2 (second).
template <typename T, int NS>
__global__ void __launch_bounds__(kBlockX)
    adj_grad_kernel(const AdjArgs a, const long long *bnodes, long long nbnd,
                    const T *conc, double *dkab, double *dkbc,
                    const int32_t *fiber, double *dw, double k1, double k2) {
  const long long t = (long long)blockIdx.x * kBlockX + threadIdx.x;
  if (t >= nbnd) return;
  const long long n = bnodes[t];
  const uint32_t lw = a.links[n];
  const int x = static_cast<int>(n % a.nx_pad);
  const int y = static_cast<int>(n / a.nx_pad);
  T mu[NS][9];
#pragma unroll
  for (int s = 0; s < NS; ++s) adj_gather<T, true>(a, s, lw, n, x, y, mu[s]);
  const T cA = conc[n];
  const T cB = NS >= 2 ? conc[a.plane + n] : T(0);
  const long long np = a.nx_pad;
#pragma unroll
  for (int j = 1; j < 9; ++j) {
    const uint32_t ty = nib(lw, j);
    if (ty != kCat && ty != kInert) continue;
    const long long m = neighbour(x, y, j, a.nx, a.ny, np);
    const double wj = double(Lattice<T>::w(j));
    double ga = -double(mu[0][j]);
    if (NS >= 2) ga += double(mu[NS >= 2 ? 1 : 0][j]);
    ga *= wj * double(cA);
    double gb = 0.0;
    if (NS >= 3)
      gb = wj * double(cB) *
           (double(mu[NS >= 3 ? 2 : 0][j]) - double(mu[NS >= 3 ? 1 : 0][j]));
    atomicAdd(dkab + m, ga);
    if (NS >= 3) atomicAdd(dkbc + m, gb);
    if (fiber != nullptr && dw != nullptr) {
      const int f = fiber[m];
      if (f >= 0) atomicAdd(dw + f, k1 * ga - k2 * gb);
    }
  }
}

}  // namespace lbm
