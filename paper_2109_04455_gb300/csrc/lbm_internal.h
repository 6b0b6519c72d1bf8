// Internal definitions shared by the host geometry builder and the CUDA
// translation unit of liblbm.  Not part of the public C ABI (include/lbm.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

// Link word of a fluid node: nibble j-1 (j = 1..8) classifies the neighbour
// x + c_j along D2Q9 direction j.  A solid or padding node has the word
// kSolidNode and is never updated.
enum LinkType : uint32_t {
  kFluid = 0,   // fluid lattice node: plain streaming
  kWall = 1,    // channel wall beyond y = -1/2 or y = ny - 1/2
  kInert = 2,   // fiber node without a rate: bounce-back
  kCat = 3,     // fiber node with a rate: bounce-back + Dawson source
  kInlet = 4,   // beyond x = -1/2
  kOutlet = 5,  // beyond x = nx - 1/2
  kPeriodic = 6,  // fluid node across a periodic edge: plain streaming from
                  // the wrapped node (a solid node across the edge is
                  // kInert / kCat, with the wrapped node's rates)
};
constexpr uint32_t kSolidNode = 0xFFFFFFFFu;

// D2Q9, textbook numbering: c_0 = 0; c_1..4 = E, N, W, S; c_5..8 = NE, NW,
// SW, SE.
constexpr int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

inline int64_t pad32(int64_t n) { return (n + 31) / 32 * 32; }
inline size_t align256(size_t n) { return (n + 255) / 256 * 256; }

void set_error(const std::string &msg);

// True when some species' most negative concentration c_min[s] is below
// -neg_tol * max(1, c_in) (neg_tol 0 selects 0.1, < 0 disables the test).
// Estimated distance of the efficiency to its steady value from the last
// three checks (Aitken's delta-squared extrapolation of a geometric
// approach): |d2| / (1 - q), q = d2 / d1; infinite when the changes do not
// contract, unless both are below `floor` (noise of reduced precisions).
inline double eps_distance(double e1, double e2, double e3, double floor) {
  const double d1 = e2 - e1, d2 = e3 - e2;
  if (d2 == 0.0) return 0.0;
  if (d1 != 0.0) {
    const double q = d2 / d1;
    if (q >= 0.0 && q < 1.0) return (d2 < 0 ? -d2 : d2) / (1.0 - q);
  }
  const double a1 = d1 < 0 ? -d1 : d1, a2 = d2 < 0 ? -d2 : d2;
  return (a1 < floor && a2 < floor) ? (a1 > a2 ? a1 : a2) : 1e300;
}

inline bool adr_negative(const lbm_adr_params *p, const double *c_min) {
  if (p->neg_tol < 0) return false;
  const double tol = p->neg_tol > 0 ? p->neg_tol : 0.1;
  double scale = 1.0;
  for (int s = 0; s < p->nspecies; ++s)
    scale = p->c_in[s] > scale ? p->c_in[s] : scale;
  for (int s = 0; s < p->nspecies; ++s)
    if (c_min[s] < -tol * scale) return true;
  return false;
}

}  // namespace lbm

struct lbm_geometry {
  int32_t nx = 0, ny = 0, nx_pad = 0;
  int64_t n_solid = 0;
  std::vector<uint8_t> solid;     // [ny][nx]
  std::vector<double> kab, kbc;   // [ny][nx_pad]
  std::vector<uint32_t> links;    // [ny][nx_pad]
  std::vector<long long> bnodes;  // fluid nodes with a non-zero link word
  std::vector<int32_t> fiber;     // [ny][nx_pad] owning fiber, -1 elsewhere
  int32_t nfibers = 0;
  int32_t periodic = 0;           // LBM_PERIODIC_X | LBM_PERIODIC_Y
  double k1 = 0.0, k2 = 0.0;
  // device copies (borrowed from the caller's workspace after upload)
  const uint32_t *d_links = nullptr;
  const long long *d_bnodes = nullptr;
  const double *d_kab = nullptr;
  const double *d_kbc = nullptr;
  bool uploaded = false;
};
