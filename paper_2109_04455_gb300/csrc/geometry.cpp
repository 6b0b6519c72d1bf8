// Host-side geometry: fiber raster, per-node reaction rates and the per-node
// link words read by the GPU kernels.
//
// Fibers are infinitely long cylinders, i.e. discs in the 2D cross-section
// (paper Sec. II.B/II.C).  Compiled with -ffp-contract=off so the disc test
// rounds the same way on every host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "lbm_internal.h"

using namespace lbm;

namespace {

// Link words of the fluid nodes (nibble j-1: type of the neighbour x + c_j,
// a solid neighbour being catalytic when either of its rates is non-zero),
// the boundary-node list and the solid count.  Across a periodic edge the
// neighbour is the wrapped node (kPeriodic when it is fluid); otherwise the
// x edges are the inlet and the outlet (their rule wins on corner links) and
// the y edges walls.
void build_links(lbm_geometry *g) {
  const int64_t nx = g->nx, ny = g->ny;
  const bool px = (g->periodic & LBM_PERIODIC_X) != 0;
  const bool py = (g->periodic & LBM_PERIODIC_Y) != 0;
  g->links.assign(static_cast<size_t>(g->nx_pad) * ny, kSolidNode);
  g->bnodes.clear();
  int64_t nsol = 0;
  for (int64_t y = 0; y < ny; ++y) {
    for (int64_t x = 0; x < nx; ++x) {
      const int64_t n = y * g->nx_pad + x;
      if (g->solid[y * nx + x]) {
        ++nsol;
        continue;  // stays kSolidNode
      }
      uint32_t word = 0;
      for (int j = 1; j < 9; ++j) {
        int64_t tx = x + kCx[j], ty = y + kCy[j];
        bool wrapped = false;
        uint32_t t = kFluid;
        if ((tx < 0 || tx >= nx) && !px) {
          t = tx < 0 ? kInlet : kOutlet;
        } else {
          if (tx < 0 || tx >= nx) {
            tx = (tx + nx) % nx;
            wrapped = true;
          }
          if ((ty < 0 || ty >= ny) && !py) {
            t = kWall;
          } else {
            if (ty < 0 || ty >= ny) {
              ty = (ty + ny) % ny;
              wrapped = true;
            }
            if (g->solid[ty * nx + tx]) {
              const int64_t m = ty * g->nx_pad + tx;
              t = (g->kab[m] != 0.0 || g->kbc[m] != 0.0) ? kCat : kInert;
            } else {
              t = wrapped ? kPeriodic : kFluid;
            }
          }
        }
        word |= t << (4 * (j - 1));
      }
      g->links[n] = word;
      if (word != 0u) g->bnodes.push_back(n);
    }
  }
  g->n_solid = nsol;
}

}  // namespace

extern "C" lbm_status lbm_geometry_create(int32_t nx, int32_t ny,
                                          const double *fibers,
                                          int32_t nfibers, double k1,
                                          double k2, lbm_geometry **out) {
  if (!out) {
    set_error("lbm_geometry_create: out is NULL");
    return LBM_EINVAL;
  }
  *out = nullptr;
  if (nx < 4 || ny < 1 || ny > 65535 || nfibers < 0 ||
      (nfibers > 0 && !fibers)) {
    set_error(
        "lbm_geometry_create: need nx >= 4, 1 <= ny <= 65535, fibers != NULL");
    return LBM_EINVAL;
  }
  if (!(k1 >= 0.0) || !(k2 >= 0.0)) {
    set_error("lbm_geometry_create: rates must be >= 0");
    return LBM_EINVAL;
  }
  lbm_geometry *g = new (std::nothrow) lbm_geometry;
  if (!g) {
    set_error("lbm_geometry_create: host allocation failed");
    return LBM_ENOMEM;
  }
  try {
    g->nx = nx;
    g->ny = ny;
    g->nx_pad = static_cast<int32_t>(pad32(nx));
    const int64_t np = static_cast<int64_t>(g->nx_pad) * ny;
    g->solid.assign(static_cast<size_t>(nx) * ny, 0);
    g->kab.assign(np, 0.0);
    g->kbc.assign(np, 0.0);
    g->links.assign(np, kSolidNode);
    g->fiber.assign(np, -1);
    g->nfibers = nfibers;
    g->k1 = k1;
    g->k2 = k2;

    // Raster fiber by fiber over its bounding box; a node keeps the first
    // fiber (in list order) that contains it.
    for (int32_t f = 0; f < nfibers; ++f) {
      const double *p = fibers + 6 * static_cast<int64_t>(f);
      const double cx = p[0], cy = p[1], r = p[2], ang = p[4], w = p[5];
      const int cat = static_cast<int>(p[3]);
      if (!(r >= 0.0) || cat < 0 || cat > 3 || !std::isfinite(cx) ||
          !std::isfinite(cy)) {
        set_error("lbm_geometry_create: bad fiber row " + std::to_string(f));
        delete g;
        return LBM_EINVAL;
      }
      const double ca = std::cos(ang), sa = std::sin(ang);
      const int64_t x0 = std::max<int64_t>(0, (int64_t)std::floor(cx - r));
      const int64_t x1 = std::min<int64_t>(nx - 1, (int64_t)std::ceil(cx + r));
      const int64_t y0 = std::max<int64_t>(0, (int64_t)std::floor(cy - r));
      const int64_t y1 = std::min<int64_t>(ny - 1, (int64_t)std::ceil(cy + r));
      for (int64_t y = y0; y <= y1; ++y) {
        for (int64_t x = x0; x <= x1; ++x) {
          uint8_t &s = g->solid[y * nx + x];
          if (s) continue;
          const double dx = static_cast<double>(x) - cx;
          const double dy = static_cast<double>(y) - cy;
          if (!(dx * dx + dy * dy <= r * r)) continue;
          s = 1;
          const int64_t n = y * g->nx_pad + x;
          double a = 0.0, b = 0.0;
          if (cat != 0 && w >= 0.0) {
            a = w * k1;
            b = (1.0 - w) * k2;
          } else if (cat == 1) {
            a = k1;
          } else if (cat == 2) {
            b = k2;
          } else if (cat == 3) {
            if (dx * ca + dy * sa >= 0.0)
              a = k1;
            else
              b = k2;
          }
          g->kab[n] = a;
          g->kbc[n] = b;
          g->fiber[n] = f;
        }
      }
    }

    build_links(g);
  } catch (const std::bad_alloc &) {
    delete g;
    set_error("lbm_geometry_create: host allocation failed");
    return LBM_ENOMEM;
  }
  *out = g;
  return LBM_OK;
}

extern "C" void lbm_geometry_destroy(lbm_geometry *g) { delete g; }

extern "C" lbm_status lbm_geometry_info(const lbm_geometry *g, int32_t *nx_pad,
                                        int64_t *n_solid) {
  if (!g) {
    set_error("lbm_geometry_info: geometry is NULL");
    return LBM_EINVAL;
  }
  if (nx_pad) *nx_pad = g->nx_pad;
  if (n_solid) *n_solid = g->n_solid;
  return LBM_OK;
}

extern "C" lbm_status lbm_geometry_fields(const lbm_geometry *g,
                                          uint8_t *solid, double *kab,
                                          double *kbc) {
  if (!g) {
    set_error("lbm_geometry_fields: geometry is NULL");
    return LBM_EINVAL;
  }
  if (solid) std::memcpy(solid, g->solid.data(), g->solid.size());
  for (int64_t y = 0; y < g->ny; ++y)
    for (int64_t x = 0; x < g->nx; ++x) {
      const int64_t n = y * g->nx_pad + x;
      if (kab) kab[y * g->nx + x] = g->kab[n];
      if (kbc) kbc[y * g->nx + x] = g->kbc[n];
    }
  return LBM_OK;
}

extern "C" lbm_status lbm_geometry_set_rates(lbm_geometry *g,
                                             const double *kab,
                                             const double *kbc) {
  if (!g) {
    set_error("lbm_geometry_set_rates: geometry is NULL");
    return LBM_EINVAL;
  }
  for (int k = 0; k < 2; ++k) {
    const double *f = k == 0 ? kab : kbc;
    if (!f) continue;
    for (int64_t y = 0; y < g->ny; ++y)
      for (int64_t x = 0; x < g->nx; ++x) {
        const double v = f[y * g->nx + x];
        if (!(v >= 0.0) || !std::isfinite(v) ||
            (v != 0.0 && !g->solid[y * g->nx + x])) {
          set_error("lbm_geometry_set_rates: rates must be finite, >= 0, "
                    "and zero on fluid nodes");
          return LBM_EINVAL;
        }
      }
  }
  try {
    for (int64_t y = 0; y < g->ny; ++y)
      for (int64_t x = 0; x < g->nx; ++x) {
        const int64_t n = y * g->nx_pad + x;
        if (kab) g->kab[n] = kab[y * g->nx + x];
        if (kbc) g->kbc[n] = kbc[y * g->nx + x];
      }
    build_links(g);
  } catch (const std::bad_alloc &) {
    set_error("lbm_geometry_set_rates: host allocation failed");
    return LBM_ENOMEM;
  }
  g->uploaded = false;   // the device copy is stale until the next upload
  return LBM_OK;
}

extern "C" lbm_status lbm_geometry_set_periodic(lbm_geometry *g,
                                                int32_t flags) {
  if (!g || (flags & ~(LBM_PERIODIC_X | LBM_PERIODIC_Y))) {
    set_error("lbm_geometry_set_periodic: NULL geometry or unknown flags");
    return LBM_EINVAL;
  }
  try {
    g->periodic = flags;
    build_links(g);
  } catch (const std::bad_alloc &) {
    set_error("lbm_geometry_set_periodic: host allocation failed");
    return LBM_ENOMEM;
  }
  g->uploaded = false;   // the device copy is stale until the next upload
  return LBM_OK;
}

extern "C" lbm_status lbm_efficiency(const double *flux, int32_t nspecies,
                                     double *eps) {
  if (!flux || !eps) {
    set_error("lbm_efficiency: NULL pointer");
    return LBM_EINVAL;
  }
  double den = 0.0, num = 0.0;
  if (nspecies == 2) {
    num = flux[1];
    den = flux[0] + flux[1];
  } else if (nspecies == 3) {
    num = flux[2];
    den = flux[0] + flux[1] + flux[2];
  } else {
    set_error("lbm_efficiency: nspecies must be 2 or 3");
    return LBM_EINVAL;
  }
  if (den == 0.0) {
    set_error("lbm_efficiency: zero total outflux");
    return LBM_EINVAL;
  }
  *eps = num / den;
  return LBM_OK;
}
