/*
 * Plain FP64 CPU oracle for the lattice-Boltzmann flow + advection-diffusion-
 * reaction (ADR) method of Sitaru & Gekle, "Analytical and computational study
 * of cascade reaction processes in catalytic fibrous membranes".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the GPU path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product library
 * never links, loads or calls it, and it shares no code with it.
 *
 * Formulation (deliberately different from the GPU path): array-of-structures
 * populations f[(y*nx + x)*9 + i], collide-then-PUSH streaming with two
 * arrays, boundary rules applied where a pushed population would leave the
 * fluid.  Every step follows the paper in its own order:
 *   Sec. III.A.2  Eq. (LBE_ADE), Eq. (BGK), the second-order equilibrium,
 *                 Eq. (Diffusion_LBM) D = c_s^2 (tau - 1/2), C = sum_i g_i,
 *                 Eq. (source_lbm) Dawson source applied only to populations
 *                 that stream into a reactive (catalytic solid) node.
 *   Sec. III.A.3  Eq. (BC) anti-bounce-back at inlet (C_w = 1 for A) and
 *                 outlet (C_w = C_b); bounce-back elsewhere; outflux on the
 *                 plane two nodes before the outlet.
 *   Sec. II.A     Eq. (A-B): efficiency from the outflow fluxes (in Python).
 * The flow lattice (D2Q9 BGK, velocity inlet, pressure outlet, bounce-back
 * walls and fibers) replaces the paper's D3Q19 MRT body-force flow of
 * Sec. III.A.1 by a 2D cross-section with inflow/outflow.
 *
 * Velocity set (textbook D2Q9 numbering): c_0 = (0,0); c_1..c_4 = (1,0),
 * (0,1), (-1,0), (0,-1); c_5..c_8 = (1,1), (-1,1), (-1,-1), (1,-1).
 * Weights 4/9, 1/9, 1/36; c_s^2 = 1/3.
 *
 * Compile: gcc -O2 -ffp-contract=off -fPIC -shared -fopenmp (no fused
 * multiply-add, so every product and sum is rounded exactly as written).
 * The time steps split the lattice rows over OpenMP threads; every node's
 * update is independent and each output slot is written by exactly one
 * node, so the result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q9 9

static const int CX[Q9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[Q9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[Q9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* boundary-mode flags */
#define ORC_PX 1            /* periodic in x (no inlet / outlet)             */
#define ORC_PY 2            /* periodic in y (no top / bottom walls)         */
#define ORC_ALLPOP 4        /* every population at a fluid node reacts with
                               the node's own rates (homogeneous reaction)   */
#define ORC_INLET_ABB_ALL 8 /* every species, not only A, gets the inlet
                               anti-bounce-back with its own c_in            */
#define ORC_NODEWISE 16     /* a fluid node with a link into a catalytic
                               solid node reacts on all its populations, with
                               the mean rates of those links (the variant the
                               paper compares against in Fig. node_vs_pop)   */

/* Second-order equilibrium of Sec. III.A.2 for density/concentration c. */
static double equilibrium(int i, double c, double ux, double uy) {
  double cu = CX[i] * ux + CY[i] * uy;
  double uu = ux * ux + uy * uy;
  return W[i] * c *
         (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Parabolic inflow profile with its zeros half a node outside rows 0 and
 * ny-1 (halfway walls); centreline value u0. */
static double inflow_u(int y, int ny, double u0) {
  double yy = (double)y;
  return 4.0 * u0 * (yy + 0.5) * ((double)ny - 0.5 - yy) /
         ((double)ny * (double)ny);
}

/* ------------------------------------------------------------------------ */
/* Geometry: fibers are discs of the 2D cross-section.                      */
/* fib holds 6 doubles per fiber: cx, cy, r, cat, janus_angle, weight.      */
/* cat 0 inert, 1 catalyses A->B (rate k1), 2 catalyses B->C (rate k2),     */
/* 3 side-by-side: A->B on the half where (p-c).n(angle) >= 0, B->C on the  */
/* other half.  weight >= 0 (for cat != 0) replaces the assignment by the   */
/* relaxed catalyst k_AB = weight*k1, k_BC = (1-weight)*k2.                 */
/* A node is solid iff its squared distance to some centre is <= r^2; the   */
/* first fiber in list order that contains it decides its rates.            */
/* ------------------------------------------------------------------------ */
int orc_raster(int nx, int ny, int nfib, const double *fib, double k1,
               double k2, uint8_t *solid, double *kab, double *kbc) {
  if (nx <= 0 || ny <= 0 || nfib < 0) return 1;
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      long n = (long)y * nx + x;
      solid[n] = 0;
      kab[n] = 0.0;
      kbc[n] = 0.0;
      for (int f = 0; f < nfib; ++f) {
        const double *p = fib + 6 * f;
        double dx = (double)x - p[0];
        double dy = (double)y - p[1];
        if (dx * dx + dy * dy <= p[2] * p[2]) {
          int cat = (int)p[3];
          solid[n] = 1;
          if (cat != 0 && p[5] >= 0.0) {
            kab[n] = p[5] * k1;
            kbc[n] = (1.0 - p[5]) * k2;
          } else if (cat == 1) {
            kab[n] = k1;
          } else if (cat == 2) {
            kbc[n] = k2;
          } else if (cat == 3) {
            if (dx * cos(p[4]) + dy * sin(p[4]) >= 0.0)
              kab[n] = k1;
            else
              kbc[n] = k2;
          }
          break;
        }
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Flow lattice (D2Q9 BGK).                                                 */
/* ------------------------------------------------------------------------ */

/* f = f^eq(rho, u) on fluid nodes, 0 on solid nodes. */
void orc_flow_init_fields(int nx, int ny, const uint8_t *solid,
                          const double *rho, const double *ux,
                          const double *uy, double *f) {
  for (long n = 0; n < (long)nx * ny; ++n)
    for (int i = 0; i < Q9; ++i)
      f[n * Q9 + i] = solid[n] ? 0.0 : equilibrium(i, rho[n], ux[n], uy[n]);
}

/* Channel start: rho = 1 and the inflow parabola on every fluid node. */
void orc_flow_init_channel(int nx, int ny, const uint8_t *solid, double u0,
                           double *f) {
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      long n = (long)y * nx + x;
      double ux = solid[n] ? 0.0 : inflow_u(y, ny, u0);
      for (int i = 0; i < Q9; ++i)
        f[n * Q9 + i] = solid[n] ? 0.0 : equilibrium(i, 1.0, ux, 0.0);
    }
}

/* rho, u from pre-collision populations (0 on solid nodes). */
void orc_flow_moments(int nx, int ny, const uint8_t *solid, const double *f,
                      double *rho, double *ux, double *uy) {
  for (long n = 0; n < (long)nx * ny; ++n) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    if (!solid[n]) {
      for (int i = 0; i < Q9; ++i) {
        r += f[n * Q9 + i];
        jx += CX[i] * f[n * Q9 + i];
        jy += CY[i] * f[n * Q9 + i];
      }
    }
    rho[n] = r;
    ux[n] = solid[n] ? 0.0 : jx / r;
    uy[n] = solid[n] ? 0.0 : jy / r;
  }
}

/* One flow time step: BGK collision, then push streaming.
 *   inlet  (population leaving through x = -1/2): velocity bounce-back
 *          f_opp = f* - 2 w rho_w (c.u_w)/c_s^2, rho_w = 1, u_w = (u_in(y),0)
 *   outlet (leaving through x = nx-1/2): pressure anti-bounce-back
 *          f_opp = -f* + 2 w rho_w [1 + (c.u_w)^2/(2c_s^4) - u_w^2/(2c_s^2)],
 *          rho_w = 1, u_w = u of the boundary node at this time step
 *   wall / fiber: halfway bounce-back f_opp = f*.
 * The x-boundary rule wins over the wall rule on corner links. */
static void flow_step(int nx, int ny, const uint8_t *solid, double tau,
                      double u0, int flags, const double *f, double *fn) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      long n = (long)y * nx + x;
      if (solid[n]) continue;
      const double *fp = f + n * Q9;
      double rho = 0.0, jx = 0.0, jy = 0.0;
      for (int i = 0; i < Q9; ++i) {
        rho += fp[i];
        jx += CX[i] * fp[i];
        jy += CY[i] * fp[i];
      }
      double ux = jx / rho, uy = jy / rho;
      double fs[Q9];
      for (int i = 0; i < Q9; ++i)
        fs[i] = fp[i] - (fp[i] - equilibrium(i, rho, ux, uy)) / tau;
      for (int i = 0; i < Q9; ++i) {
        int tx = x + CX[i], ty = y + CY[i];
        int io = OPP[i];
        if (tx < 0 || tx >= nx) {
          if (flags & ORC_PX) {
            tx = (tx + nx) % nx;
          } else if (tx < 0) {
            double cu = CX[i] * inflow_u(y, ny, u0);
            fn[n * Q9 + io] = fs[i] - 2.0 * W[i] * 1.0 * cu / CS2;
            continue;
          } else {
            double cu = CX[i] * ux + CY[i] * uy;
            double uu = ux * ux + uy * uy;
            fn[n * Q9 + io] =
                -fs[i] + 2.0 * W[i] * 1.0 *
                             (1.0 + cu * cu / (2.0 * CS2 * CS2) -
                              uu / (2.0 * CS2));
            continue;
          }
        }
        if (ty < 0 || ty >= ny) {
          if (flags & ORC_PY) {
            ty = (ty + ny) % ny;
          } else {
            fn[n * Q9 + io] = fs[i];
            continue;
          }
        }
        long t = (long)ty * nx + tx;
        if (solid[t])
          fn[n * Q9 + io] = fs[i];
        else
          fn[t * Q9 + i] = fs[i];
      }
    }
  }
}

/* nsteps flow steps in place on f (ftmp is scratch of the same size). */
int orc_flow_steps(int nx, int ny, const uint8_t *solid, double tau, double u0,
                   int flags, long nsteps, double *f, double *ftmp) {
  if (tau <= 0.5) return 1;
  long nn = (long)nx * ny * Q9;
  memset(ftmp, 0, sizeof(double) * nn);
  double *a = f, *b = ftmp;
  for (long s = 0; s < nsteps; ++s) {
    flow_step(nx, ny, solid, tau, u0, flags, a, b);
    double *t = a;
    a = b;
    b = t;
  }
  if (a != f) memcpy(f, a, sizeof(double) * nn);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* ADR lattice: ns species (1 = A, 2 = A,B, 3 = A,B,C).                      */
/* g holds ns blocks of nx*ny*9 doubles (species-major, then node, then i). */
/* ------------------------------------------------------------------------ */

/* g = g^eq(c0, u) on fluid nodes, 0 on solid nodes. */
void orc_adr_init(int nx, int ny, int ns, const uint8_t *solid,
                  const double *ux, const double *uy, const double *c0,
                  double *g) {
  long nn = (long)nx * ny;
  for (int s = 0; s < ns; ++s)
    for (long n = 0; n < nn; ++n)
      for (int i = 0; i < Q9; ++i)
        g[(s * nn + n) * Q9 + i] =
            solid[n] ? 0.0 : equilibrium(i, c0[s * nn + n], ux[n], uy[n]);
}

/* C_s = sum_i g_{s,i} (pre-collision). */
void orc_adr_conc(int nx, int ny, int ns, const uint8_t *solid,
                  const double *g, double *c) {
  long nn = (long)nx * ny;
  for (int s = 0; s < ns; ++s)
    for (long n = 0; n < nn; ++n) {
      double acc = 0.0;
      if (!solid[n])
        for (int i = 0; i < Q9; ++i) acc += g[(s * nn + n) * Q9 + i];
      c[s * nn + n] = acc;
    }
}

/* Post-collision populations gs[s][i] at fluid node (x, y):
 *   g* = g - (g - g^eq(C, u)) / tau_s + Q,
 * with the Dawson source (Eq. source_lbm) on the populations that stream
 * into a solid lattice node (rates of that node):
 *   Q_A = -k_AB w C_A,  Q_B = +k_AB w C_A - k_BC w C_B,  Q_C = +k_BC w C_B,
 * all concentrations taken before collision at this node and time.  With
 * ORC_ALLPOP every population reacts with the node's own rates instead.
 * With ORC_NODEWISE a node with at least one link into a catalytic solid
 * node (non-zero k_AB or k_BC) reacts on every population i = 0..8, with
 * k_AB, k_BC the means over those links. */
static void adr_collide(int nx, int ny, int ns, const uint8_t *solid,
                        const double *kab, const double *kbc, double ux,
                        double uy, const double *tau, int flags, int x, int y,
                        const double *g, double gs[3][Q9]) {
  long nn = (long)nx * ny;
  long n = (long)y * nx + x;
  double c[3] = {0.0, 0.0, 0.0};
  for (int s = 0; s < ns; ++s)
    for (int i = 0; i < Q9; ++i) c[s] += g[(s * nn + n) * Q9 + i];
  for (int s = 0; s < ns; ++s)
    for (int i = 0; i < Q9; ++i) {
      double gi = g[(s * nn + n) * Q9 + i];
      gs[s][i] = gi - (gi - equilibrium(i, c[s], ux, uy)) / tau[s];
    }
  if (flags & ORC_NODEWISE) {
    double sa = 0.0, sb = 0.0;
    int ncat = 0;
    for (int i = 1; i < Q9; ++i) {
      int tx = x + CX[i], ty = y + CY[i];
      if (tx < 0 || tx >= nx) {
        if (!(flags & ORC_PX)) continue;
        tx = (tx + nx) % nx;
      }
      if (ty < 0 || ty >= ny) {
        if (!(flags & ORC_PY)) continue;
        ty = (ty + ny) % ny;
      }
      long t = (long)ty * nx + tx;
      if (!solid[t] || (kab[t] == 0.0 && kbc[t] == 0.0)) continue;
      sa += kab[t];
      sb += kbc[t];
      ++ncat;
    }
    if (ncat == 0) return;
    double ka = sa / ncat, kb = sb / ncat;
    for (int i = 0; i < Q9; ++i) {
      double ra = ka * W[i] * c[0];
      double rb = (ns >= 3) ? kb * W[i] * c[1] : 0.0;
      gs[0][i] -= ra;
      if (ns >= 2) gs[1][i] += ra - rb;
      if (ns >= 3) gs[2][i] += rb;
    }
    return;
  }
  for (int i = 0; i < Q9; ++i) {
    double ka = 0.0, kb = 0.0;
    if (flags & ORC_ALLPOP) {
      ka = kab[n];
      kb = kbc[n];
    } else {
      if (i == 0) continue;
      int tx = x + CX[i], ty = y + CY[i];
      if (tx < 0 || tx >= nx) {
        if (!(flags & ORC_PX)) continue; /* inlet / outlet: not a fiber */
        tx = (tx + nx) % nx;
      }
      if (ty < 0 || ty >= ny) {
        if (!(flags & ORC_PY)) continue; /* channel wall: not a fiber */
        ty = (ty + ny) % ny;
      }
      long t = (long)ty * nx + tx;
      if (!solid[t]) continue;
      ka = kab[t];
      kb = kbc[t];
    }
    double ra = ka * W[i] * c[0];
    double rb = (ns >= 3) ? kb * W[i] * c[1] : 0.0;
    gs[0][i] -= ra;
    if (ns >= 2) gs[1][i] += ra - rb;
    if (ns >= 3) gs[2][i] += rb;
  }
}

/* One ADR step: collision + source, then push streaming with
 *   inlet : anti-bounce-back g_opp = -g* + 2 w c_in  for species 0 (and for
 *           every species with ORC_INLET_ABB_ALL), else bounce-back g_opp = g*
 *   outlet: anti-bounce-back g_opp = -g* + 2 w C_b, C_b = sum_j g*_j of the
 *           boundary node (equal to its concentration when it has no
 *           catalytic link)
 *   wall / fiber: bounce-back g_opp = g* (the source is already inside g*). */
static void adr_step(int nx, int ny, int ns, const uint8_t *solid,
                     const double *kab, const double *kbc, const double *ux,
                     const double *uy, const double *tau, const double *cin,
                     int flags, const double *g, double *gn) {
  long nn = (long)nx * ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    double gs[3][Q9];
    for (int x = 0; x < nx; ++x) {
      long n = (long)y * nx + x;
      if (solid[n]) continue;
      adr_collide(nx, ny, ns, solid, kab, kbc, ux[n], uy[n], tau, flags, x, y,
                  g, gs);
      for (int s = 0; s < ns; ++s) {
        double cb = 0.0;
        for (int i = 0; i < Q9; ++i) cb += gs[s][i];
        double *out = gn + s * nn * Q9;
        for (int i = 0; i < Q9; ++i) {
          int tx = x + CX[i], ty = y + CY[i];
          int io = OPP[i];
          if (tx < 0 || tx >= nx) {
            if (flags & ORC_PX) {
              tx = (tx + nx) % nx;
            } else if (tx < 0) {
              if (s == 0 || (flags & ORC_INLET_ABB_ALL))
                out[n * Q9 + io] = -gs[s][i] + 2.0 * W[i] * cin[s];
              else
                out[n * Q9 + io] = gs[s][i];
              continue;
            } else {
              out[n * Q9 + io] = -gs[s][i] + 2.0 * W[i] * cb;
              continue;
            }
          }
          if (ty < 0 || ty >= ny) {
            if (flags & ORC_PY) {
              ty = (ty + ny) % ny;
            } else {
              out[n * Q9 + io] = gs[s][i];
              continue;
            }
          }
          long t = (long)ty * nx + tx;
          if (solid[t])
            out[n * Q9 + io] = gs[s][i];
          else
            out[t * Q9 + i] = gs[s][i];
        }
      }
    }
  }
}

int orc_adr_steps(int nx, int ny, int ns, const uint8_t *solid,
                  const double *kab, const double *kbc, const double *ux,
                  const double *uy, const double *tau, const double *cin,
                  int flags, long nsteps, double *g, double *gtmp) {
  if (ns < 1 || ns > 3) return 1;
  for (int s = 0; s < ns; ++s)
    if (tau[s] <= 0.5) return 1;
  long nt = (long)ns * nx * ny * Q9;
  memset(gtmp, 0, sizeof(double) * nt);
  double *a = g, *b = gtmp;
  for (long k = 0; k < nsteps; ++k) {
    adr_step(nx, ny, ns, solid, kab, kbc, ux, uy, tau, cin, flags, a, b);
    double *t = a;
    a = b;
    b = t;
  }
  if (a != g) memcpy(g, a, sizeof(double) * nt);
  return 0;
}

/* Outflux on the plane x = xp (Sec. III.A.3): per node the post-collision
 * populations moving right minus those moving left, summed over the plane
 * and divided by ny (the average over the plane's nodes).  flux[s] = N_s. */
void orc_adr_flux(int nx, int ny, int ns, const uint8_t *solid,
                  const double *kab, const double *kbc, const double *ux,
                  const double *uy, const double *tau, int flags,
                  const double *g, int xp, double *flux) {
  double gs[3][Q9];
  for (int s = 0; s < ns; ++s) flux[s] = 0.0;
  for (int y = 0; y < ny; ++y) {
    long n = (long)y * nx + xp;
    if (solid[n]) continue;
    adr_collide(nx, ny, ns, solid, kab, kbc, ux[n], uy[n], tau, flags, xp, y,
                g, gs);
    for (int s = 0; s < ns; ++s)
      for (int i = 0; i < Q9; ++i) flux[s] += CX[i] * gs[s][i];
  }
  for (int s = 0; s < ns; ++s) flux[s] /= (double)ny;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of the ADR lattice (frozen u).                          */
/*                                                                          */
/* The step is affine in the pre-collision state: g' = P(K g) + b, with K    */
/* the per-node collision + source (linear in g) and P the push streaming    */
/* with its boundary rules (b holds the constant inlet terms).  The          */
/* efficiency depends on the post-collision populations g* = K g on the      */
/* flux plane through the outfluxes N_s; dNds[s] = d eps / d N_s.            */
/* At the steady state the adjoint of the pre-collision state solves         */
/*   nu = K^T (P^T nu + l),   l_{s,i}(x) = dNds[s] c_ix / ny on the plane,   */
/* iterated here from nu = 0.  mu = P^T nu + l is then the adjoint of g*,    */
/* and a rate k of solid node n enters only through the source of the links  */
/* x -> n, so                                                                 */
/*   d eps/d k_AB(n) = sum_{x + c_j = n} w_j C_A(x) (mu_{B,j} - mu_{A,j})(x) */
/*   d eps/d k_BC(n) = sum_{x + c_j = n} w_j C_B(x) (mu_{C,j} - mu_{B,j})(x) */
/* (for one species only the -mu_A term; without C only the A, B terms).     */
/* ------------------------------------------------------------------------ */

/* mu = P^T nu + l at fluid node (x, y) for species s: each post-collision
 * population went to exactly one place in the forward push; its adjoint is
 * read back from there. */
static void adj_gather(int nx, int ny, int ns, const uint8_t *solid, int flags,
                       const double *dNds, int xp, int s, int x, int y,
                       const double *nu, double mu[Q9]) {
  long nn = (long)nx * ny;
  long n = (long)y * nx + x;
  const double *v = nu + s * nn * Q9;
  for (int i = 0; i < Q9; ++i) mu[i] = 0.0;
  for (int i = 0; i < Q9; ++i) {
    int tx = x + CX[i], ty = y + CY[i];
    int io = OPP[i];
    if (tx < 0 || tx >= nx) {
      if (flags & ORC_PX) {
        tx = (tx + nx) % nx;
      } else if (tx < 0) {
        /* inlet: g_opp = -g* + const (anti-bounce-back) or g_opp = g* */
        if (s == 0 || (flags & ORC_INLET_ABB_ALL))
          mu[i] += -v[n * Q9 + io];
        else
          mu[i] += v[n * Q9 + io];
        continue;
      } else {
        /* outlet: g_opp = -g*_i + 2 w_i sum_j g*_j */
        mu[i] += -v[n * Q9 + io];
        for (int j = 0; j < Q9; ++j) mu[j] += 2.0 * W[i] * v[n * Q9 + io];
        continue;
      }
    }
    if (ty < 0 || ty >= ny) {
      if (flags & ORC_PY) {
        ty = (ty + ny) % ny;
      } else {
        mu[i] += v[n * Q9 + io];
        continue;
      }
    }
    long t = (long)ty * nx + tx;
    if (solid[t])
      mu[i] += v[n * Q9 + io];
    else
      mu[i] += v[t * Q9 + i];
  }
  if (x == xp)
    for (int i = 0; i < Q9; ++i) mu[i] += dNds[s] * CX[i] / (double)ny;
}

/* Rates of the solid node that direction i of fluid node (x, y) points to
 * (0 if it points to fluid, a wall, the inlet or the outlet). */
static int link_rates(int nx, int ny, const uint8_t *solid, const double *kab,
                      const double *kbc, int flags, int x, int y, int i,
                      double *ka, double *kb, long *target) {
  int tx = x + CX[i], ty = y + CY[i];
  *ka = 0.0;
  *kb = 0.0;
  if (tx < 0 || tx >= nx) {
    if (!(flags & ORC_PX)) return 0;
    tx = (tx + nx) % nx;
  }
  if (ty < 0 || ty >= ny) {
    if (!(flags & ORC_PY)) return 0;
    ty = (ty + ny) % ny;
  }
  long t = (long)ty * nx + tx;
  if (!solid[t]) return 0;
  *ka = kab[t];
  *kb = kbc[t];
  *target = t;
  return 1;
}

/* nu <- K^T (P^T nu + l), nsteps times. */
int orc_adr_adjoint_steps(int nx, int ny, int ns, const uint8_t *solid,
                          const double *kab, const double *kbc,
                          const double *ux, const double *uy,
                          const double *tau, int flags, const double *dNds,
                          int xp, long nsteps, double *nu, double *tmp) {
  if (ns < 1 || ns > 3 || (flags & (ORC_ALLPOP | ORC_NODEWISE))) return 1;
  long nn = (long)nx * ny;
  long nt = (long)ns * nn * Q9;
  memset(tmp, 0, sizeof(double) * nt);
  double *a = nu, *b = tmp;
  for (long step = 0; step < nsteps; ++step) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
      double mu[3][Q9];
      for (int x = 0; x < nx; ++x) {
        long n = (long)y * nx + x;
        if (solid[n]) continue;
        for (int s = 0; s < ns; ++s)
          adj_gather(nx, ny, ns, solid, flags, dNds, xp, s, x, y, a, mu[s]);
        /* K^T: g*_{s,i} = g_{s,i} - (g_{s,i} - C_s e_i)/tau_s + Q_{s,i}(C),
         * e_i = equilibrium(i, 1, u), C_s = sum_m g_{s,m}. */
        double cross[3] = {0.0, 0.0, 0.0}; /* sum_{s,i} mu_{s,i} dQ_{s,i}/dC_s' */
        for (int i = 1; i < Q9; ++i) {
          double ka, kb;
          long t;
          if (!link_rates(nx, ny, solid, kab, kbc, flags, x, y, i, &ka, &kb,
                          &t))
            continue;
          /* dQ_A/dC_A = -ka w, dQ_B/dC_A = +ka w, dQ_B/dC_B = -kb w,
           * dQ_C/dC_B = +kb w (the B->C terms only with three species) */
          cross[0] += -ka * W[i] * mu[0][i];
          if (ns >= 2) cross[0] += ka * W[i] * mu[1][i];
          if (ns >= 3) {
            cross[1] += -kb * W[i] * mu[1][i];
            cross[1] += kb * W[i] * mu[2][i];
          }
        }
        for (int s = 0; s < ns; ++s) {
          double feq_part = 0.0; /* sum_i mu_i (1/tau) e_i */
          for (int i = 0; i < Q9; ++i)
            feq_part += mu[s][i] * equilibrium(i, 1.0, ux[n], uy[n]) / tau[s];
          for (int m = 0; m < Q9; ++m)
            b[(s * nn + n) * Q9 + m] =
                mu[s][m] * (1.0 - 1.0 / tau[s]) + feq_part + cross[s];
        }
      }
    }
    double *t = a;
    a = b;
    b = t;
  }
  if (a != nu) memcpy(nu, a, sizeof(double) * nt);
  return 0;
}

/* Gradient of eps with respect to the rates of every solid node, from the
 * pre-collision steady state g and the adjoint nu (see above). */
void orc_adr_gradient(int nx, int ny, int ns, const uint8_t *solid,
                      const double *kab, const double *kbc, const double *ux,
                      const double *uy, const double *tau, int flags,
                      const double *dNds, int xp, const double *g,
                      const double *nu, double *dkab, double *dkbc) {
  long nn = (long)nx * ny;
  double mu[3][Q9];
  (void)ux;
  (void)uy;
  (void)tau;
  for (long n = 0; n < nn; ++n) {
    dkab[n] = 0.0;
    dkbc[n] = 0.0;
  }
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      long n = (long)y * nx + x;
      if (solid[n]) continue;
      double c[3] = {0.0, 0.0, 0.0};
      for (int s = 0; s < ns; ++s) {
        for (int i = 0; i < Q9; ++i) c[s] += g[(s * nn + n) * Q9 + i];
        adj_gather(nx, ny, ns, solid, flags, dNds, xp, s, x, y, nu, mu[s]);
      }
      for (int i = 1; i < Q9; ++i) {
        double ka, kb;
        long t;
        if (!link_rates(nx, ny, solid, kab, kbc, flags, x, y, i, &ka, &kb, &t))
          continue;
        double da = -mu[0][i];
        if (ns >= 2) da += mu[1][i];
        dkab[t] += W[i] * c[0] * da;
        if (ns >= 3) dkbc[t] += W[i] * c[1] * (mu[2][i] - mu[1][i]);
      }
    }
  }
}

/* Index of the fiber that owns each node (first in list order), -1 fluid. */
void orc_fiber_ids(int nx, int ny, int nfib, const double *fib, int32_t *ids) {
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      long n = (long)y * nx + x;
      ids[n] = -1;
      for (int f = 0; f < nfib; ++f) {
        const double *p = fib + 6 * f;
        double dx = (double)x - p[0];
        double dy = (double)y - p[1];
        if (dx * dx + dy * dy <= p[2] * p[2]) {
          ids[n] = f;
          break;
        }
      }
    }
}

/* Threads the time steps use (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
