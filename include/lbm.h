/*
 * liblbm -- GB300 (sm_103a) lattice-Boltzmann solver for flow and
 * advection-diffusion-reaction (ADR) through a 2D cross-section of catalytic
 * fibrous membranes (Sitaru & Gekle, "Analytical and computational study of
 * cascade reaction processes in catalytic fibrous membranes", arXiv
 * 2109.04455).
 *
 * Pipeline (Sec. III.A, the hybrid one-way scheme): geometry -> steady flow
 * (D2Q9 BGK) -> frozen velocity u -> ADR lattices for species A, B, C with
 * first-order surface reactions A->B (rate k1) and B->C (rate k2) -> outflow
 * fluxes -> efficiency (Eq. A-B).
 *
 * Conventions common to every entry point:
 *  - Every call returns an lbm_status; on failure lbm_last_error() gives a
 *    message (per calling thread).  Nothing aborts or traps.
 *  - The library never allocates device memory.  The caller allocates every
 *    device buffer, sized by the *_ws_bytes queries, and keeps it alive while
 *    a geometry or solver object refers to it.  Device pointers are at least
 *    256-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls that report numbers
 *    (lbm_flow_solve, lbm_adr_run with info, lbm_adr_solve) synchronise it.
 *  - Lattice: nodes (x, y), 0 <= x < nx (flow direction), 0 <= y < ny.  Device
 *    fields are row-major [ny][nx_pad], x contiguous, nx_pad = nx rounded up
 *    to a multiple of 32; multi-component fields put the component first
 *    ([2][ny][nx_pad] for u, [nspecies][ny][nx_pad] for concentrations).
 *    Columns x >= nx are padding (value 0 on output).
 *  - Inlet at x = -1/2, outlet at x = nx - 1/2, halfway bounce-back walls at
 *    y = -1/2 and y = ny - 1/2.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,         /* bad argument (null pointer, size, tau <= 1/2) */
  LBM_ENOMEM = 2,         /* a caller-provided workspace is too small      */
  LBM_ECUDA = 3,          /* a CUDA runtime call or kernel launch failed   */
  LBM_ENOTCONVERGED = 4,  /* max_steps reached above the tolerance          */
  LBM_EUNSTABLE = 5       /* NaN or Inf met in the residual / flux sums, or
                             (ADR) a concentration below -neg_tol           */
} lbm_status;

typedef enum {
  LBM_F64 = 0,    /* populations stored and computed in double              */
  LBM_F32 = 1,    /* populations stored and computed in float               */
  LBM_F16DEV = 2  /* populations stored in half as (g - w_i*R) * 2^14, R the
                     concentration of the storing node (itself kept in half
                     beside them); computed in float; interior populations
                     rounded stochastically (reproducible: the random bits
                     hash the node and the step).  The per-step residual
                     then has a noise floor (~6e-6 on a 2048 x 512 cascade
                     lattice), so a tol below it is not reached */
} lbm_precision;

/* Message of the last failed call on this thread ("" if none). */
const char *lbm_last_error(void);

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. II.B/II.C: fibers are infinitely long cylinders, i.e.     */
/* discs in the 2D cross-section).                                          */
/* ------------------------------------------------------------------------ */
typedef struct lbm_geometry lbm_geometry;

/* Rasterise fibers on an nx x ny lattice (host work, no GPU needed).
 * fibers: host, nfibers rows of 6 doubles: cx, cy, r, cat, janus_angle,
 *   weight.  cat 0 inert, 1 catalyses A->B (rate k1), 2 catalyses B->C
 *   (rate k2), 3 side-by-side fiber (Sec. II.C): A->B on the half where
 *   (p - c).(cos a, sin a) >= 0, B->C on the other half.  weight >= 0 on a
 *   catalytic fiber replaces that by the relaxed assignment k_AB = weight*k1,
 *   k_BC = (1 - weight)*k2 on all its nodes; use -1 for none.
 * A node is solid iff (x - cx)^2 + (y - cy)^2 <= r^2 for some fiber; the first
 * such fiber in list order sets its rates.  Needs nx >= 4 and
 * 1 <= ny <= 65535 (one grid row of blocks per lattice row).
 * On success *out owns host memory; free it with lbm_geometry_destroy. */
lbm_status lbm_geometry_create(int32_t nx, int32_t ny, const double *fibers,
                               int32_t nfibers, double k1, double k2,
                               lbm_geometry **out);
void lbm_geometry_destroy(lbm_geometry *g);

/* nx_pad and the number of solid nodes. Either pointer may be NULL. */
lbm_status lbm_geometry_info(const lbm_geometry *g, int32_t *nx_pad,
                             int64_t *n_solid);

/* Host copies of the raster: solid (ny*nx bytes, 1 = solid) and the per-node
 * rates k_AB, k_BC (ny*nx doubles each, row-major, unpadded).  Any output
 * pointer may be NULL. */
lbm_status lbm_geometry_fields(const lbm_geometry *g, uint8_t *solid,
                               double *kab, double *kbc);

/* Replace the per-node rates by host fields kab, kbc (ny*nx doubles each,
 * row-major, unpadded; either may be NULL to keep that rate): any catalyst
 * distribution over the solid nodes, e.g. one that follows the per-node
 * gradients of lbm_adr_adjoint.  Rates must be finite, >= 0 and zero on
 * fluid nodes (LBM_EINVAL otherwise, nothing changed).  The link words are
 * rebuilt (a solid node is catalytic when either rate is non-zero).  The
 * device copy is stale afterwards: call lbm_geometry_upload again (same
 * workspace size) before creating solvers; solvers created earlier keep
 * reading the device copy until that upload overwrites it.  The per-fiber
 * weight gradient of lbm_adr_adjoint assumes the relaxed assignment
 * k_AB = w k1, k_BC = (1 - w) k2; its per-node gradients hold for any
 * rates. */
lbm_status lbm_geometry_set_rates(lbm_geometry *g, const double *kab,
                                  const double *kbc);

/* Periodic edges (Sec. IV.B: the pure-diffusion cascade runs in a box that
 * is periodic in every direction, without flow).  LBM_PERIODIC_X joins the
 * x edges (no inlet and no outlet: a population leaving at x = nx - 1/2
 * enters at x = -1/2 and the reverse), LBM_PERIODIC_Y the y edges (no
 * walls).  A fiber node across an edge bounces back and reacts with its own
 * rates, as anywhere else.  Rebuilds the link words; as after
 * lbm_geometry_set_rates, upload again before creating solvers.  Flags 0
 * restores the channel (inlet, outlet, walls).  The flow lattice's inlet
 * and outlet rules then apply to no link: a periodic box has no imposed
 * flow, and an ADR solve in it is usually given u = 0. */
#define LBM_PERIODIC_X 1
#define LBM_PERIODIC_Y 2
lbm_status lbm_geometry_set_periodic(lbm_geometry *g, int32_t flags);

/* Device bytes lbm_geometry_upload needs. */
size_t lbm_geometry_ws_bytes(const lbm_geometry *g);

/* Copy the link table and the rate fields into the caller's device buffer
 * dev_ws (>= lbm_geometry_ws_bytes bytes) on `stream` and wait for the copy.
 * The geometry keeps (borrows) dev_ws for the solver calls below. */
lbm_status lbm_geometry_upload(lbm_geometry *g, void *dev_ws, size_t ws_bytes,
                               void *stream);

/* Solve calls report: */
typedef struct {
  int64_t steps;     /* time steps taken since initialisation              */
  double residual;   /* per-step relative L1 change at the last check      */
  int32_t converged; /* 1 if residual < tol at the last check              */
  double flux[3];    /* outfluxes N_A, N_B, N_C (ADR only)                  */
  double eps;        /* efficiency (ADR only; 0 if undefined)               */
  double c_min[3];   /* ADR: most negative concentration of each species at
                        the last (checked) step, 0 if none is negative.
                        The explicit scheme is not positivity preserving:
                        near tau -> 1/2 (high Pe) sharp fronts undershoot,
                        and a diverging lattice shows up here long before
                        its sums overflow                                   */
  double mass[3];    /* ADR: sum over the lattice of |C_s| at the last step
                        (the amount of each species when C_s >= 0; the
                        residual's denominator)                             */
} lbm_solve_info;

/* ------------------------------------------------------------------------ */
/* Flow: D2Q9 BGK, standing in for the paper's D3Q19 MRT flow (Sec.         */
/* III.A.1, Eq. LBE).  Pull streaming with halfway bounce-back on fibers and */
/* walls, velocity bounce-back inlet with the parabola                       */
/*   u_in(y) = 4 u0 (y + 1/2)(ny - 1/2 - y)/ny^2   (rho_w = 1)               */
/* and pressure anti-bounce-back outlet (rho_w = 1, u_w = the boundary       */
/* node's velocity).  Starts from rho = 1, u = (u_in(y), 0).                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  double tau;          /* relaxation time (> 1/2)                           */
  double u0;           /* inflow centreline velocity                        */
  int64_t max_steps;   /* step cap (or exact count when tol <= 0)           */
  double tol;          /* stop when residual < tol; <= 0: run max_steps     */
  int32_t check_every; /* steps per convergence check (>= 2)                */
  int32_t precision;   /* LBM_F64 or LBM_F32 (LBM_F16DEV runs as LBM_F32)   */
} lbm_flow_params;

size_t lbm_flow_ws_bytes(const lbm_geometry *g, int32_t precision);

/* Run the flow and write u (device, [2][ny][nx_pad], double for LBM_F64 else
 * float; 0 on solid and padding nodes) at the final step.  residual =
 * sum|u(t)-u(t-1)|_1 / sum|u(t)|_1.  Returns LBM_ENOTCONVERGED (with u and
 * info filled) when tol > 0 is not reached within max_steps. */
lbm_status lbm_flow_solve(const lbm_geometry *g, const lbm_flow_params *p,
                          void *f_ws, size_t f_ws_bytes, void *u_out,
                          void *stream, lbm_solve_info *info);

/* ------------------------------------------------------------------------ */
/* ADR lattices (Sec. III.A.2-3): per species s, BGK (Eq. BGK) towards the   */
/* second-order equilibrium with the frozen u, tau_s = 3 D_s + 1/2 (Eq.      */
/* Diffusion_LBM), C_s = sum_i g_{s,i}.  Dawson source (Eq. source_lbm) only */
/* on populations that stream into a catalytic solid node n:                 */
/*   Q_A = -k_AB(n) w_i C_A, Q_B = +k_AB(n) w_i C_A - k_BC(n) w_i C_B,       */
/*   Q_C = +k_BC(n) w_i C_B   (pre-collision C at the fluid node).           */
/* Boundaries (Eq. BC): fibers and walls bounce-back; inlet anti-bounce-back */
/* g = -g* + 2 w_i c_in for species A (bounce-back for B, C unless           */
/* LBM_ADR_INLET_ABB_ALL); outlet anti-bounce-back with C_w = sum_j g*_j of   */
/* the boundary node.  All species advance in one kernel pass per step.      */
/* Start: C_A = 1 on fluid nodes, B = C = 0, g = g^eq.                       */
/* Outflux (Sec. III.A.3): N_s = (1/ny) sum_y sum_i c_ix g*_{s,i}(x_plane,y) */
/* of the post-collision populations, accumulated in double.                  */
/* ------------------------------------------------------------------------ */
#define LBM_ADR_INLET_ABB_ALL 1 /* anti-bounce-back inlet for every species */
/* Reaction variant the paper compares the link-wise source with (Fig.      */
/* node_vs_pop): a fluid node with at least one link into a catalytic solid */
/* node reacts on all nine populations, Q_i = w_i (-k_AB C_A, ...), with     */
/* k_AB, k_BC the means of the rates over those links.  Not differentiable  */
/* by lbm_adr_adjoint (LBM_EINVAL).                                          */
#define LBM_ADR_NODEWISE 2

typedef struct {
  int32_t nspecies;    /* 1 (A only), 2 (A->B) or 3 (A->B->C)               */
  int32_t precision;   /* lbm_precision                                     */
  double tau[3];       /* relaxation time per species (> 1/2)               */
  double c_in[3];      /* inlet concentration per species (A: 1)            */
  int64_t max_steps;   /* lbm_adr_solve: step cap (exact count if tol <= 0) */
  double tol;          /* lbm_adr_solve: stop when residual < tol           */
  int32_t check_every; /* lbm_adr_solve: steps per check (>= 2)             */
  int32_t x_plane;     /* flux plane; < 0 selects nx - 3                    */
  int32_t flags;       /* LBM_ADR_* bits                                    */
  double neg_tol;      /* checked steps report LBM_EUNSTABLE when some C_s
                          < -neg_tol * max(1, c_in[0..nspecies)); 0 selects
                          0.1, < 0 turns the test off (c_min is reported
                          either way)                                        */
  double eps_tol;      /* lbm_adr_solve / lbm_batch_solve, > 0: a lattice
                          converges only when, besides residual < tol, the
                          distance of its efficiency to the steady value is
                          estimated below eps_tol: Aitken's delta-squared
                          extrapolation of the last three checks, e1, e2,
                          e3 with d1 = e2 - e1, d2 = e3 - e2 and
                          q = d2 / d1 in [0, 1), gives |d2| / (1 - q)
                          (changes that do not contract count as not
                          converged unless both are below eps_tol / 10,
                          the noise of reduced precisions).  A per-step
                          residual alone is a poor steady-state test where
                          diffusion dominates (low Pe).  <= 0: off         */
} lbm_adr_params;

/* Device bytes of the ADR workspace (two population buffers, the
 * concentration scratch and the reduction partials). */
size_t lbm_adr_ws_bytes(const lbm_geometry *g, const lbm_adr_params *p);

typedef struct lbm_adr_solver lbm_adr_solver;

/* Bind a solver to an uploaded geometry, the device velocity u ([2][ny]
 * [nx_pad], double for LBM_F64 else float) and a workspace ws.  Host object
 * only; nothing runs on the GPU. */
lbm_status lbm_adr_create(const lbm_geometry *g, const lbm_adr_params *p,
                          const void *u, void *ws, size_t ws_bytes,
                          lbm_adr_solver **out);
void lbm_adr_destroy(lbm_adr_solver *s);

/* Set the initial state (C_A = 1, others 0, g = g^eq) and steps = 0. */
lbm_status lbm_adr_init(lbm_adr_solver *s, void *stream);

/* Advance nsteps time steps.  info == NULL: enqueue only (no host sync).
 * info != NULL (nsteps >= 2): the last two steps also record C, the
 * residual (its per-node terms summed in double), the amount of each
 * species and the most negative concentration at the last step, the
 * outflux on the plane is reduced, the stream is synchronised and info is
 * filled; LBM_EUNSTABLE (info still filled) if a sum is not finite or a
 * concentration is below -neg_tol (see lbm_adr_params). */
lbm_status lbm_adr_run(lbm_adr_solver *s, int64_t nsteps, void *stream,
                       lbm_solve_info *info);

/* Copy C_s at the last checked step (device, [nspecies][ny][nx_pad], double
 * for LBM_F64 else float) to conc_out. */
lbm_status lbm_adr_conc(lbm_adr_solver *s, void *conc_out, void *stream);

/* One-shot solve: create, init, run in chunks of check_every until
 * residual < tol (or exactly max_steps if tol <= 0), copy C to conc_out
 * (may be NULL), destroy.  LBM_ENOTCONVERGED if tol was not reached. */
lbm_status lbm_adr_solve(const lbm_geometry *g, const lbm_adr_params *p,
                         const void *u, void *ws, size_t ws_bytes,
                         void *conc_out, void *stream, lbm_solve_info *info);

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of the ADR lattice: gradient of the efficiency (Eq. A-B) */
/* with respect to the per-node rates k_AB, k_BC of the fiber nodes, and to  */
/* relaxed per-fiber catalyst weights w_f (k_AB = w_f k1, k_BC = (1-w_f) k2) */
/* through the chain rule.  The frozen-flow ADR step is affine in the state, */
/* g*(t+1) = K (P g*(t) + b) (P: pull and link rules, K: per-node collision  */
/* and the Dawson source of Eq. source_lbm), so the adjoint of the           */
/* pre-collision populations solves nu = K^T (P^T nu + l), l = d eps/d g* on */
/* the flux plane; it is iterated from nu = 0 with the transposed (gather)    */
/* stream-collide.  Then d eps/dk(n) = sum over the links x -> n of          */
/* mu^T dK/dk g, mu = P^T nu + l.  Not in the paper: it differentiates the   */
/* paper's discrete scheme.                                                   */
/* ------------------------------------------------------------------------ */

/* Checkpoint / resume (no counterpart in the paper): the populations of the
 * current state (and, for LBM_F16DEV, the half reference concentrations)
 * are the whole state of a run.  lbm_adr_state_save copies them, behind a
 * header (lattice size, species count, precision, step count), into the
 * caller's host buffer of >= lbm_adr_state_bytes bytes (pinned or pageable)
 * and waits for the copy; LBM_ENOMEM if the buffer is smaller.
 * lbm_adr_state_load copies a saved state into a solver created for the same
 * geometry size, species count and precision (LBM_EINVAL otherwise, nothing
 * changed) and restores the step count, so that continuing from it gives
 * bit for bit the run that was saved (the stochastic rounding of
 * LBM_F16DEV is seeded by the step count).  The loaded state has no
 * recorded concentrations: run with info before lbm_adr_conc or the
 * adjoint. */
size_t lbm_adr_state_bytes(const lbm_adr_solver *s);
lbm_status lbm_adr_state_save(lbm_adr_solver *s, void *host, size_t bytes,
                              void *stream);
lbm_status lbm_adr_state_load(lbm_adr_solver *s, const void *host,
                              size_t bytes, void *stream);

/* Device bytes of the adjoint workspace (LBM_F64 or LBM_F32 precision). */
size_t lbm_adr_adjoint_ws_bytes(const lbm_geometry *g, const lbm_adr_params *p);

/* Adjoint at the solver's current state, which must come from a run with
 * info (lbm_adr_run / lbm_adr_solve loop) so that its concentrations are
 * recorded; precision LBM_F64 or LBM_F32 (populations and adjoint alike).
 * Iterates max_steps times (tol <= 0) or in chunks of check_every until the
 * relative L1 change of nu per iteration is below tol.  Outputs (device,
 * zeroed first, accumulated in double): dkab, dkbc [ny][nx_pad] (non-zero on
 * fiber nodes only), dw [nfibers] (may be NULL).  info: iterations, adjoint
 * residual, converged, and the forward outfluxes and efficiency used. */
lbm_status lbm_adr_adjoint(lbm_adr_solver *s, int64_t max_steps, double tol,
                           int32_t check_every, void *ws, size_t ws_bytes,
                           void *dkab, void *dkbc, void *dw, void *stream,
                           lbm_solve_info *info);

/* ------------------------------------------------------------------------ */
/* Batched ADR solves (a Pe x Da sweep over many lattices of uneven size).  */
/* Every active lattice advances in the same persistent launch per time     */
/* step (interior row tiles and boundary-node chunks of all lattices in one */
/* work list); a check interval (check_every steps, the last two recording  */
/* the residual, then the per-lattice sums and outfluxes) is captured once  */
/* as a CUDA graph and replayed; a lattice leaves the work list once its    */
/* residual is below its tol or it reached its max_steps.  The per-node     */
/* arithmetic is that of lbm_adr_solve, so each lattice's result equals its */
/* unbatched solve.  The launch shape (tile width 128 or 256, persistent    */
/* grid size) is chosen by timing the candidates on the batch.              */
/* ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

/* Device bytes for `count` lattices (all with the same nspecies, 2 or 3, and
 * the same precision); 0 if the arguments are invalid. */
size_t lbm_batch_ws_bytes(int32_t count, const lbm_geometry *const *geoms,
                          const lbm_adr_params *params);

/* geoms[i] uploaded, params[i] its ADR settings (tol, max_steps and x_plane
 * per lattice; check_every of params[0] for all, rounded up to even; a
 * lattice runs whole check intervals, so max_steps is rounded up to a
 * multiple of it; tol <= 0 runs exactly that many steps),
 * u[i] its device velocity.  ws holds every lattice's populations. */
lbm_status lbm_batch_create(int32_t count, const lbm_geometry *const *geoms,
                            const lbm_adr_params *params,
                            const void *const *u, void *ws, size_t ws_bytes,
                            lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);

/* Time the launch-shape candidates on this batch and keep the fastest
 * (tile width in *tile, blocks in *grid; either may be NULL).  Runs by
 * itself on the first lbm_batch_solve. */
lbm_status lbm_batch_tune(lbm_batch *b, void *stream, int32_t *tile,
                          int32_t *grid);

/* The chosen launch shape and the measured ms per step of the candidates
 * (tile 128 then 256, grids 1, 2, 4, 8 x resident blocks; 8 floats). */
lbm_status lbm_batch_tuning(const lbm_batch *b, int32_t *tile, int32_t *grid,
                            float *ms_per_step);

/* Solve every lattice from its initial state; infos[count] receives steps,
 * residual, converged, outfluxes, efficiency and c_min per lattice.  A
 * lattice whose sums go non-finite or whose concentration falls below
 * -neg_tol stops there (LBM_EUNSTABLE overall, the others run on).
 * LBM_ENOTCONVERGED if any lattice stopped at max_steps. */
lbm_status lbm_batch_solve(lbm_batch *b, void *stream, lbm_solve_info *infos);

/* Concentrations of lattice `index` at its last checked step (after
 * lbm_batch_solve: its final state), copied to conc_out (device,
 * [nspecies][ny][nx_pad] of that lattice, double for LBM_F64 else float)
 * on `stream`.  LBM_EINVAL for a bad index or before any solve. */
lbm_status lbm_batch_conc(const lbm_batch *b, int32_t index, void *conc_out,
                          void *stream);

/* ------------------------------------------------------------------------ */
/* Random walk particle tracking (Sec. III.B), the paper's second method for */
/* the efficiency of a 2D cross-section.  Per time step dt (the paper: 0.5)  */
/* a particle moves by dt u(x) (u bilinear in the LBM velocity field, nodes  */
/* at integer positions, indices clamped to the lattice) and by a step of    */
/* length sqrt(4 D dt) in a uniformly random direction; it reflects          */
/* elastically off the walls y = -1/2, ny - 1/2 and off every fiber (a disc  */
/* of radius R + radius_offset: 0.5 puts the surface where the LBM's halfway */
/* bounce-back puts it); within the reactive shell of width delta (the       */
/* paper: 0.2) around a catalytic fiber it reacts with probability k dt      */
/* (A -> B at the fiber's k_AB, B -> C at its k_BC; side-by-side fibers by    */
/* side, relaxed weights as in lbm_geometry_create; the first fiber in list  */
/* order whose shell holds the particle decides; one reaction per step).     */
/* The entrance strip x in [-1/2, 1/2) is held at `density` particles of A   */
/* per unit area: each step the A particles that end there are removed and  */
/* the strip seeded anew; A crossing x = -1/2 returns to that reservoir, B   */
/* and C reflect there.  A particle crossing x = nx - 1/2 leaves and counts  */
/* for its species; eps follows Eq. (A-B) from these counts.  Random numbers */
/* come from per-particle SplitMix64 streams (draw k of particle `id` at     */
/* step t: output 64 t + k + 1 of the stream seeded by output id + 1 of the  */
/* stream of `seed`), and every arithmetic step is one IEEE operation, so a  */
/* run is reproducible bit for bit whatever the storage order.               */
/* ------------------------------------------------------------------------ */
#define LBM_RWPT_PERIODIC 1    /* box periodic in x and y: no inlet, outlet,
                                  walls or entrance strip (positions wrap)   */
#define LBM_RWPT_HOMOGENEOUS 2 /* every particle reacts with k1 dt (A) and
                                  k2 dt (B) per step wherever it is (the
                                  homogeneous-reaction check of Appendix C)  */
typedef struct {
  double D;              /* diffusivity                                      */
  double dt;             /* time step                                        */
  double delta;          /* reactive shell width                             */
  double density;        /* particles per unit area: entrance strip and the
                            initial fill of the box with A                   */
  double radius_offset;  /* reflecting radius = R + radius_offset            */
  uint64_t seed;
  int32_t nspecies;      /* 1, 2 or 3                                        */
  int32_t flags;         /* LBM_RWPT_* bits                                  */
} lbm_rwpt_params;

typedef struct {
  int64_t steps;         /* steps since lbm_rwpt_init                        */
  int64_t window_steps;  /* steps since the counts were last reset           */
  int64_t alive;         /* particles in the box                             */
  int64_t out[3];        /* particles of A, B, C that left through the outlet
                            in the window                                    */
  double eps;            /* Eq. (A-B) from out[] (0 if undefined)            */
  int32_t overflow;      /* 1 if the capacity was exceeded (LBM_ENOMEM)      */
} lbm_rwpt_info;

typedef struct lbm_rwpt lbm_rwpt;

/* Device bytes for `capacity` particles and `nfibers` fibers. */
size_t lbm_rwpt_ws_bytes(int64_t capacity, int32_t nfibers);

/* Bind a particle system to a channel of nx x ny nodes, a fiber table (host,
 * rows of 6 doubles as in lbm_geometry_create, with rates k1 and k2 per
 * unit time), the device velocity u ([2][ny][nx_pad] double, or NULL for no
 * flow) and the workspace ws.  LBM_EINVAL for k dt > 1. */
lbm_status lbm_rwpt_create(int32_t nx, int32_t ny, const double *fibers,
                           int32_t nfibers, double k1, double k2,
                           const lbm_rwpt_params *p, const void *u,
                           int64_t capacity, void *ws, size_t ws_bytes,
                           lbm_rwpt **out);
void lbm_rwpt_destroy(lbm_rwpt *r);

/* Fill the box with A at the density (none inside the fibers), step 0,
 * counts 0. */
lbm_status lbm_rwpt_init(lbm_rwpt *r, void *stream);

/* Advance nsteps steps (no host synchronisation when info is NULL);
 * with info, synchronise and report.  LBM_ENOMEM if the capacity was ever
 * exceeded (the surplus particles were dropped). */
lbm_status lbm_rwpt_run(lbm_rwpt *r, int64_t nsteps, void *stream,
                        lbm_rwpt_info *info);

/* Zero the outlet counts and start a new window. */
lbm_status lbm_rwpt_reset_counts(lbm_rwpt *r, void *stream);

/* Copy the particles (in storage order, which varies from run to run) to
 * host arrays of max_count entries; *count receives their number
 * (LBM_ENOMEM if it exceeds max_count). */
lbm_status lbm_rwpt_particles(lbm_rwpt *r, void *stream, int64_t max_count,
                              int64_t *count, double *x, double *y,
                              int32_t *species, uint64_t *id);

/* Eq. (A-B): eps = N_B/(N_A+N_B) for nspecies 2, N_C/(N_A+N_B+N_C) for 3.
 * Host arithmetic only.  LBM_EINVAL for other nspecies or a zero sum. */
lbm_status lbm_efficiency(const double *flux, int32_t nspecies, double *eps);

/* Double-precision FMA throughput of the current device in TFLOP/s (2 flops
 * per FMA), measured by a short kernel of independent FMA chains (best of
 * three timed launches after a warm-up, a few ms in all; synchronises
 * `stream`).  No counterpart in the paper: it is the measured denominator of
 * the FP64 step's roofline, since that step is bound by the FP64 pipe. */
lbm_status lbm_fp64_fma_tflops(void *stream, double *tflops);

/* Outfluxes N_s on the plane x_plane (< 0 selects nx - 3) of the solver's
 * current state, written to flux_out (host, 3 doubles; 0 for absent
 * species), without any device workspace.  The paper has no counterpart:
 * this serves callers that cannot allocate device memory where they need
 * the fluxes, such as a monitor or plugin inside an application whose own
 * memory pool has reserved the whole GPU (a cudaMalloc would fail or
 * fragment it), or a time-critical loop that must not pay cudaMalloc's
 * implicit device synchronisation.  Its partial sums live in a fixed 6 KB
 * device array that every GPU loading this library holds until the process
 * exits; it covers at most 65536 lattice rows, and a larger ny is rejected
 * with LBM_EINVAL.  Every call looks up that array's device address on the
 * solver's device (cudaGetSymbolAddress, which allocates nothing), so the
 * address stays right after a device reset; the call synchronises `stream`,
 * so it is not for use inside a stream capture.  All calls share the one
 * array and it keeps the last call's values (each call rewrites every slot
 * it reads, so nothing needs clearing); calls whose GPU work overlaps
 * (other streams or threads) race on it and must be serialised by the
 * caller. */
lbm_status lbm_adr_outflux_noalloc(lbm_adr_solver *s, int32_t x_plane,
                                   void *stream, double *flux_out);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
