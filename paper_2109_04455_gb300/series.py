"""The paper's 2D experiment series, run on the batched lattice solver.

* Isolated A->B fiber (Sec. II.B: R = 5 in the middle of a 300 x 300 box):
  efficiency against Pe, next to the collision-zone model of Sec. IV.A.
* A->B->C cascade (Sec. II.C, 1000 x 300 box, Da = 150) on two R = 5 fibers
  whose surfaces are xi apart along the flow, and on one side-by-side R = 10
  fiber; the model of Sec. IV.B for fibers far apart is the product of the
  two single-fiber efficiencies.
* Membranes of n = 6 random R = 5 fibers (2D analogue of Sec. IV, three
  seeds): one A->B membrane (Da = 150, 1.5) against Eq. (eff_memb), and an
  A->B membrane followed by a B->C membrane (Da = 150) against
  Eq. (eff_ABC_memb), the square of the membrane efficiency.
* Production rate of the final species (Appendix A).

The inflow velocity u0 is fixed and Pe is set through D (so the flow depends
only on the geometry): each geometry's flow is solved once, in FP64, and
shared by all of its Pe values.  Every ADR lattice of one species count then
advances in one lbm_batch.  Pe values whose rate k = Da D / R^2 reaches 1 per
time step are left out (the explicit source empties a node in one step), and
so are those whose tau_c = 3 D + 1/2 falls below 0.52 (with u0 = 0.05 the BGK
advection-diffusion lattice goes unstable there: Pe = 100 at R = 5 gives
tau_c = 0.5075 and a non-finite state).
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs, lbm


# ---------------------------------------------------------------------------
# collision-zone model (Sec. IV.A)
# ---------------------------------------------------------------------------
def collision_zone(pe: float, r: float) -> float:
    """Width d of the collision zone: positive root of Eq. (d),
    d^2 / (2D) - (pi / u0) d - pi R / u0 = 0, written with Pe = u0 R / D:
    d = R (pi/Pe + sqrt(pi^2/Pe^2 + 2 pi/Pe))."""
    a = math.pi / pe
    return r * (a + math.sqrt(a * a + 2.0 * math.pi / pe))


def model_efficiency(pe: float, da: float, r: float, width: float,
                     shell: float = 0.5) -> float:
    """Eq. (eps): eps = eps_coll (1 - exp(-k alpha t_D)) with
    eps_coll = d / (2 l) (half the molecules of the collision zone diffuse
    towards the fiber, l the channel width; capped at 1), t_D = d^2 / (2D),
    alpha = ((R + shell)^2 - R^2) / ((R + d)^2 - R^2) (the ratio of the
    reaction shell's area to the collision zone's), k = Da D / R^2.  The
    product k alpha t_D = Da alpha d^2 / (2 R^2) does not depend on u0."""
    d = collision_zone(pe, r)
    eps_coll = min(1.0, 0.5 * d / width)
    alpha = ((r + shell) ** 2 - r * r) / ((r + d) ** 2 - r * r)
    return eps_coll * (1.0 - math.exp(-da * alpha * d * d / (2.0 * r * r)))


def membrane_model(pe: float, da: float, r: float, width: float, n: int,
                   shell: float = 0.5) -> float:
    """Eq. (eff_memb): each of the n fibers of a membrane converts the share
    eps of what the fibers before it left, so
    eps_mem = sum_{i=1..n} eps (1 - eps)^(i-1) = 1 - (1 - eps)^n, with eps
    the isolated-fiber model of Eq. (eps)."""
    e = model_efficiency(pe, da, r, width, shell)
    return 1.0 - (1.0 - e) ** n


def production_rate(flux, ny: int, nspecies: int) -> float:
    """Appendix A: final product leaving the reactor per time step (per unit
    fiber length), N_final * ny with N_s the plane-averaged outflux."""
    return float(flux[nspecies - 1]) * ny


# ---------------------------------------------------------------------------
# the series
# ---------------------------------------------------------------------------
DEFAULT_PE = (1.0, 2.0, 3.0, 5.0, 7.0, 10.0, 20.0, 30.0)
TAU_MIN = 0.52
# efficiency against Da at fixed Pe (Sec. IV.A, Fig. singleAB_Da)
DA_SERIES_PE = (1.0, 7.0, 20.0)
DA_SERIES = tuple(float(v) for v in np.logspace(-1, 3, 9))


def da_workloads(pes=DA_SERIES_PE, das=DA_SERIES):
    """The isolated A->B fiber at Pe = 1, 7, 20 over Da = 0.1 .. 1000 (the
    values with k = Da D / R^2 < 1 per step)."""
    out = [("isolated_fiber", inputs.isolated_fiber(pe, da))
           for pe in pes for da in das]
    return [(k, w) for k, w in out
            if max(w.k1, w.k2) < 1.0 and w.tau_c >= TAU_MIN]


def workloads(pes=DEFAULT_PE, xis=(2.0, 20.0, 100.0),
              das_isolated=(150.0, 1.5), membrane_seeds=(0, 1, 2)):
    """(geometry key, workload) pairs of the series with k < 1 and
    tau_c >= TAU_MIN."""
    out = []
    for seed in membrane_seeds:
        for da in das_isolated:
            for pe in pes:
                out.append((f"membrane_AB_seed{seed}",
                            inputs.fiber_membrane(pe, da, seed)))
        for pe in pes:
            out.append((f"membrane_cascade_seed{seed}",
                        inputs.fiber_membrane(pe, 150.0, seed, cascade=True)))
    for da in das_isolated:
        for pe in pes:
            out.append(("isolated_fiber", inputs.isolated_fiber(pe, da)))
    for xi in xis:
        for pe in pes:
            out.append((f"fiber_pair_xi{xi:g}", inputs.fiber_pair(xi, pe)))
    for pe in pes:
        out.append(("side_by_side", inputs.side_by_side_fiber(pe)))
    return [(k, w) for k, w in out
            if max(w.k1, w.k2) < 1.0 and w.tau_c >= TAU_MIN]


def solve_flows(items, flow_tol: float = 1e-9, flow_max: int = 400000,
                device="cuda"):
    """FP64 flow of each distinct geometry key; returns {key: u}."""
    flows = {}
    for key, w in items:
        if key in flows:
            continue
        g = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload(device)
        u, info = lbm.lbm_flow_solve(g, w.tau_flow, w.u0, flow_max,
                                     tol=flow_tol, check_every=1000,
                                     precision=lbm.LBM_F64)
        flows[key] = (u, info)
    return flows


def run(items=None, flows=None, precision: int = lbm.LBM_F32,
        tol: float = 1e-6, max_steps: int = 200000, check_every: int = 1000,
        device="cuda", flags: int = 0):
    """Steady efficiencies of the series.  Returns (rows, batches): one dict
    per lattice (geometry key, Pe, Da, eps, model eps where the paper gives
    one, production rate, steps, converged) and the Batch objects' launch
    shapes.  flags: LBM_ADR_* bits for every lattice (LBM_ADR_NODEWISE: the
    node-wise reaction the paper compares with in Fig. node_vs_pop)."""
    items = workloads() if items is None else items
    flows = solve_flows(items, device=device) if flows is None else flows
    rows = []
    shapes = []
    for ns in (2, 3):
        sel = [(k, w) for k, w in items if w.nspecies == ns]
        if not sel:
            continue
        geoms, params, us = [], [], []
        for key, w in sel:
            geoms.append(lbm.Geometry(w.nx, w.ny, w.fibers, w.k1,
                                      w.k2).upload(device))
            params.append(lbm.adr_params(ns, w.tau_c, w.c_in,
                                         precision=precision,
                                         max_steps=max_steps, tol=tol,
                                         check_every=check_every,
                                         flags=flags))
            u = flows[key][0]
            us.append(u if precision == lbm.LBM_F64 else u.float())
        b = lbm.Batch(geoms, params, us, device)
        shapes.append(b.tune())
        infos = b.solve()
        b.close()
        for (key, w), info in zip(sel, infos):
            row = {"geometry": key, "pe": w.pe, "da": w.da1,
                   "nx": w.nx, "ny": w.ny, "nspecies": ns,
                   "eps": info["eps"], "flux": info["flux"][:ns],
                   "production_rate": production_rate(info["flux"], w.ny, ns),
                   "steps": info["steps"], "converged": info["converged"],
                   "residual": info["residual"]}
            if key == "isolated_fiber":
                row["model_eps"] = model_efficiency(w.pe, w.da1, w.r_ref,
                                                    float(w.ny))
            elif key.startswith("membrane_"):
                n = w.fibers.shape[0] // (2 if ns == 3 else 1)
                em = membrane_model(w.pe, w.da1, w.r_ref, float(w.ny), n)
                row["model_eps"] = em if ns == 2 else em * em
            rows.append(row)
    # Eq. (eps_ABC) for the pairs: the square of one fiber's efficiency,
    # stated for fibers whose collision zones do not overlap (xi > 2d)
    for row, (key, w) in zip(rows, [it for ns in (2, 3) for it in items
                                    if it[1].nspecies == ns]):
        if key.startswith("fiber_pair"):
            xi = w.fibers[1, 0] - w.fibers[0, 0] - 2.0 * w.r_ref
            e1 = model_efficiency(w.pe, w.da1, w.r_ref, float(w.ny))
            row["xi"] = float(xi)
            row["model_eps"] = e1 * e1
            row["model_applies"] = bool(xi > 2.0 * collision_zone(w.pe,
                                                                  w.r_ref))
    return rows, shapes


# ---------------------------------------------------------------------------
# pure-diffusion cascade (Sec. IV.B, Figs. noflow and noflow_k001)
# ---------------------------------------------------------------------------
def noflow_cascade(kind: str, da: float, steps: int = 200000,
                   every: int = 1000, precision: int = lbm.LBM_F64,
                   n: int = 300, device="cuda"):
    """Total amounts of A, B and C over time in the periodic box of
    inputs.noflow_box (start: C_A = 1 on every fluid node, u = 0), each as a
    fraction of the fluid nodes.  Returns a dict with the time points, the
    three curves and the workload."""
    import torch
    w = inputs.noflow_box(kind, da, n=n)
    g = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2)
    g.set_periodic(lbm.LBM_PERIODIC_X | lbm.LBM_PERIODIC_Y).upload(device)
    fluid = w.nx * w.ny - g.n_solid
    dtype = torch.float64 if precision == lbm.LBM_F64 else torch.float32
    u = torch.zeros((2, w.ny, g.nx_pad), dtype=dtype, device=g.ws.device)
    prm = lbm.adr_params(3, w.tau_c, (0.0, 0.0, 0.0), precision=precision)
    sv = lbm.ADRSolver(g, prm, u).init()
    t, curves = [], [[], [], []]
    done = 0
    while done < steps:
        info = sv.run(every)
        done += every
        t.append(done)
        for s in range(3):
            curves[s].append(info["mass"][s] / fluid)
    sv.close()
    return {"t": t, "A": curves[0], "B": curves[1], "C": curves[2],
            "workload": w, "k1": w.k1, "k2": w.k2, "tau_c": w.tau_c}


def as_table(rows) -> np.ndarray:
    """(geometry index, Pe, Da, eps) as an array, for plotting."""
    keys = sorted({r["geometry"] for r in rows})
    return np.array([[keys.index(r["geometry"]), r["pe"], r["da"], r["eps"]]
                     for r in rows])
