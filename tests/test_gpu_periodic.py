"""Periodic edges (lbm_geometry_set_periodic) on the GPU path, against the
FP64 oracle's periodic modes:
* the flow lattice periodic in x and y (a decaying shear flow from the
  parabolic start);
* the ADR lattice in a box periodic in both directions with an arbitrary
  velocity field, fibers touching the edges (so catalytic links cross
  them), FP64 to 1e-10, FP32 to its float rounding;
* the node-wise variant on a fully reactive periodic lattice against the
  homogeneous closed form C_A = (1 - k1)^t;
* the discrete adjoint on a periodic lattice against the oracle's;
* the pure-diffusion cascade of Sec. IV.B (no flow, box periodic in both
  directions): oracle parity, and A + B + C conserved."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2109_04455_gb300 import inputs, lbm, series  # noqa: E402

pytestmark = pytest.mark.gpu
PXY = lbm.LBM_PERIODIC_X | lbm.LBM_PERIODIC_Y


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04455_gb300 import _build
    _build.build()
    oracle.build()
    lbm.load()


def _dev_u(ux, uy, nx_pad, dtype):
    ny, nx = ux.shape
    u = torch.zeros((2, ny, nx_pad), dtype=dtype)
    u[0, :, :nx] = torch.from_numpy(ux)
    u[1, :, :nx] = torch.from_numpy(uy)
    return u.cuda()


# fibers cut by the edges: their nodes sit next to the opposite edge's nodes
NX, NY = 75, 41
FIBERS = np.array([[1.2, 20.3, 3.0, 1, 0, -1],      # cut by x = 0
                   [37.4, 0.6, 3.5, 2, 0, -1],      # cut by y = 0
                   [72.9, 39.7, 2.5, 3, 2.1, -1],   # corner, side-by-side
                   [36.0, 22.0, 4.0, 1, 0, 0.4]])   # interior, relaxed


def _geometry(k1, k2, flags=PXY):
    return lbm.Geometry(NX, NY, FIBERS, k1, k2).set_periodic(flags).upload()


def test_periodic_flow_matches_oracle():
    solid, _, _ = oracle.raster(NX, NY, FIBERS, 0.0, 0.0)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, 300,
                                   flags=oracle.PX | oracle.PY)
    geom = _geometry(0.0, 0.0)
    u, _ = lbm.lbm_flow_solve(geom, 0.8, 0.05, 300, precision=lbm.LBM_F64)
    ug = u.cpu().numpy()[:, :, :NX]
    assert np.abs(ug[0] - ux).max() < 1e-12
    assert np.abs(ug[1] - uy).max() < 1e-12
    assert np.abs(uy).max() > 1e-4          # the fibers deflect the flow


@pytest.mark.parametrize("flags", [PXY, lbm.LBM_PERIODIC_X,
                                   lbm.LBM_PERIODIC_Y])
def test_periodic_adr_matches_oracle(flags):
    """FP64 against the oracle at 600 steps; an arbitrary velocity field
    carries populations across the periodic edges.  With only one
    direction periodic the other keeps its inlet / outlet or walls."""
    k1, k2 = 0.08, 0.05
    solid, kab, kbc = oracle.raster(NX, NY, FIBERS, k1, k2)
    rng = np.random.default_rng(5)
    ux = (0.04 * np.sin(2 * np.pi * np.arange(NY) / NY)[:, None]
          + 0.01 * rng.random((NY, NX))) * (solid == 0)
    uy = (0.03 * np.cos(2 * np.pi * np.arange(NX) / NX)[None, :]
          + 0.01 * rng.random((NY, NX))) * (solid == 0)
    oflags = (oracle.PX if flags & lbm.LBM_PERIODIC_X else 0) | \
        (oracle.PY if flags & lbm.LBM_PERIODIC_Y else 0)
    taus = [0.7, 0.62, 0.9]
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, taus, [1, 0, 0],
                             flags=oflags)
    ref = prob.run(600, xp=40)
    geom = _geometry(k1, k2, flags)
    for prec, tol in ((lbm.LBM_F64, 1e-10), (lbm.LBM_F32, 2e-5)):
        dt = torch.float64 if prec == lbm.LBM_F64 else torch.float32
        prm = lbm.adr_params(3, taus, precision=prec, max_steps=600,
                             x_plane=40)
        conc, info = lbm.lbm_adr_solve(geom, prm,
                                       _dev_u(ux, uy, geom.nx_pad, dt))
        c = conc.double().cpu().numpy()[:, :, :NX]
        rel = np.linalg.norm(c - ref["conc"]) / np.linalg.norm(ref["conc"])
        assert rel < tol, (prec, rel)
        assert np.allclose(info["flux"], ref["flux"], rtol=100 * tol,
                           atol=1e-14)
        assert np.allclose(info["mass"], np.abs(ref["conc"]).sum(axis=(1, 2)),
                           rtol=10 * tol)
    assert ref["conc"][1].max() > 1e-3 and ref["conc"][2].max() > 1e-5


@pytest.mark.parametrize("k1,k2", [(0.05, 0.02), (0.3, 0.6)])
def test_periodic_nodewise_homogeneous_closed_form(k1, k2):
    """Node-wise reactions (LBM_ADR_NODEWISE) on a periodic lattice with an
    isolated catalytic solid node at every (odd x, odd y): every fluid node
    has catalytic links of equal rates, u = 0, so the fluid state stays
    uniform and follows C_A = (1 - k1)^t,
    C_B = k1/(k2 - k1) [(1 - k1)^t - (1 - k2)^t] exactly (the oracle's own
    pin of this variant)."""
    nx, ny = 40, 24
    fib = [[x, y, 0.0, 1, 0, 0.5] for y in range(1, ny, 2)
           for x in range(1, nx, 2)]
    # relaxed weight 0.5 on every node: k_AB = k1', k_BC = k2'
    geom = lbm.Geometry(nx, ny, np.array(fib), 2 * k1, 2 * k2)
    geom.set_periodic(PXY).upload()
    n_fluid = nx * ny - geom.n_solid
    assert geom.n_solid == len(fib)
    u = torch.zeros((2, ny, geom.nx_pad), dtype=torch.float64, device="cuda")
    prm = lbm.adr_params(3, 0.9, (0, 0, 0), precision=lbm.LBM_F64,
                         flags=lbm.LBM_ADR_NODEWISE)
    sv = lbm.ADRSolver(geom, prm, u).init()
    t = 0
    for n in (2, 3, 5, 20):
        info = sv.run(n)
        t += n
        a = (1 - k1) ** t
        b = k1 / (k2 - k1) * ((1 - k1) ** t - (1 - k2) ** t)
        got = np.array(info["mass"]) / n_fluid
        assert np.allclose(got, [a, b, 1 - a - b], rtol=1e-12, atol=1e-15)


def test_periodic_adjoint_matches_oracle():
    """The discrete adjoint (gradient of eps with respect to every fiber
    node's rates) on a lattice periodic in y with inlet and outlet in x:
    links across the y edges enter the transposed streaming."""
    k1, k2 = 0.1, 0.08
    flags = lbm.LBM_PERIODIC_Y
    solid, kab, kbc = oracle.raster(NX, NY, FIBERS, k1, k2)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, 400, flags=oracle.PY)
    taus = [0.7, 0.8, 0.75]
    steps, iters = 1500, 1500
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, taus, [1, 0, 0],
                             flags=oracle.PY)
    fwd = prob.run(steps)
    adj = oracle.adjoint(prob, fwd["g"], iters)
    geom = _geometry(k1, k2, flags)
    prm = lbm.adr_params(3, taus, precision=lbm.LBM_F64)
    sv = lbm.ADRSolver(geom, prm, _dev_u(ux, uy, geom.nx_pad,
                                         torch.float64)).init()
    sv.run(steps)
    dkab, dkbc, _, info = sv.adjoint(iters, tol=0.0, check_every=iters)
    ga = dkab.cpu().numpy()[:, :NX]
    gb = dkbc.cpu().numpy()[:, :NX]
    for got, want in ((ga, adj["dkab"]), (gb, adj["dkbc"])):
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
        assert np.linalg.norm(want) > 0


def test_noflow_cascade_matches_oracle_and_conserves():
    """Sec. IV.B on a reduced box (120 x 120, fibers as in the paper's
    setups, Da = 150): 3000 steps of the GPU against the oracle (periodic in
    x and y, u = 0), and A + B + C constant at every check (no inlet, no
    outlet; the sources of each link add to zero)."""
    for kind in ("pair", "side_by_side"):
        out = series.noflow_cascade(kind, 150.0, steps=3000, every=500,
                                    n=120)
        w = out["workload"]
        tot = np.array(out["A"]) + np.array(out["B"]) + np.array(out["C"])
        assert np.abs(tot - 1.0).max() < 1e-12
        solid, kab, kbc = oracle.raster(w.nx, w.ny, w.fibers, w.k1, w.k2)
        z = np.zeros((w.ny, w.nx))
        prob = oracle.ADRProblem(solid, kab, kbc, z, z, [w.tau_c] * 3,
                                 [0, 0, 0], flags=oracle.PX | oracle.PY)
        g = prob.init()
        fluid = (solid == 0).sum()
        for i, t in enumerate(out["t"]):
            prob.steps(g, t - (out["t"][i - 1] if i else 0))
            c = prob.conc(g).sum(axis=(1, 2)) / fluid
            got = [out["A"][i], out["B"][i], out["C"][i]]
            assert np.allclose(got, c, rtol=1e-10, atol=1e-14), (kind, t)
        assert out["C"][-1] > 1e-4 and out["A"][-1] < 0.999
