"""The adjoint as configured for the two-membrane cascade lattice (2048 x 512,
80 fibers, Pe = 10, Da1 = Da2 = 1) with relaxed catalyst weights
(k_AB = w_f k1, k_BC = (1 - w_f) k2 on every node of fiber f):
* FP64 populations: d eps/d w_f projected on a random direction over 16
  random fibers against the central difference (h = 1e-2) of two FP64
  steady solves warm-started from the base state's checkpoint, to 1e-3
  relative;
* FP32 populations with FP64 flux and residual sums: the FP32 steady state
  and its adjoint (FP64's iteration count) give d eps/d w within 1e-3
  (relative L2 over every fiber) of FP64's, and each of the 16 fibers'
  d eps/d w_f within 1e-3 relative;
* against the oracle's own FP64 adjoint at this size at equal step and
  iteration counts (per-node gradients of every fiber node, 1e-10).
(Per-fiber central differences at h = 1e-4 need longer, fixed solves: a
solve stopped by the per-step residual leaves a fraction of so small a
perturbation unrelaxed; bench.py --workload adjoint-check runs them.)"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
from paper_2109_04455_gb300 import inputs, lbm  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04455_gb300 import _build
    _build.build()
    oracle.build()
    lbm.load()


def _cascade():
    w = inputs.two_membrane_cascade(seed=0, pe=10.0)
    fib = w.fibers.copy()
    # relaxed weights inside (0, 1) so that both signs of a step are valid
    fib[:, 5] = np.where(fib[:, 3] == 1, 0.9, 0.1)
    return w, fib


def _steady(w, fib, u, tol, prec=lbm.LBM_F64, start=None):
    geom = lbm.Geometry(w.nx, w.ny, fib, w.k1, w.k2).upload()
    prm = lbm.adr_params(3, w.tau_c, precision=prec)
    sv = lbm.ADRSolver(geom, prm, u).init()
    if start is not None:
        sv.state_load(start)
    info = sv.solve(tol, 1000, 1000000)
    assert info["converged"], info
    return geom, sv, info


def test_cascade_adjoint_f64_and_f32():
    w, fib = _cascade()
    nf = fib.shape[0]
    geom0 = lbm.Geometry(w.nx, w.ny, fib, w.k1, w.k2).upload()
    u, finfo = lbm.lbm_flow_solve(geom0, w.tau_flow, w.u0, 400000, tol=1e-10,
                                  check_every=1000, precision=lbm.LBM_F64)
    assert finfo["converged"]
    _, sv, info = _steady(w, fib, u, 1e-12)
    base = sv.state_save()
    _, _, dw, ainfo = sv.adjoint(1000000, tol=1e-12, check_every=1000,
                                 nfibers=nf)
    assert ainfo["converged"] and ainfo["eps"] == info["eps"]
    dw = dw.cpu().numpy()
    rng = np.random.default_rng(4)
    pick = rng.choice(nf, 16, replace=False)
    v = np.zeros(nf)
    v[pick] = rng.standard_normal(16)
    v /= np.linalg.norm(v)
    h = 1e-2
    eps = []
    for sgn in (1.0, -1.0):
        fb = fib.copy()
        fb[:, 5] += sgn * h * v
        eps.append(_steady(w, fb, u, 1e-12, start=base)[2]["eps"])
    fd = (eps[0] - eps[1]) / (2 * h)
    ad = float(dw @ v)
    assert abs(fd) > 1e-3 * np.abs(dw).max()      # a non-trivial direction
    assert ad == pytest.approx(fd, rel=1e-3)
    # FP32 populations, FP64 sums
    _, sv32, _ = _steady(w, fib, u.float(), 1e-7, prec=lbm.LBM_F32)
    _, _, dw32, _ = sv32.adjoint(ainfo["steps"], tol=0.0,
                                 check_every=ainfo["steps"], nfibers=nf)
    dw32 = dw32.cpu().numpy()
    assert np.linalg.norm(dw32 - dw) < 1e-3 * np.linalg.norm(dw)
    assert np.allclose(dw32[pick], dw[pick], rtol=1e-3, atol=0)


def test_cascade_adjoint_matches_oracle_at_equal_counts():
    """Forward 1200 steps and 1200 adjoint iterations from nu = 0 on both
    sides, with the oracle's own flow (2000 steps), efficiency on the plane
    x = 720 just behind the first membrane (the adjoint starts there and
    reaches that membrane's fibers within these iterations): the per-node
    gradients with respect to k_AB and k_BC of every fiber node agree to
    1e-10 (relative L2), and the weight gradients to 1e-9."""
    w, fib = _cascade()
    nsteps, nit, nflow, xp = 1200, 1200, 2000, 720
    solid, kab, kbc = oracle.raster(w.nx, w.ny, fib, w.k1, w.k2)
    _, ux, uy, _ = oracle.flow_run(solid, w.tau_flow, w.u0, nflow)
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, [w.tau_c] * 3,
                             [1, 0, 0])
    fwd = prob.run(nsteps, xp=xp)
    ref = oracle.adjoint(prob, fwd["g"], nit, xp=xp)
    ids = oracle.fiber_ids(w.nx, w.ny, fib)
    dw_ref = oracle.fiber_weight_gradient(ids, ref["dkab"], ref["dkbc"],
                                          w.k1, w.k2, fib.shape[0])
    geom = lbm.Geometry(w.nx, w.ny, fib, w.k1, w.k2).upload()
    ud = torch.zeros((2, w.ny, geom.nx_pad), dtype=torch.float64)
    ud[0, :, :w.nx] = torch.from_numpy(ux)
    ud[1, :, :w.nx] = torch.from_numpy(uy)
    prm = lbm.adr_params(3, w.tau_c, precision=lbm.LBM_F64, x_plane=xp)
    sv = lbm.ADRSolver(geom, prm, ud.cuda()).init()
    sv.run(nsteps)
    dkab, dkbc, dw, _ = sv.adjoint(nit, tol=0.0, check_every=nit,
                                   nfibers=fib.shape[0])
    for got, want in ((dkab, ref["dkab"]), (dkbc, ref["dkbc"])):
        g = got.cpu().numpy()[:, :w.nx]
        assert np.linalg.norm(want) > 0
        assert np.linalg.norm(g - want) <= 1e-10 * np.linalg.norm(want)
    dw = dw.cpu().numpy()
    assert np.abs(dw_ref).max() > 0
    assert np.allclose(dw, dw_ref, rtol=1e-9, atol=1e-9 * np.abs(dw_ref).max())
