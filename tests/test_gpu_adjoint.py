"""Discrete adjoint on the GPU (lbm_adr_adjoint) against the oracle's FP64
adjoint at equal iteration counts, and against central finite differences of
the GPU's own FP64 steady state (relative agreement 1e-3)."""
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


def _geometry(weights=True):
    nx, ny = 150, 40
    rng = inputs.SplitMix64(5)
    rows = inputs.place_fibers(rng, 30, 70, ny, 4, 3, 5, 2.0,
                               lambda r: (1, 0.0))
    rows += inputs.place_fibers(rng, 80, 120, ny, 4, 3, 5, 2.0,
                                lambda r: (2, 0.0),
                                [(f[0], f[1], f[2]) for f in rows])
    fib = np.asarray(rows)
    if weights:
        fib[:, 5] = np.linspace(0.9, 0.1, fib.shape[0])   # relaxed weights
    return nx, ny, fib, 0.06, 0.05


def _dev_u(ux, uy, nx_pad, dtype):
    ny, nx = ux.shape
    u = torch.zeros((2, ny, nx_pad), dtype=dtype)
    u[0, :, :nx] = torch.from_numpy(ux)
    u[1, :, :nx] = torch.from_numpy(uy)
    return u.cuda()


@pytest.mark.parametrize("ns", [2, 3])
def test_adjoint_f64_matches_oracle_adjoint(ns):
    nx, ny, fib, k1, k2 = _geometry()
    solid, kab, kbc = oracle.raster(nx, ny, fib, k1, k2)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, 600)
    taus = [0.7, 0.8, 0.9][:ns]
    cin = [1.0, 0.0, 0.0][:ns]
    fsteps, asteps = 800, 500
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, taus, cin)
    fwd = prob.run(fsteps)
    ref = oracle.adjoint(prob, fwd["g"], asteps)

    geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
    u = _dev_u(ux, uy, geom.nx_pad, torch.float64)
    prm = lbm.adr_params(ns, taus, cin, precision=lbm.LBM_F64)
    sv = lbm.ADRSolver(geom, prm, u).init()
    info = sv.run(fsteps)
    assert abs(info["eps"] - fwd["eps"]) < 1e-12
    dkab, dkbc, dw, ainfo = sv.adjoint(asteps, nfibers=fib.shape[0])
    assert ainfo["steps"] == asteps
    ga = dkab.cpu().numpy()[:, :nx]
    gb = dkbc.cpu().numpy()[:, :nx]
    na = np.linalg.norm(ref["dkab"])
    assert na > 0
    assert np.linalg.norm(ga - ref["dkab"]) / na < 1e-10
    if ns == 3:
        nb = np.linalg.norm(ref["dkbc"])
        assert nb > 0 and np.linalg.norm(gb - ref["dkbc"]) / nb < 1e-10
    # per-fiber weights from the oracle's own node -> fiber map
    ids = oracle.fiber_ids(nx, ny, fib)
    dwr = oracle.fiber_weight_gradient(ids, ref["dkab"], ref["dkbc"], k1, k2,
                                       fib.shape[0])
    assert np.allclose(dw.cpu().numpy(), dwr, rtol=1e-9,
                       atol=1e-12 * np.abs(dwr).max())
    # gradients live on fiber nodes only
    assert np.all(ga[solid == 0] == 0.0)


def _steady_eps(nx, ny, fib, k1, k2, u, taus, prec=lbm.LBM_F64):
    geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
    prm = lbm.adr_params(3, taus, precision=prec, max_steps=200000,
                         tol=1e-13, check_every=500)
    _, info = lbm.lbm_adr_solve(geom, prm, u, want_conc=False,
                                raise_not_converged=True)
    return info["eps"]


def test_adjoint_fiber_weights_match_finite_differences():
    """Steady cascade on the GPU (FP64, residual 1e-13): d eps/d w_f from the
    converged adjoint against central differences with h = 1e-4 on every
    fiber's relaxed weight."""
    nx, ny, fib, k1, k2 = _geometry()
    geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
    u, _ = lbm.lbm_flow_solve(geom, 0.8, 0.05, 30000, tol=1e-10,
                              check_every=500, precision=lbm.LBM_F64)
    taus = [0.7] * 3
    prm = lbm.adr_params(3, taus, precision=lbm.LBM_F64)
    sv = lbm.ADRSolver(geom, prm, u).init()
    info = sv.solve(1e-13, 500, 200000)
    assert info["converged"]
    _, _, dw, ainfo = sv.adjoint(200000, tol=1e-13, check_every=500,
                                 nfibers=fib.shape[0])
    assert ainfo["converged"]
    dw = dw.cpu().numpy()
    h = 1e-4
    for f in range(fib.shape[0]):
        vals = []
        for sgn in (1, -1):
            fb = fib.copy()
            fb[f, 5] += sgn * h
            vals.append(_steady_eps(nx, ny, fb, k1, k2, u, taus))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert dw[f] == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(dw).max())


def test_adjoint_f32_close_to_f64():
    nx, ny, fib, k1, k2 = _geometry()
    solid, _, _ = oracle.raster(nx, ny, fib, k1, k2)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, 3000)
    out = {}
    for prec, dt in ((lbm.LBM_F64, torch.float64),
                     (lbm.LBM_F32, torch.float32)):
        geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
        u = _dev_u(ux, uy, geom.nx_pad, dt)
        sv = lbm.ADRSolver(geom, lbm.adr_params(3, [0.7] * 3,
                                                precision=prec), u).init()
        sv.solve(1e-12 if prec == lbm.LBM_F64 else 1e-7, 500, 100000)
        _, _, dw, _ = sv.adjoint(100000, tol=1e-10 if prec == lbm.LBM_F64
                                 else 1e-6, check_every=500,
                                 nfibers=fib.shape[0])
        out[prec] = dw.cpu().numpy()
    d64, d32 = out[lbm.LBM_F64], out[lbm.LBM_F32]
    assert np.abs(d32 - d64).max() <= 1e-3 * np.abs(d64).max()


def test_autograd_function_matches_finite_differences():
    """torch.autograd through MembraneProblem.efficiency: backward() runs the
    adjoint; compare with central differences of the forward (h = 1e-4)."""
    from paper_2109_04455_gb300.autograd import MembraneProblem
    nx, ny, fib, k1, k2 = _geometry()
    prob = MembraneProblem(nx, ny, fib, k1, k2, [0.7] * 3, tol=1e-13,
                           check_every=500)
    w = torch.tensor(fib[:, 5], dtype=torch.float64, requires_grad=True)
    eps = prob.efficiency(w)
    eps.backward()
    g = w.grad.numpy()
    h = 1e-4
    for f in (0, fib.shape[0] - 1):
        vals = []
        for sgn in (1, -1):
            w2 = w.detach().clone()
            w2[f] += sgn * h
            vals.append(float(prob.efficiency(w2)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert g[f] == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(g).max())


def test_adjoint_refuses_nodewise_variant():
    """The node-wise reaction variant has no adjoint: LBM_EINVAL, and the
    solver stays usable."""
    nx, ny, fib, k1, k2 = _geometry()
    geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
    u = torch.zeros((2, ny, geom.nx_pad), dtype=torch.float64, device="cuda")
    u[0, :, :nx] = 0.02
    prm = lbm.adr_params(3, [0.62] * 3, precision=lbm.LBM_F64,
                         flags=lbm.LBM_ADR_NODEWISE)
    sv = lbm.ADRSolver(geom, prm, u).init()
    sv.run(10)
    with pytest.raises(lbm.LBMError) as e:
        sv.adjoint(10)
    assert e.value.status == lbm.LBM_EINVAL
    assert sv.run(10)["steps"] == 20
