"""The adjoint at the size of the two-membrane cascade lattice (2048 x 512,
80 fibers, Pe = 10, Da = 1): the FP64 gradient of the steady efficiency
with respect to the relaxed catalyst weights, projected on a random
direction over 16 random fibers, against a central difference of two
steady solves along that direction (warm-started from the base state's
checkpoint)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2109_04455_gb300 import inputs, lbm  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04455_gb300 import _build
    _build.build()
    lbm.load()


def _steady(w, fib, u, tol, start=None):
    geom = lbm.Geometry(w.nx, w.ny, fib, w.k1, w.k2).upload()
    prm = lbm.adr_params(3, w.tau_c, precision=lbm.LBM_F64)
    sv = lbm.ADRSolver(geom, prm, u).init()
    if start is not None:
        sv.state_load(start)
    info = sv.solve(tol, 1000, 800000)
    assert info["converged"], info
    return geom, sv, info


def test_cascade_lattice_directional_derivative():
    w = inputs.two_membrane_cascade(seed=0, pe=10.0)
    fib = w.fibers.copy()
    # relaxed weights inside (0, 1) so that both signs of the step are valid
    fib[:, 5] = np.where(fib[:, 3] == 1, 0.9, 0.1)
    geom0 = lbm.Geometry(w.nx, w.ny, fib, w.k1, w.k2).upload()
    u, finfo = lbm.lbm_flow_solve(geom0, w.tau_flow, w.u0, 400000, tol=1e-10,
                                  check_every=1000, precision=lbm.LBM_F64)
    assert finfo["converged"]
    _, sv, info = _steady(w, fib, u, 1e-12)
    base = sv.state_save()
    _, _, dw, ainfo = sv.adjoint(800000, tol=1e-12, check_every=1000,
                                 nfibers=fib.shape[0])
    assert ainfo["converged"]
    assert ainfo["eps"] == info["eps"]
    dw = dw.cpu().numpy()
    rng = np.random.default_rng(4)
    v = np.zeros(fib.shape[0])
    pick = rng.choice(fib.shape[0], 16, replace=False)
    v[pick] = rng.standard_normal(16)
    v /= np.linalg.norm(v)
    # h = 1e-2 (at most 2.5e-3 on one weight here): the difference of the
    # two efficiencies, 2 h |d eps/d v| ~ 9e-8, stays far above what is left
    # of their convergence at a per-step residual of 1e-12
    h = 1e-2
    eps = []
    for sgn in (1.0, -1.0):
        fb = fib.copy()
        fb[:, 5] += sgn * h * v
        eps.append(_steady(w, fb, u, 1e-12, start=base)[2]["eps"])
    fd = (eps[0] - eps[1]) / (2 * h)
    ad = float(dw @ v)
    assert abs(fd) > 1e-3 * np.abs(dw).max()      # a non-trivial direction
    assert ad == pytest.approx(fd, rel=2e-3)
