"""Failure detection on the GPU path without any fault: the explicit ADR
scheme loses positivity, and then stability, as tau_c -> 1/2 (high Pe, the
warning of the paper's Appendix C).  The check steps report the most
negative concentration of each species (info c_min) and return
LBM_EUNSTABLE once it falls below -neg_tol * max(1, c_in).  Both cases are
made by host-side parameters only, and the oracle (FP64, same step counts)
decides what the GPU must report."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2109_04455_gb300 import inputs, lbm  # noqa: E402

pytestmark = pytest.mark.gpu
NX, NY, R = 130, 48, 6.0
FIBERS = np.array([[40.3, 22.2, R, 1, 0, -1], [75.7, 28.1, R, 2, 0, -1]])


@pytest.fixture(scope="module")
def lattice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04455_gb300 import _build
    _build.build()
    oracle.build()
    solid, kab, kbc = oracle.raster(NX, NY, FIBERS, 1.0, 1.0)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, 3000)
    geom = lbm.Geometry(NX, NY, FIBERS, 1.0, 1.0).upload()
    u = torch.zeros((2, NY, geom.nx_pad), dtype=torch.float64)
    u[0, :, :NX] = torch.from_numpy(ux)
    u[1, :, :NX] = torch.from_numpy(uy)
    return solid, kab, kbc, ux, uy, u.cuda()


def _rates(pe, da):
    d = inputs.diffusivity_from_pe(0.05, R, pe)
    return inputs.tau_from_diffusivity(d), inputs.rate_from_da(da, d, R)


def _gpu_chunks(lattice, pe, da, nchunks, neg_tol=0.0):
    """Runs of 100 steps with info through the C ABI; stops at the first
    status that is not LBM_OK.  Returns [(status, info dict)]."""
    solid, kab, kbc, ux, uy, u = lattice
    tau, k = _rates(pe, da)
    geom = lbm.Geometry(NX, NY, FIBERS, k, k).upload()
    prm = lbm.adr_params(3, tau, precision=lbm.LBM_F64, neg_tol=neg_tol)
    sv = lbm.ADRSolver(geom, prm, u).init()
    out = []
    for _ in range(nchunks):
        info = lbm.lbm_solve_info()
        st = lbm.load().lbm_adr_run(sv.handle, 100,
                                    lbm._stream_ptr(None), ctypes.byref(info))
        out.append((st, info.as_dict()))
        if st != lbm.LBM_OK:
            break
    return out


def _oracle_chunks(lattice, pe, da, nchunks):
    """Most negative concentration (or 0) at the last step of each chunk of
    100 steps (the step whose minimum the GPU reports)."""
    solid, kab, kbc, ux, uy, _ = lattice
    tau, k = _rates(pe, da)
    prob = oracle.ADRProblem(solid, kab * k, kbc * k, ux, uy, [tau] * 3,
                             [1, 0, 0])
    g = prob.init()
    out = []
    for _ in range(nchunks):
        prob.steps(g, 100)
        out.append(np.minimum(prob.conc(g).min(axis=(1, 2)), 0.0))
    return out


def test_diverging_lattice_reports_unstable(lattice):
    """Pe = 400 (tau_c = 0.5022): the lattice diverges.  The GPU stops with
    LBM_EUNSTABLE at the first check whose concentration is below -0.1,
    the same check as the oracle's, while every sum is still finite."""
    runs = _gpu_chunks(lattice, 400, 1, 30)
    st, info = runs[-1]
    assert st == lbm.LBM_EUNSTABLE
    assert np.isfinite(info["residual"]) and np.isfinite(info["eps"])
    assert min(info["c_min"]) < -0.1
    assert all(s == lbm.LBM_OK for s, _ in runs[:-1])
    ref = _oracle_chunks(lattice, 400, 1, len(runs))
    first = next(i for i, m in enumerate(ref) if m.min() < -0.1)
    assert first == len(runs) - 1
    assert info["steps"] == 100 * len(runs)
    assert np.allclose(info["c_min"], ref[-1], rtol=1e-9, atol=1e-12)
    assert "below -neg_tol" in lbm.load().lbm_last_error().decode()


def test_bounded_undershoot_is_reported(lattice):
    """Pe = 100, Da = 1000 (tau_c = 0.509): B undershoots to about -2.7%
    near the catalytic surface and stays there.  c_min equals the oracle's
    at every check; the default threshold (0.1) lets the run go on, a
    threshold of 0.01 stops it at the first check below -0.01."""
    n = 15
    runs = _gpu_chunks(lattice, 100, 1000, n)
    ref = _oracle_chunks(lattice, 100, 1000, n)
    assert all(s == lbm.LBM_OK for s, _ in runs) and len(runs) == n
    for (_, info), m in zip(runs, ref):
        assert np.allclose(info["c_min"], m, rtol=1e-9, atol=1e-13)
    assert runs[-1][1]["c_min"][1] < -0.02
    strict = _gpu_chunks(lattice, 100, 1000, n, neg_tol=0.01)
    first = next(i for i, m in enumerate(ref) if m.min() < -0.01)
    assert strict[-1][0] == lbm.LBM_EUNSTABLE and len(strict) == first + 1
    # the test can be turned off
    off = _gpu_chunks(lattice, 400, 1, 12, neg_tol=-1.0)
    assert all(s == lbm.LBM_OK for s, _ in off) and len(off) == 12
    assert min(off[-1][1]["c_min"]) < -0.1


def test_efficiency_convergence_test():
    """eps_tol (lbm_adr_solve and the batch): on a diffusion-dominated
    cascade lattice (Pe = 1, tau_c = 1.7), where a per-step residual of
    1e-6 is reached long before the efficiency settles, adding the
    efficiency test (Aitken extrapolation of the last three checks) lands
    within a few eps_tol of the FP64 steady value (residual 1e-12), in the
    single solve and in the batch alike."""
    w = inputs.two_membrane_cascade(seed=3, pe=1.0, nx=512, ny=96,
                                    bands=((100, 180), (250, 330)),
                                    per_band=6)
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    u, fi = lbm.lbm_flow_solve(geom, w.tau_flow, w.u0, 400000, tol=1e-10,
                               check_every=1000, precision=lbm.LBM_F64)
    assert fi["converged"]

    def solve(tol, eps_tol, prec=lbm.LBM_F64):
        prm = lbm.adr_params(3, w.tau_c, precision=prec, max_steps=2000000,
                             tol=tol, eps_tol=eps_tol, check_every=1000)
        return lbm.lbm_adr_solve(geom, prm, u if prec == lbm.LBM_F64
                                 else u.float(), want_conc=False)[1]

    ref = solve(1e-12, 0.0)
    assert ref["converged"] and ref["eps"] > 1e-3
    loose = solve(1e-6, 0.0)
    tight = solve(1e-6, 1e-6)
    assert tight["converged"] and tight["steps"] >= loose["steps"]
    assert abs(tight["eps"] - ref["eps"]) < 5e-6, (ref, loose, tight)
    assert abs(tight["eps"] - ref["eps"]) <= abs(loose["eps"] - ref["eps"])
    b = lbm.Batch([geom], [lbm.adr_params(3, w.tau_c, precision=lbm.LBM_F32,
                                          max_steps=2000000, tol=1e-6,
                                          eps_tol=1e-5, check_every=1000)],
                  [u.float()])
    info = b.solve()[0]
    assert info["converged"]
    assert abs(info["eps"] - ref["eps"]) < 5e-5, (ref, info)
