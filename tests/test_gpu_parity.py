"""GPU path (liblbm.so through its C ABI) against the FP64 CPU oracle.

Tolerances:
* FP64: velocity to 1e-12 absolute; concentrations to 1e-10 relative L2 and
  efficiency to 1e-10 absolute, at equal step counts (both sides run the same
  deterministic scheme; only rounding order differs).
* FP32: efficiency to 1e-4 absolute; FP16 deviation storage: 1e-3.
Lattices are small enough for the oracle to finish in seconds while still
spanning several 128-node row blocks with a ragged tail (nx not a multiple
of 32), and cover every link type: inlet, outlet, wall, corner, inert,
A->B, B->C and side-by-side fibers, relaxed catalyst weights.
"""
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


def _case(name):
    if name == "small":      # one row block of 128 with a ragged tail
        nx, ny = 70, 26
        fib = [[22.4, 12.3, 4.0, 1, 0, -1], [44.1, 13.6, 4.0, 2, 0, -1],
               [33.0, 5.5, 2.0, 3, 0.7, -1], [55.2, 20.1, 2.5, 0, 0, -1]]
    elif name == "ragged":   # three row blocks, last one mostly padding
        nx, ny = 261, 37
        rng = inputs.SplitMix64(11)
        rows = inputs.place_fibers(rng, 40, 120, ny, 5, 3, 5, 2.0,
                                   lambda r: (1, 0.0))
        rows += inputs.place_fibers(rng, 140, 220, ny, 5, 3, 5, 2.0,
                                    lambda r: (3, r.uniform_range(0, 6.28)),
                                    [(f[0], f[1], f[2]) for f in rows])
        rows[2][5] = 0.35      # one relaxed catalyst weight
        rows[-1][3] = 2.0
        fib = rows
    elif name == "empty":    # no fibers, tiny lattice
        nx, ny = 5, 3
        fib = np.zeros((0, 6))
    else:
        raise KeyError(name)
    return nx, ny, np.asarray(fib, dtype=np.float64).reshape(-1, 6)


def _dev_u(ux, uy, nx_pad, dtype):
    ny, nx = ux.shape
    u = torch.zeros((2, ny, nx_pad), dtype=dtype)
    u[0, :, :nx] = torch.from_numpy(ux)
    u[1, :, :nx] = torch.from_numpy(uy)
    return u.cuda()


def _run_gpu_adr(geom, u, ns, taus, cin, prec, steps, flags=0, xp=-1):
    prm = lbm.adr_params(ns, taus, cin, precision=prec, max_steps=steps,
                         flags=flags, x_plane=xp)
    conc, info = lbm.lbm_adr_solve(geom, prm, u)
    return conc.double().cpu().numpy()[:, :, :geom.nx], info


# ---------------------------------------------------------------------------
# flow
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["small", "ragged", "empty"])
def test_flow_f64_matches_oracle(name):
    nx, ny, fib = _case(name)
    steps = 400
    geom = lbm.Geometry(nx, ny, fib, 0.05, 0.07).upload()
    u, info = lbm.lbm_flow_solve(geom, 0.8, 0.05, steps,
                                 precision=lbm.LBM_F64)
    solid, _, _ = oracle.raster(nx, ny, fib, 0.05, 0.07)
    _, ux, uy, res = oracle.flow_run(solid, 0.8, 0.05, steps)
    ug = u.cpu().numpy()
    assert np.abs(ug[0, :, :nx] - ux).max() < 1e-12
    assert np.abs(ug[1, :, :nx] - uy).max() < 1e-12
    assert np.all(ug[:, :, nx:] == 0.0)
    assert np.all(ug[:, :, :nx][:, solid == 1] == 0.0)
    assert info["steps"] == steps
    # the residual is a difference of nearly equal fields: compare to the
    # rounding level of the velocities once the flow has settled
    assert info["residual"] == pytest.approx(res, rel=1e-6, abs=1e-14)


def test_flow_f32_matches_oracle():
    nx, ny, fib = _case("ragged")
    steps = 400
    geom = lbm.Geometry(nx, ny, fib, 0.0, 0.0).upload()
    u, _ = lbm.lbm_flow_solve(geom, 0.8, 0.05, steps, precision=lbm.LBM_F32)
    solid, _, _ = oracle.raster(nx, ny, fib, 0.0, 0.0)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, steps)
    ug = u.double().cpu().numpy()
    # float rounding of O(0.1) populations, damped over the run
    assert np.abs(ug[0, :, :nx] - ux).max() < 5e-6
    assert np.abs(ug[1, :, :nx] - uy).max() < 5e-6


def test_flow_solve_to_tolerance_matches_oracle_steps():
    """Convergence loop: checks every 100 steps, stops below tol; the oracle
    with the same residual definition stops at the same step."""
    nx, ny, fib = _case("small")
    geom = lbm.Geometry(nx, ny, fib, 0.0, 0.0).upload()
    tol = 1e-6
    u, info = lbm.lbm_flow_solve(geom, 0.8, 0.05, 20000, tol=tol,
                                 check_every=100, precision=lbm.LBM_F64)
    assert info["converged"] and info["residual"] < tol
    solid, _, _ = oracle.raster(nx, ny, fib, 0.0, 0.0)
    f = oracle.flow_init_channel(solid, 0.05)
    steps = 0
    while True:
        oracle.flow_steps(f, solid, 0.8, 0.05, 99)
        _, ux0, uy0 = oracle.flow_moments(f, solid)
        oracle.flow_steps(f, solid, 0.8, 0.05, 1)
        _, ux, uy = oracle.flow_moments(f, solid)
        steps += 100
        if oracle.flow_residual(ux0, uy0, ux, uy) < tol:
            break
    assert info["steps"] == steps


# ---------------------------------------------------------------------------
# ADR, fed with the oracle's velocity field
# ---------------------------------------------------------------------------
def _oracle_case(name, flow_steps=300):
    nx, ny, fib = _case(name)
    k1, k2 = 0.05, 0.07
    solid, kab, kbc = oracle.raster(nx, ny, fib, k1, k2)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, flow_steps)
    return nx, ny, fib, k1, k2, solid, kab, kbc, ux, uy


_ORACLE_FLAGS = {0: 0, lbm.LBM_ADR_INLET_ABB_ALL: oracle.INLET_ABB_ALL,
                 lbm.LBM_ADR_NODEWISE: oracle.NODEWISE}


@pytest.mark.parametrize("name,ns,flags", [
    ("small", 3, 0), ("small", 2, 0), ("small", 1, 0),
    ("ragged", 3, 0), ("ragged", 3, lbm.LBM_ADR_INLET_ABB_ALL),
    ("small", 3, lbm.LBM_ADR_NODEWISE), ("ragged", 2, lbm.LBM_ADR_NODEWISE),
    ("ragged", 3, lbm.LBM_ADR_NODEWISE | lbm.LBM_ADR_INLET_ABB_ALL),
    ("empty", 2, 0)])
def test_adr_f64_matches_oracle(name, ns, flags):
    nx, ny, fib, k1, k2, solid, kab, kbc, ux, uy = _oracle_case(name)
    taus = [0.62, 0.7, 0.9][:ns]
    cin = [1.0, 0.0, 0.0][:ns]
    steps = 500
    geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
    u = _dev_u(ux, uy, geom.nx_pad, torch.float64)
    conc, info = _run_gpu_adr(geom, u, ns, taus, cin, lbm.LBM_F64, steps,
                              flags)
    oflags = 0
    for bit, obit in _ORACLE_FLAGS.items():
        if flags & bit:
            oflags |= obit
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, taus, cin,
                             flags=oflags)
    ref = prob.run(steps)
    rel = np.linalg.norm(conc - ref["conc"]) / np.linalg.norm(ref["conc"])
    assert rel < 1e-10
    for s in range(ns):
        assert info["flux"][s] == pytest.approx(ref["flux"][s], rel=1e-10,
                                                abs=1e-15)
    if ns >= 2:
        assert abs(info["eps"] - ref["eps"]) < 1e-10
    assert info["residual"] == pytest.approx(ref["residual"], rel=1e-6,
                                             abs=1e-15)
    assert info["steps"] == steps


def test_adr_flux_plane_anywhere():
    nx, ny, fib, k1, k2, solid, kab, kbc, ux, uy = _oracle_case("ragged")
    geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
    u = _dev_u(ux, uy, geom.nx_pad, torch.float64)
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, [0.62] * 3, [1, 0, 0])
    ref = prob.run(300)
    for xp in (0, 130, nx - 1):
        _, info = _run_gpu_adr(geom, u, 3, [0.62] * 3, [1, 0, 0],
                               lbm.LBM_F64, 300, xp=xp)
        want = prob.flux(ref["g"], xp)
        assert np.allclose(info["flux"], want, rtol=1e-10, atol=1e-15)


# concentration tolerance: float rounding (~6e-8 per operation) accumulated
# over 1500 steps of a damped map stays near 1e-5; half storage 1e-2
@pytest.mark.parametrize("prec,tol_eps,tol_c", [(lbm.LBM_F32, 1e-4, 1e-4),
                                                (lbm.LBM_F16DEV, 1e-3, 1e-2)])
def test_adr_reduced_precision(prec, tol_eps, tol_c):
    nx, ny, fib, k1, k2, solid, kab, kbc, ux, uy = _oracle_case("ragged")
    steps, xp = 1500, 130
    geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
    u = _dev_u(ux, uy, geom.nx_pad, torch.float32)
    conc, info = _run_gpu_adr(geom, u, 3, [0.62] * 3, [1, 0, 0], prec, steps,
                              xp=xp)
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, [0.62] * 3, [1, 0, 0])
    ref = prob.run(steps, xp=xp)
    rel = np.linalg.norm(conc - ref["conc"]) / np.linalg.norm(ref["conc"])
    assert rel < tol_c
    assert abs(info["eps"] - ref["eps"]) < tol_eps
    # the A->B efficiency on this plane is O(0.1), so the tolerance bites
    e2_gpu = lbm.lbm_efficiency(list(info["flux"][:2]) + [0.0], 2)
    e2_ref = oracle.efficiency(ref["flux"][:2], 2)
    assert e2_ref > 10 * tol_eps
    assert abs(e2_gpu - e2_ref) < tol_eps


def test_adr_steady_solve_f64():
    """Solve to a residual of 1e-9 (checked every 100 steps) on both sides:
    same stopping step, same efficiency."""
    nx, ny, fib, k1, k2, solid, kab, kbc, ux, uy = _oracle_case("small", 3000)
    taus = [0.9] * 3
    geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
    u = _dev_u(ux, uy, geom.nx_pad, torch.float64)
    prm = lbm.adr_params(3, taus, precision=lbm.LBM_F64, max_steps=40000,
                         tol=1e-9, check_every=100)
    conc, info = lbm.lbm_adr_solve(geom, prm, u)
    assert info["converged"]
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, taus, [1, 0, 0])
    ref = prob.solve(1e-9, 100, 40000)
    assert ref["converged"] and ref["steps"] == info["steps"]
    assert abs(info["eps"] - ref["eps"]) < 1e-10
    assert 0 < info["eps"] < 1


# ---------------------------------------------------------------------------
# whole path: GPU flow -> GPU ADR against oracle flow -> oracle ADR
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def single_fiber_oracle():
    """The single-fiber A->B channel in full: 200x100, R = 8 at (60, 50),
    u0 = 0.05, tau = 0.8, 20000 flow steps; Pe = 10 (tau_c = 0.62), Da = 1,
    20000 ADR steps."""
    w = inputs.single_fiber()
    solid, kab, kbc = oracle.raster(w.nx, w.ny, w.fibers, w.k1, w.k2)
    _, ux, uy, fres = oracle.flow_run(solid, w.tau_flow, w.u0, w.flow_steps)
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, [w.tau_c] * 2, [1, 0])
    ref = prob.run(w.adr_steps)
    return w, ux, uy, ref


def test_single_fiber_full_path_f64(single_fiber_oracle):
    w, ux, uy, ref = single_fiber_oracle
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    u, _ = lbm.lbm_flow_solve(geom, w.tau_flow, w.u0, w.flow_steps,
                              precision=lbm.LBM_F64)
    ug = u.cpu().numpy()[:, :, :w.nx]
    assert np.abs(ug[0] - ux).max() < 1e-12 and np.abs(ug[1] - uy).max() < 1e-12
    conc, info = _run_gpu_adr(geom, u, 2, [w.tau_c] * 2, [1, 0], lbm.LBM_F64,
                              w.adr_steps)
    rel = np.linalg.norm(conc - ref["conc"]) / np.linalg.norm(ref["conc"])
    assert rel < 1e-10
    assert abs(info["eps"] - ref["eps"]) < 1e-10
    assert ref["eps"] > 1e-3


@pytest.mark.parametrize("prec,tol", [(lbm.LBM_F32, 1e-4),
                                      (lbm.LBM_F16DEV, 1e-3)])
def test_single_fiber_full_path_reduced(single_fiber_oracle, prec, tol):
    w, ux, uy, ref = single_fiber_oracle
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    u, _ = lbm.lbm_flow_solve(geom, w.tau_flow, w.u0, w.flow_steps,
                              precision=lbm.LBM_F32)
    _, info = _run_gpu_adr(geom, u, 2, [w.tau_c] * 2, [1, 0], prec,
                           w.adr_steps)
    assert abs(info["eps"] - ref["eps"]) < tol


# ---------------------------------------------------------------------------
# status codes from the device path (no fault is provoked: a NaN velocity is
# ordinary arithmetic that the residual check must report)
# ---------------------------------------------------------------------------
def test_nan_velocity_reports_unstable():
    nx, ny, fib = _case("small")
    geom = lbm.Geometry(nx, ny, fib, 0.05, 0.05).upload()
    u = torch.full((2, ny, geom.nx_pad), float("nan"), dtype=torch.float32,
                   device="cuda")
    prm = lbm.adr_params(3, 0.7, precision=lbm.LBM_F32, max_steps=10)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_adr_solve(geom, prm, u)
    assert e.value.status == lbm.LBM_EUNSTABLE


def test_workspace_too_small_and_not_converged():
    import ctypes
    nx, ny, fib = _case("small")
    geom = lbm.Geometry(nx, ny, fib, 0.05, 0.05).upload()
    u = torch.zeros((2, ny, geom.nx_pad), dtype=torch.float32, device="cuda")
    prm = lbm.adr_params(3, 0.7, precision=lbm.LBM_F32, max_steps=10)
    need = lbm.load().lbm_adr_ws_bytes(geom.handle, ctypes.byref(prm))
    ws = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    st = lbm.load().lbm_adr_create(geom.handle, ctypes.byref(prm),
                                   ctypes.c_void_p(u.data_ptr()),
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                   ctypes.byref(h))
    assert st == lbm.LBM_ENOMEM
    prm = lbm.adr_params(3, 0.7, precision=lbm.LBM_F32, max_steps=200,
                         tol=1e-30, check_every=100)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_adr_solve(geom, prm, u, raise_not_converged=True)
    assert e.value.status == lbm.LBM_ENOTCONVERGED


# ---------------------------------------------------------------------------
# the two-membrane cascade lattice in full size (2048 x 512, 80 fibers, Pe = 1),
# at a fixed step count the oracle (OpenMP over rows) finishes in a minute or
# two; the flux plane sits just downstream of the A->B membrane
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cascade_oracle():
    w = inputs.two_membrane_cascade(seed=0, pe=1.0)
    nflow, nadr, xp = 2000, 2000, 720
    solid, kab, kbc = oracle.raster(w.nx, w.ny, w.fibers, w.k1, w.k2)
    _, ux, uy, _ = oracle.flow_run(solid, w.tau_flow, w.u0, nflow)
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, [w.tau_c] * 3,
                             [1, 0, 0])
    ref = prob.run(nadr, xp=xp)
    return w, ux, uy, ref, nflow, nadr, xp


def test_cascade_full_lattice_pe100_f64(cascade_oracle):
    """The same lattice at Pe = 100, where tau_c = 0.512 comes close to the
    1/2 stability limit (Appendix C warns of negative populations there):
    FP64 matches the oracle at 2000 steps, and the most negative
    concentration the check steps report equals the oracle's (B undershoots
    a little behind the catalytic fibers; it is reported, not an error)."""
    w0, ux, uy, _, nflow, nadr, xp = cascade_oracle
    w = inputs.two_membrane_cascade(seed=0, pe=100.0)
    assert abs(w.tau_c - 0.512) < 1e-12
    solid, kab, kbc = oracle.raster(w.nx, w.ny, w.fibers, w.k1, w.k2)
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, [w.tau_c] * 3,
                             [1, 0, 0])
    ref = prob.run(nadr, xp=xp)
    cmin = np.minimum(ref["conc"].min(axis=(1, 2)), 0.0)
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    u = _dev_u(ux, uy, geom.nx_pad, torch.float64)
    conc, info = _run_gpu_adr(geom, u, 3, [w.tau_c] * 3, [1, 0, 0],
                              lbm.LBM_F64, nadr, xp=xp)
    rel = np.linalg.norm(conc - ref["conc"]) / np.linalg.norm(ref["conc"])
    assert rel < 1e-10
    assert np.allclose(info["flux"], ref["flux"], rtol=1e-10, atol=1e-15)
    assert ref["conc"][1].max() > 1e-4       # B is made at the membrane
    assert np.allclose(info["c_min"], cmin, rtol=1e-8, atol=1e-14)


def test_cascade_full_lattice_f64(cascade_oracle):
    w, ux, uy, ref, nflow, nadr, xp = cascade_oracle
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    u, _ = lbm.lbm_flow_solve(geom, w.tau_flow, w.u0, nflow,
                              precision=lbm.LBM_F64)
    ug = u.cpu().numpy()[:, :, :w.nx]
    assert np.abs(ug[0] - ux).max() < 1e-12 and np.abs(ug[1] - uy).max() < 1e-12
    conc, info = _run_gpu_adr(geom, u, 3, [w.tau_c] * 3, [1, 0, 0],
                              lbm.LBM_F64, nadr, xp=xp)
    rel = np.linalg.norm(conc - ref["conc"]) / np.linalg.norm(ref["conc"])
    assert rel < 1e-10
    assert np.allclose(info["flux"], ref["flux"], rtol=1e-10, atol=1e-15)
    assert ref["flux"][1] > 1e-4          # B crosses the plane


@pytest.mark.parametrize("prec,tol", [(lbm.LBM_F32, 1e-4),
                                      (lbm.LBM_F16DEV, 1e-3)])
def test_cascade_full_lattice_reduced(cascade_oracle, prec, tol):
    w, ux, uy, ref, nflow, nadr, xp = cascade_oracle
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    u = _dev_u(ux, uy, geom.nx_pad, torch.float32)
    _, info = _run_gpu_adr(geom, u, 3, [w.tau_c] * 3, [1, 0, 0], prec, nadr,
                           xp=xp)
    e_ref = oracle.efficiency(ref["flux"][:2], 2)
    e_gpu = lbm.lbm_efficiency(list(info["flux"][:2]) + [0.0], 2)
    assert e_ref > 10 * tol
    assert abs(e_gpu - e_ref) < tol


def test_per_node_rate_fields_match_oracle():
    """lbm_geometry_set_rates: a random catalyst field over the solid nodes
    (both rates, each node its own values) gives the oracle's state at 400
    steps; re-uploading into the same buffer updates a solver created
    earlier."""
    nx, ny, fib, k1, k2, solid, kab, kbc, ux, uy = _oracle_case("ragged")
    rng = np.random.default_rng(7)
    kab2 = np.where(solid == 1, rng.uniform(0.0, 0.2, solid.shape), 0.0)
    kbc2 = np.where(solid == 1, rng.uniform(0.0, 0.1, solid.shape), 0.0)
    ys, xs = np.nonzero(solid == 1)
    kab2[ys[::3], xs[::3]] = 0.0                      # B->C only
    kab2[ys[1::5], xs[1::5]] = kbc2[ys[1::5], xs[1::5]] = 0.0   # inert
    geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
    ws_ptr = geom.ws.data_ptr()
    u = _dev_u(ux, uy, geom.nx_pad, torch.float64)
    geom.set_rates(kab2, kbc2).upload()
    assert geom.ws.data_ptr() == ws_ptr
    conc, info = _run_gpu_adr(geom, u, 3, [0.62, 0.7, 0.9], [1, 0, 0],
                              lbm.LBM_F64, 400)
    prob = oracle.ADRProblem(solid, kab2, kbc2, ux, uy, [0.62, 0.7, 0.9],
                             [1, 0, 0])
    ref = prob.run(400)
    rel = np.linalg.norm(conc - ref["conc"]) / np.linalg.norm(ref["conc"])
    assert rel < 1e-10
    assert np.allclose(info["flux"], ref["flux"], rtol=1e-10, atol=1e-15)
    # the raster's own rates differ: that run is not the same
    prob0 = oracle.ADRProblem(solid, kab, kbc, ux, uy, [0.62, 0.7, 0.9],
                              [1, 0, 0])
    ref0 = prob0.run(400)
    assert np.linalg.norm(ref0["conc"] - ref["conc"]) > 1e-6
