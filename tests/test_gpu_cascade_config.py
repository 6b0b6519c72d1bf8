"""The two-membrane cascade lattice as specified (2048 x 512, 40 + 40 R = 8
fibers, seed 0, Da1 = Da2 = 1) at Pe = 1, 10 and 100 (tau_c = 1.7, 0.62,
0.512): FP64 solved to a per-step residual of 1e-9, then FP32 run the same
number of steps from the same start on the same FP64 flow; the outlet
efficiency of Eq. (A-B) (x = nx - 3, three species) agrees within 1e-4.
(FP32 stopped at its own per-step residual of 1e-6 is no steady state at
Pe = 1: it ends 5e-4 off; see the cascade workload of bench.py.)  At
Pe = 100 the scheme is close to its tau = 1/2 limit: B undershoots behind
the catalytic fibers, which the check steps report (c_min) while the run
stays stable."""
import pytest

torch = pytest.importorskip("torch")

from paper_2109_04455_gb300 import inputs, lbm  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def flow():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04455_gb300 import _build
    _build.build()
    w = inputs.two_membrane_cascade(seed=0, pe=10.0)
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    u, info = lbm.lbm_flow_solve(geom, w.tau_flow, w.u0, 1000000, tol=1e-9,
                                 check_every=1000, precision=lbm.LBM_F64)
    assert info["converged"]
    return u


@pytest.mark.parametrize("pe", [1.0, 10.0, 100.0])
def test_cascade_config_steady_f64_and_f32(flow, pe):
    w = inputs.two_membrane_cascade(seed=0, pe=pe)
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    prm = lbm.adr_params(3, w.tau_c, precision=lbm.LBM_F64,
                         max_steps=1000000, tol=1e-9, check_every=1000)
    _, r64 = lbm.lbm_adr_solve(geom, prm, flow, want_conc=False)
    assert r64["converged"] and r64["residual"] < 1e-9
    prm = lbm.adr_params(3, w.tau_c, precision=lbm.LBM_F32,
                         max_steps=r64["steps"], check_every=1000)
    _, r32 = lbm.lbm_adr_solve(geom, prm, flow.float(), want_conc=False)
    assert r32["steps"] == r64["steps"]
    msg = dict(pe=pe, f64=r64, f32=r32)
    assert r64["eps"] > 1e-6, msg                 # C leaves the channel
    assert abs(r32["eps"] - r64["eps"]) < 1e-4, msg
    # outflux shares of A, B, C (at Pe = 1 the FP32 state stops moving at a
    # fixed point of round-to-nearest, a per-step residual of 2e-12, and its
    # shares end 2.4e-4 off, eps 3.3e-5 off)
    s64 = [f / sum(r64["flux"]) for f in r64["flux"]]
    s32 = [f / sum(r32["flux"]) for f in r32["flux"]]
    assert max(abs(a - b) for a, b in zip(s32, s64)) < 1e-3, msg
    if pe == 100.0:
        assert -1e-3 < min(r64["c_min"]) < 0.0, msg
