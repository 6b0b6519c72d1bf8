"""Checkpoint / resume of the ADR state (lbm_adr_state_save / _load):
continuing from a saved state gives the saved run bit for bit, in every
precision (the FP16 rounding is seeded by the restored step count);
mismatched or truncated states are refused."""
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


def _setup(prec):
    w = inputs.fiber_pair(2.0, 10.0, nx=400, ny=120, x1=150.0)
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    u, _ = lbm.lbm_flow_solve(geom, w.tau_flow, w.u0, 800,
                              precision=lbm.LBM_F64)
    if prec != lbm.LBM_F64:
        u = u.float()
    prm = lbm.adr_params(3, w.tau_c, precision=prec)
    return geom, u, prm


@pytest.mark.parametrize("prec", [lbm.LBM_F64, lbm.LBM_F32, lbm.LBM_F16DEV])
def test_resume_is_bit_identical(prec):
    geom, u, prm = _setup(prec)
    a = lbm.ADRSolver(geom, prm, u).init()
    a.run(301, check=False)
    ckpt = a.state_save()
    info_a = a.run(250)
    conc_a = a.conc().cpu().numpy()
    b = lbm.ADRSolver(geom, prm, u).init()
    b.run(17, check=False)                 # some other state first
    b.state_load(ckpt)
    with pytest.raises(lbm.LBMError):
        b.conc()                           # nothing recorded since the load
    info_b = b.run(250)
    conc_b = b.conc().cpu().numpy()
    assert info_b["steps"] == info_a["steps"] == 551
    assert np.array_equal(conc_a, conc_b)
    assert info_a["flux"] == info_b["flux"] and info_a["eps"] == info_b["eps"]


def test_mismatched_or_truncated_state_refused():
    geom, u, prm = _setup(lbm.LBM_F32)
    a = lbm.ADRSolver(geom, prm, u).init()
    a.run(10, check=False)
    ckpt = a.state_save()
    g64, u64, p64 = _setup(lbm.LBM_F64)
    b = lbm.ADRSolver(g64, p64, u64).init()
    for bad in (ckpt, ckpt[:100], ckpt[: ckpt.size - 1]):
        with pytest.raises(lbm.LBMError) as e:
            (b if bad is ckpt else a).state_load(bad)
        assert e.value.status == lbm.LBM_EINVAL
    # a refused load changed nothing
    assert a.run(10)["steps"] == 20
