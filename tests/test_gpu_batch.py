"""Batched solves (lbm_batch_*): every lattice of a batch of uneven sizes
gives the same steps and efficiency as its own lbm_adr_solve (the per-node
arithmetic is shared), in every precision; the autotuner picks a valid
launch shape; reduced precisions stay within their efficiency tolerance of
the FP64 batch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2109_04455_gb300 import inputs, lbm  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lattices():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04455_gb300 import _build
    _build.build()
    out = []
    for i, (nx, ny) in enumerate([(300, 64), (173, 45), (420, 96), (96, 30)]):
        rng = inputs.SplitMix64(100 + i)
        rows = inputs.place_fibers(rng, 0.25 * nx, 0.45 * nx, ny, 3, 3, 5,
                                   2.0, lambda r: (1, 0.0))
        rows += inputs.place_fibers(
            rng, 0.55 * nx, 0.8 * nx, ny, 3, 3, 5, 2.0,
            lambda r: (3, r.uniform_range(0, 6.28)),
            [(f[0], f[1], f[2]) for f in rows])
        fib = np.asarray(rows)
        k1, k2 = 0.02 * (i + 1), 0.03
        geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
        u64, _ = lbm.lbm_flow_solve(geom, 0.8, 0.05, 2000,
                                    precision=lbm.LBM_F64)
        out.append((geom, u64, 0.6 + 0.1 * i))
    return out


def _params(lat, prec, tol, max_steps):
    return [lbm.adr_params(3, tau, precision=prec, max_steps=max_steps,
                           tol=tol, check_every=200)
            for (_, _, tau) in lat]


@pytest.mark.parametrize("prec", [lbm.LBM_F64, lbm.LBM_F32, lbm.LBM_F16DEV])
def test_batch_equals_unbatched(lattices, prec):
    tol = 1e-9 if prec == lbm.LBM_F64 else 1e-5
    params = _params(lattices, prec, tol, 6000)
    us = [u if prec == lbm.LBM_F64 else u.float() for (_, u, _) in lattices]
    b = lbm.Batch([g for (g, _, _) in lattices], params, us)
    infos = b.solve()
    t = b.tuning()
    assert t["tile"] in (128, 256) and t["grid"] > 0
    for (geom, _, _), prm, u, inf in zip(lattices, params, us, infos):
        _, ref = lbm.lbm_adr_solve(geom, prm, u, want_conc=False)
        assert inf["steps"] == ref["steps"]
        assert inf["converged"] == ref["converged"]
        assert abs(inf["eps"] - ref["eps"]) <= 1e-13
        assert np.allclose(inf["flux"], ref["flux"], rtol=1e-13, atol=0)


def test_batch_reduced_precision_against_f64(lattices):
    res = {}
    for prec in (lbm.LBM_F64, lbm.LBM_F32, lbm.LBM_F16DEV):
        params = _params(lattices, prec, 0.0, 3000)   # fixed step count
        us = [u if prec == lbm.LBM_F64 else u.float() for (_, u, _) in lattices]
        b = lbm.Batch([g for (g, _, _) in lattices], params, us)
        res[prec] = b.solve()
    for i in range(len(lattices)):
        e64 = res[lbm.LBM_F64][i]["eps"]
        assert abs(res[lbm.LBM_F32][i]["eps"] - e64) < 1e-4
        assert abs(res[lbm.LBM_F16DEV][i]["eps"] - e64) < 1e-3
