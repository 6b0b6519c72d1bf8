"""Batched solves (lbm_batch_*): every lattice of a batch of uneven sizes
gives the same steps and efficiency as its own lbm_adr_solve (the per-node
arithmetic is shared), in every precision; the autotuner picks a valid
launch shape; reduced precisions stay within their efficiency tolerance of
the FP64 batch; and the batch itself matches the FP64 CPU oracle lattice by
lattice (concentration fields and outfluxes, Sec. III.A.2-3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
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


# ---------------------------------------------------------------------------
# the batch against the oracle
# ---------------------------------------------------------------------------
ORACLE_STEPS = 4000


@pytest.fixture(scope="module")
def oracle_lattices():
    """Four lattices of uneven, ragged size (nx not a multiple of 32), each
    with an A->B band and a band of side-by-side fibers, one relaxed
    catalyst weight and one inert fiber; their own tau and rates; flux plane
    just behind the second band.  The oracle computes its own flow."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04455_gb300 import _build
    _build.build()
    oracle.build()
    out = []
    for i, (nx, ny) in enumerate([(301, 64), (173, 45), (419, 96), (97, 30)]):
        rng = inputs.SplitMix64(200 + i)
        rows = inputs.place_fibers(rng, 0.2 * nx, 0.45 * nx, ny, 3, 3, 5,
                                   2.0, lambda r: (1, 0.0))
        rows += inputs.place_fibers(
            rng, 0.5 * nx, 0.78 * nx, ny, 3, 3, 5, 2.0,
            lambda r: (3, r.uniform_range(0, 6.28)),
            [(f[0], f[1], f[2]) for f in rows])
        rows[1][5] = 0.3 + 0.1 * i          # relaxed weight
        rows[-1][3] = 0.0                   # inert
        fib = np.asarray(rows)
        k1, k2 = 0.1 + 0.05 * i, 0.15
        taus = [0.62 + 0.05 * i, 0.7, 0.8 - 0.04 * i]
        xp = int(0.85 * nx)
        solid, kab, kbc = oracle.raster(nx, ny, fib, k1, k2)
        _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, 1500)
        prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, taus, [1, 0, 0])
        ref = prob.run(ORACLE_STEPS, xp=xp)
        geom = lbm.Geometry(nx, ny, fib, k1, k2).upload()
        u64, _ = lbm.lbm_flow_solve(geom, 0.8, 0.05, 1500,
                                    precision=lbm.LBM_F64)
        out.append((geom, u64, taus, xp, ref))
    return out


def _oracle_batch(lats, prec):
    params = [lbm.adr_params(3, taus, precision=prec,
                             max_steps=ORACLE_STEPS, tol=0.0,
                             check_every=200, x_plane=xp)
              for (_, _, taus, xp, _) in lats]
    us = [u if prec == lbm.LBM_F64 else u.float() for (_, u, _, _, _) in lats]
    return lbm.Batch([g for (g, _, _, _, _) in lats], params, us)


def test_batch_f64_matches_oracle(oracle_lattices):
    b = _oracle_batch(oracle_lattices, lbm.LBM_F64)
    infos = b.solve()
    for i, ((geom, _, _, _, ref), inf) in enumerate(zip(oracle_lattices,
                                                        infos)):
        assert inf["steps"] == ORACLE_STEPS
        c = b.conc(i).cpu().numpy()[:, :, :geom.nx]
        rel = np.linalg.norm(c - ref["conc"]) / np.linalg.norm(ref["conc"])
        assert rel < 1e-10, (i, rel)
        assert np.allclose(inf["flux"], ref["flux"], rtol=1e-10,
                           atol=1e-15), (i, inf["flux"], ref["flux"])
        assert abs(inf["eps"] - ref["eps"]) < 1e-10
        assert ref["flux"][1] > 1e-3 * ref["flux"][0]
        assert ref["flux"][2] > 1e-5 * ref["flux"][0]
        # the check steps also report the most negative concentration
        assert all(-1e-6 < m <= 0.0 for m in inf["c_min"])


@pytest.mark.parametrize("prec,tol", [(lbm.LBM_F32, 1e-4),
                                      (lbm.LBM_F16DEV, 1e-3)])
def test_batch_reduced_precision_matches_oracle(oracle_lattices, prec, tol):
    b = _oracle_batch(oracle_lattices, prec)
    infos = b.solve()
    for (geom, _, _, _, ref), inf in zip(oracle_lattices, infos):
        assert abs(inf["eps"] - ref["eps"]) < tol
        # each species' share of the outflux, which the tolerance resolves
        got = np.array(inf["flux"]) / sum(inf["flux"])
        want = np.asarray(ref["flux"]) / sum(ref["flux"])
        assert np.abs(got - want).max() < tol
        assert want[1] > 10 * tol
