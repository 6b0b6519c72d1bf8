"""lbm_adr_outflux_noalloc: the outflux entry point for callers that cannot
allocate device memory (it keeps its partial sums in a fixed device array of
the library instead of a caller workspace).  Its values must equal those of
the regular path (lbm_adr_run with info), call after call.  This file is
collected last so that a failure here cannot hide any other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2109_04455_gb300 import inputs, lbm  # noqa: E402

pytestmark = pytest.mark.gpu
PLANE = 130


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04455_gb300 import _build
    _build.build()
    lbm.load()


def _solver(prec, nx=261, ny=37):
    rng = inputs.SplitMix64(11)
    rows = inputs.place_fibers(rng, 40, 120, ny, 5, 3, 5, 2.0,
                               lambda r: (1, 0.0))
    rows += inputs.place_fibers(rng, 140, 220, ny, 5, 3, 5, 2.0,
                                lambda r: (2, 0.0),
                                [(f[0], f[1], f[2]) for f in rows])
    geom = lbm.Geometry(nx, ny, np.asarray(rows), 0.05, 0.07).upload()
    flow_prec = lbm.LBM_F64 if prec == lbm.LBM_F64 else lbm.LBM_F32
    u, _ = lbm.lbm_flow_solve(geom, 0.8, 0.05, 500, precision=flow_prec)
    # flux plane just downstream of the A->B fibers, where B is present
    prm = lbm.adr_params(3, [0.62] * 3, precision=prec, x_plane=PLANE)
    return geom, lbm.ADRSolver(geom, prm, u).init()


@pytest.mark.parametrize("prec", [lbm.LBM_F64, lbm.LBM_F32, lbm.LBM_F16DEV])
def test_outflux_noalloc_matches_regular_path(prec):
    geom, sv = _solver(prec)
    for nsteps in (400, 250):          # two calls in a row
        info = sv.run(nsteps)
        got = lbm.lbm_adr_outflux_noalloc(sv, x_plane=PLANE)
        # same double sums of the same stored values, in another order
        assert np.allclose(got, info["flux"], rtol=1e-12, atol=1e-15)
    assert abs(got[0]) > 0 and abs(got[1]) > 0


@pytest.mark.parametrize("prec", [lbm.LBM_F64, lbm.LBM_F32, lbm.LBM_F16DEV])
def test_outflux_noalloc_many_row_blocks(prec):
    """ny = 600 spans three 256-row blocks of the partial kernel, so the
    final kernel folds several block partials before dividing by ny."""
    geom, sv = _solver(prec, nx=261, ny=600)
    for nsteps in (300, 200):
        info = sv.run(nsteps)
        got = lbm.lbm_adr_outflux_noalloc(sv, x_plane=PLANE)
        assert np.allclose(got, info["flux"], rtol=1e-12, atol=1e-15)
    assert abs(got[0]) > 0 and abs(got[1]) > 0


def test_outflux_noalloc_rejects_plane_outside():
    geom, sv = _solver(lbm.LBM_F32)
    sv.run(10)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_adr_outflux_noalloc(sv, x_plane=geom.nx)
    assert e.value.status == lbm.LBM_EINVAL
