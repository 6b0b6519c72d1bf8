"""The paper's 2D experiment geometries (Sec. II.B / II.C: isolated fiber,
fiber pair at surface distance xi, side-by-side fiber) on the GPU against
the oracle at a fixed step count, and the batched series runner against
single-lattice solves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
from paper_2109_04455_gb300 import inputs, lbm, series  # noqa: E402

pytestmark = pytest.mark.gpu

NFLOW, NADR = 1500, 1500


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04455_gb300 import _build
    _build.build()
    oracle.build()
    lbm.load()


CASES = {
    # name: (workload, flux plane just downstream of the catalysts, ADR
    # steps: the cascade membrane needs B to reach its second band)
    "isolated_da150": (lambda: inputs.isolated_fiber(7.0, 150.0), 170, NADR),
    "pair_xi2": (lambda: inputs.fiber_pair(2.0, 10.0), 330, NADR),
    "side_by_side": (lambda: inputs.side_by_side_fiber(10.0), 330, NADR),
    "membrane_cascade": (lambda: inputs.fiber_membrane(10.0, 150.0, 1,
                                                       cascade=True), 560,
                         4000),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_series_geometry_f64_matches_oracle(name):
    make, xp, nadr = CASES[name]
    w = make()
    ns = w.nspecies
    cin = list(w.c_in)[:ns]
    solid, kab, kbc = oracle.raster(w.nx, w.ny, w.fibers, w.k1, w.k2)
    _, ux, uy, _ = oracle.flow_run(solid, w.tau_flow, w.u0, NFLOW)
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, [w.tau_c] * ns, cin)
    ref = prob.run(nadr, xp=xp)

    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    gs, ga, gb = geom.fields()
    assert np.array_equal(gs, solid)
    assert np.array_equal(ga, kab) and np.array_equal(gb, kbc)
    u, _ = lbm.lbm_flow_solve(geom, w.tau_flow, w.u0, NFLOW,
                              precision=lbm.LBM_F64)
    ug = u.cpu().numpy()[:, :, :w.nx]
    assert np.abs(ug[0] - ux).max() < 1e-12 and np.abs(ug[1] - uy).max() < 1e-12
    prm = lbm.adr_params(ns, w.tau_c, cin, precision=lbm.LBM_F64,
                         max_steps=nadr, x_plane=xp)
    conc, info = lbm.lbm_adr_solve(geom, prm, u)
    conc = conc.cpu().numpy()[:, :, :w.nx]
    rel = np.linalg.norm(conc - ref["conc"]) / np.linalg.norm(ref["conc"])
    assert rel < 1e-10
    assert np.allclose(info["flux"][:ns], ref["flux"][:ns], rtol=1e-10,
                       atol=1e-15)
    # the first product crosses the plane (and the final one is produced)
    assert ref["flux"][1] > 1e-6
    assert ref["flux"][ns - 1] > 0.0


def test_series_runner_matches_single_solves():
    """Two Pe values per geometry, fixed step count: every row of the
    batched runner equals lbm_adr_solve of the same lattice."""
    items = series.workloads(pes=(10.0, 30.0), xis=(20.0,),
                             das_isolated=(150.0,), membrane_seeds=(0,))
    assert {k for k, _ in items} == {"isolated_fiber", "fiber_pair_xi20",
                                     "side_by_side", "membrane_AB_seed0",
                                     "membrane_cascade_seed0"}
    flows = series.solve_flows(items, flow_tol=0.0, flow_max=2000)
    rows, shapes = series.run(items, flows, precision=lbm.LBM_F32, tol=0.0,
                              max_steps=2000, check_every=500)
    assert len(rows) == len(items) and len(shapes) == 2
    by_key = {(r["geometry"], r["pe"]): r for r in rows}
    for key, w in items:
        r = by_key[(key, w.pe)]
        geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
        prm = lbm.adr_params(w.nspecies, w.tau_c, w.c_in,
                             precision=lbm.LBM_F32, max_steps=2000)
        _, info = lbm.lbm_adr_solve(geom, prm, flows[key][0].float(),
                                    want_conc=False)
        assert r["steps"] == info["steps"] == 2000
        assert abs(r["eps"] - info["eps"]) <= 1e-13
        assert r["production_rate"] == pytest.approx(
            info["flux"][w.nspecies - 1] * w.ny, rel=1e-12)
        assert ("model_eps" in r) == (key != "side_by_side")
