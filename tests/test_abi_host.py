"""Host-side checks of liblbm (no GPU): the library loads and exports every
entry point the header declares, the host raster matches the oracle's
bit for bit, argument errors come back as status codes, and the host-only
efficiency call follows Eq. (A-B)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2109_04455_gb300 import inputs, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2109_04455_gb300 import _build
    _build.build()
    return lbm.load()


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(lbm_\w+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "lbm_adr_run" in names and "lbm_flow_solve" in names
    for n in names:
        assert hasattr(lib, n), f"liblbm.so does not export {n}"
    # the binding wraps each of them under the same name
    for n in names:
        assert n in lbm._SIGS, f"binding misses {n}"


@pytest.mark.parametrize("make", [
    lambda: inputs.single_fiber(),
    lambda: inputs.two_membrane_cascade(seed=1),
    lambda: inputs.sweep_instance(5),
    lambda: inputs.sweep_instance(42),
    lambda: inputs.isolated_fiber(7.0, 150.0),
    lambda: inputs.fiber_pair(2.0, 10.0),
    lambda: inputs.side_by_side_fiber(10.0),
])
def test_host_raster_matches_oracle(lib, make):
    w = make()
    fib = w.fibers.copy()
    if w.name.startswith("cascade"):
        fib[::7, 5] = 0.3   # a few relaxed catalyst weights
    g = lbm.Geometry(w.nx, w.ny, fib, w.k1, w.k2)
    s, a, b = g.fields()
    so, ao, bo = oracle.raster(w.nx, w.ny, fib, w.k1, w.k2)
    assert np.array_equal(s, so)
    assert np.array_equal(a, ao)
    assert np.array_equal(b, bo)
    assert g.n_solid == int(so.sum())
    assert g.nx_pad % 32 == 0 and g.nx_pad >= w.nx


def test_argument_errors_are_status_codes(lib):
    h = ctypes.c_void_p()
    st = lib.lbm_geometry_create(2, 5, None, 0, 0.0, 0.0, ctypes.byref(h))
    assert st == lbm.LBM_EINVAL
    assert b"nx >= 4" in lib.lbm_last_error()
    bad = np.array([[5.0, 5.0, -1.0, 1, 0, -1]])
    st = lib.lbm_geometry_create(10, 10, bad.ctypes.data_as(ctypes.c_void_p),
                                 1, 0.1, 0.1, ctypes.byref(h))
    assert st == lbm.LBM_EINVAL
    g = lbm.Geometry(16, 8, np.zeros((0, 6)), 0.0, 0.0)
    # solver calls on a geometry that was never uploaded
    p = lbm.lbm_flow_params(0.8, 0.05, 10, 0.0, 10, lbm.LBM_F32)
    info = lbm.lbm_solve_info()
    st = lib.lbm_flow_solve(g.handle, ctypes.byref(p), ctypes.c_void_p(256),
                            1 << 20, ctypes.c_void_p(512), None,
                            ctypes.byref(info))
    assert st == lbm.LBM_EINVAL and b"not uploaded" in lib.lbm_last_error()
    prm = lbm.adr_params(3, 0.5, precision=lbm.LBM_F32)
    assert lib.lbm_adr_ws_bytes(g.handle, ctypes.byref(prm)) == 0  # tau 1/2
    with pytest.raises(lbm.LBMError):
        lbm.lbm_efficiency([0.0, 0.0, 0.0], 3)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_efficiency([1.0, 0.0, 0.0], 1)
    # lattice height limit (one grid row of blocks per lattice row)
    st = lib.lbm_geometry_create(8, 65536, None, 0, 0.0, 0.0, ctypes.byref(h))
    assert st == lbm.LBM_EINVAL
    g1 = lbm.Geometry(8, 65535, np.zeros((0, 6)), 0.0, 0.0)
    assert g1.nx_pad == 32 and g1.n_solid == 0
    g1.close()
    # negative rates, unknown ADR flag bits
    st = lib.lbm_geometry_create(10, 10, None, 0, -0.1, 0.0, ctypes.byref(h))
    assert st == lbm.LBM_EINVAL
    prm = lbm.adr_params(3, 0.62, precision=lbm.LBM_F32, flags=1 << 5)
    assert lib.lbm_adr_ws_bytes(g.handle, ctypes.byref(prm)) == 0
    prm = lbm.adr_params(3, 0.62, precision=lbm.LBM_F32,
                         flags=lbm.LBM_ADR_NODEWISE |
                         lbm.LBM_ADR_INLET_ABB_ALL)
    assert lib.lbm_adr_ws_bytes(g.handle, ctypes.byref(prm)) > 0


def test_efficiency_host_call(lib):
    for flux in ([0.7, 0.2, 0.1], [3.0, 1.0, 0.0]):
        assert lbm.lbm_efficiency(flux, 3) == pytest.approx(
            oracle.efficiency(flux, 3), abs=1e-16)
        assert lbm.lbm_efficiency(flux, 2) == pytest.approx(
            oracle.efficiency(flux, 2), abs=1e-16)


def test_workspace_sizes_scale_with_precision(lib):
    g = lbm.Geometry(200, 100, inputs.single_fiber().fibers, 0.1, 0.0)
    sizes = {}
    for name, prec in lbm.PRECISIONS.items():
        prm = lbm.adr_params(3, 0.62, precision=prec)
        sizes[name] = lib.lbm_adr_ws_bytes(g.handle, ctypes.byref(prm))
    plane = g.nx_pad * 100
    # two population buffers dominate: 2 x 27 planes x element size
    assert sizes["f64"] >= 2 * 27 * plane * 8
    assert sizes["f32"] >= 2 * 27 * plane * 4
    assert sizes["f16dev"] >= 2 * 27 * plane * 2
    assert sizes["f16dev"] < sizes["f32"] < sizes["f64"]
    assert lib.lbm_geometry_ws_bytes(g.handle) >= plane * (4 + 16)


def test_set_rates_rebuilds_links_and_validates(lib):
    """lbm_geometry_set_rates: per-node rates replace the raster's, the
    catalytic / inert link types follow them, bad fields are refused and
    leave the geometry unchanged."""
    w = inputs.fiber_pair(20.0, 10.0)
    g = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2)
    solid, kab, kbc = g.fields()
    new_ab = np.where(solid == 1, 0.0, 0.0)
    ys, xs = np.nonzero(solid)
    new_ab[ys[::2], xs[::2]] = 0.125        # every other solid node
    g.set_rates(new_ab, None)
    s2, a2, b2 = g.fields()
    assert np.array_equal(s2, solid)
    assert np.array_equal(a2, new_ab) and np.array_equal(b2, kbc)
    for bad in (np.where(solid == 0, 0.1, 0.0),    # rate on a fluid node
                np.full(solid.shape, -1.0) * solid,
                np.where(solid == 1, np.nan, 0.0)):
        with pytest.raises(lbm.LBMError) as e:
            g.set_rates(bad, None)
        assert e.value.status == lbm.LBM_EINVAL
    _, a3, _ = g.fields()
    assert np.array_equal(a3, new_ab)
    # all rates zero: no catalytic links left
    g.set_rates(np.zeros(solid.shape), np.zeros(solid.shape))
    _, a4, b4 = g.fields()
    assert not a4.any() and not b4.any()


def test_set_periodic_status_and_stale_upload(lib):
    """lbm_geometry_set_periodic: unknown flags are refused; setting the
    flags rebuilds the link words and leaves the device copy stale, so a
    solver cannot be created before the next upload."""
    g = lbm.Geometry(16, 8, np.array([[8.0, 4.0, 2.0, 1, 0, -1]]), 0.1, 0.0)
    assert lib.lbm_geometry_set_periodic(g.handle, 4) == lbm.LBM_EINVAL
    assert lib.lbm_geometry_set_periodic(None, 1) == lbm.LBM_EINVAL
    for flags in (lbm.LBM_PERIODIC_X, lbm.LBM_PERIODIC_Y,
                  lbm.LBM_PERIODIC_X | lbm.LBM_PERIODIC_Y, 0):
        assert lib.lbm_geometry_set_periodic(g.handle, flags) == lbm.LBM_OK
    prm = lbm.adr_params(3, 0.8)
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(256)
    st = lib.lbm_adr_create(g.handle, ctypes.byref(prm), fake, fake, 1 << 20,
                            ctypes.byref(h))
    assert st == lbm.LBM_EINVAL
    assert b"not uploaded" in lib.lbm_last_error()
    # the raster itself does not change
    s, a, _ = g.fields()
    so, ao, _ = oracle.raster(16, 8, [[8.0, 4.0, 2.0, 1, 0, -1]], 0.1, 0.0)
    assert np.array_equal(s, so) and np.array_equal(a, ao)


def test_batch_and_particle_argument_errors(lib):
    """The batch, particle-tracking and outflux entry points check their
    arguments on the host before any device work: each refusal is a status
    code with a message, and the workspace queries return 0 for what the
    create calls would refuse."""
    g = lbm.Geometry(40, 16, np.array([[20.0, 8.0, 3.0, 1, 0, -1]]), 0.1, 0.0)
    geoms = (ctypes.c_void_p * 2)(g.handle.value, g.handle.value)
    prm = (lbm.lbm_adr_params * 2)(lbm.adr_params(3, 0.8),
                                   lbm.adr_params(3, 0.8))
    us = (ctypes.c_void_p * 2)(256, 512)
    ws = ctypes.c_void_p(4096)
    out = ctypes.c_void_p()
    # geometries that were never uploaded
    assert lib.lbm_batch_ws_bytes(2, geoms, prm) == 0
    st = lib.lbm_batch_create(2, geoms, prm, us, ws, 1 << 20,
                              ctypes.byref(out))
    assert st == lbm.LBM_EINVAL and b"uploaded" in lib.lbm_last_error()
    assert out.value is None
    assert lib.lbm_batch_create(0, geoms, prm, us, ws, 1 << 20,
                                ctypes.byref(out)) == lbm.LBM_EINVAL
    assert lib.lbm_batch_create(2, geoms, prm, us, ws, 1 << 20,
                                None) == lbm.LBM_EINVAL
    assert b"out is NULL" in lib.lbm_last_error()

    # particle tracking: workspace size grows with capacity and fibers
    assert lib.lbm_rwpt_ws_bytes(0, 1) == 0
    assert lib.lbm_rwpt_ws_bytes(10, -1) == 0
    s1 = lib.lbm_rwpt_ws_bytes(1000, 2)
    assert s1 > 0
    assert lib.lbm_rwpt_ws_bytes(2000, 2) > s1
    assert lib.lbm_rwpt_ws_bytes(1000, 20) > s1
    fib = np.array([[20.0, 8.0, 3.0, 1, 0, -1]])
    fp = fib.ctypes.data_as(ctypes.c_void_p)

    def create(nx=40, ny=16, k1=0.1, k2=0.0, capacity=1000, wsp=ws,
               nbytes=1 << 20, **kw):
        p = lbm.lbm_rwpt_params(D=kw.get("D", 0.1), dt=kw.get("dt", 0.5),
                                delta=0.2, density=1.0, radius_offset=0.5,
                                seed=1, nspecies=kw.get("nspecies", 2),
                                flags=kw.get("flags", 0))
        h = ctypes.c_void_p()
        return lib.lbm_rwpt_create(nx, ny, fp, 1, k1, k2, ctypes.byref(p),
                                   None, capacity, wsp, nbytes,
                                   ctypes.byref(h))

    assert create(nx=1) == lbm.LBM_EINVAL
    assert create(capacity=0) == lbm.LBM_EINVAL
    assert create(dt=0.0) == lbm.LBM_EINVAL
    assert create(nspecies=4) == lbm.LBM_EINVAL
    assert create(k1=3.0) == lbm.LBM_EINVAL          # k dt > 1
    assert b"k dt" in lib.lbm_last_error()
    assert create(flags=1 << 4) == lbm.LBM_EINVAL    # unknown flag bit
    assert create(wsp=ctypes.c_void_p(4096 + 16)) == lbm.LBM_EINVAL
    assert b"aligned" in lib.lbm_last_error()
    assert create(nbytes=16) == lbm.LBM_ENOMEM
    assert b"too small" in lib.lbm_last_error()

    # outflux without workspace: NULL solver or output
    flux = (ctypes.c_double * 3)()
    assert lib.lbm_adr_outflux_noalloc(None, -1, None, flux) == lbm.LBM_EINVAL
    assert b"NULL" in lib.lbm_last_error()
