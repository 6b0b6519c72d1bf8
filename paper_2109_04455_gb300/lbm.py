"""ctypes binding of ``liblbm.so`` (C ABI in ``include/lbm.h``).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  PyTorch provides device memory (``torch.empty`` on ``cuda``)
and streams; the library itself never allocates device memory.  If the
library has not been built, :func:`load` raises -- there is no other path.

Function names follow the C ABI (``lbm_geometry_create`` ...); the small
classes below only own the handles and the torch buffers they borrow.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the library (e.g. one compiled with
# other launch-shape options); by default the in-tree build.
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENOTCONVERGED, \
    LBM_EUNSTABLE = range(6)
LBM_F64, LBM_F32, LBM_F16DEV = range(3)
LBM_ADR_INLET_ABB_ALL = 1
LBM_ADR_NODEWISE = 2
LBM_PERIODIC_X = 1
LBM_PERIODIC_Y = 2
PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32, "f16dev": LBM_F16DEV}

_STATUS = {LBM_EINVAL: "EINVAL", LBM_ENOMEM: "ENOMEM", LBM_ECUDA: "ECUDA",
           LBM_ENOTCONVERGED: "ENOTCONVERGED", LBM_EUNSTABLE: "EUNSTABLE"}


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class lbm_solve_info(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("residual", ctypes.c_double),
                ("converged", ctypes.c_int32),
                ("flux", ctypes.c_double * 3), ("eps", ctypes.c_double),
                ("c_min", ctypes.c_double * 3), ("mass", ctypes.c_double * 3)]

    def as_dict(self):
        return dict(steps=int(self.steps), residual=float(self.residual),
                    converged=bool(self.converged),
                    flux=[float(v) for v in self.flux], eps=float(self.eps),
                    c_min=[float(v) for v in self.c_min],
                    mass=[float(v) for v in self.mass])


class lbm_flow_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("u0", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("tol", ctypes.c_double),
                ("check_every", ctypes.c_int32),
                ("precision", ctypes.c_int32)]


class lbm_adr_params(ctypes.Structure):
    _fields_ = [("nspecies", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tau", ctypes.c_double * 3), ("c_in", ctypes.c_double * 3),
                ("max_steps", ctypes.c_int64), ("tol", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("x_plane", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("neg_tol", ctypes.c_double),
                ("eps_tol", ctypes.c_double)]


class lbm_rwpt_params(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("dt", ctypes.c_double),
                ("delta", ctypes.c_double), ("density", ctypes.c_double),
                ("radius_offset", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("nspecies", ctypes.c_int32), ("flags", ctypes.c_int32)]


class lbm_rwpt_info(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("window_steps", ctypes.c_int64),
                ("alive", ctypes.c_int64), ("out", ctypes.c_int64 * 3),
                ("eps", ctypes.c_double), ("overflow", ctypes.c_int32)]

    def as_dict(self):
        return dict(steps=int(self.steps),
                    window_steps=int(self.window_steps),
                    alive=int(self.alive), out=[int(v) for v in self.out],
                    eps=float(self.eps), overflow=bool(self.overflow))


LBM_RWPT_PERIODIC = 1
LBM_RWPT_HOMOGENEOUS = 2


# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_geometry_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P,
                                           ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_double, _P]),
    "lbm_geometry_destroy": (None, [_P]),
    "lbm_geometry_info": (ctypes.c_int, [_P, _P, _P]),
    "lbm_geometry_fields": (ctypes.c_int, [_P, _P, _P, _P]),
    "lbm_geometry_set_rates": (ctypes.c_int, [_P, _P, _P]),
    "lbm_geometry_set_periodic": (ctypes.c_int, [_P, ctypes.c_int32]),
    "lbm_adr_state_bytes": (ctypes.c_size_t, [_P]),
    "lbm_adr_state_save": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "lbm_adr_state_load": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "lbm_geometry_ws_bytes": (ctypes.c_size_t, [_P]),
    "lbm_geometry_upload": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "lbm_flow_ws_bytes": (ctypes.c_size_t, [_P, ctypes.c_int32]),
    "lbm_flow_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t, _P, _P,
                                      _P]),
    "lbm_adr_ws_bytes": (ctypes.c_size_t, [_P, _P]),
    "lbm_adr_create": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_size_t, _P]),
    "lbm_adr_destroy": (None, [_P]),
    "lbm_adr_init": (ctypes.c_int, [_P, _P]),
    "lbm_adr_run": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P]),
    "lbm_adr_conc": (ctypes.c_int, [_P, _P, _P]),
    "lbm_adr_solve": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_size_t, _P, _P,
                                     _P]),
    "lbm_efficiency": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "lbm_fp64_fma_tflops": (ctypes.c_int, [_P, _P]),
    "lbm_adr_outflux_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "lbm_batch_ws_bytes": (ctypes.c_size_t, [ctypes.c_int32, _P, _P]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P,
                                        ctypes.c_size_t, _P]),
    "lbm_batch_destroy": (None, [_P]),
    "lbm_batch_tune": (ctypes.c_int, [_P, _P, _P, _P]),
    "lbm_batch_tuning": (ctypes.c_int, [_P, _P, _P, _P]),
    "lbm_batch_solve": (ctypes.c_int, [_P, _P, _P]),
    "lbm_batch_conc": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "lbm_rwpt_ws_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int32]),
    "lbm_rwpt_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P,
                                       ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_double, _P, _P,
                                       ctypes.c_int64, _P, ctypes.c_size_t,
                                       _P]),
    "lbm_rwpt_destroy": (None, [_P]),
    "lbm_rwpt_init": (ctypes.c_int, [_P, _P]),
    "lbm_rwpt_run": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P]),
    "lbm_rwpt_reset_counts": (ctypes.c_int, [_P, _P]),
    "lbm_rwpt_particles": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P,
                                          _P, _P]),
    "lbm_adr_adjoint_ws_bytes": (ctypes.c_size_t, [_P, _P]),
    "lbm_adr_adjoint": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_int32, _P, ctypes.c_size_t,
                                       _P, _P, _P, _P, _P]),
}

_lib = None


def load():
    """Open liblbm.so (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int):
    if status != LBM_OK:
        raise LBMError(status, load().lbm_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _device_bytes(nbytes: int, device="cuda"):
    import torch
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def lbm_fp64_fma_tflops(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device (TFLOP/s)."""
    v = ctypes.c_double()
    _check(load().lbm_fp64_fma_tflops(_stream_ptr(stream), ctypes.byref(v)))
    return v.value


def lbm_efficiency(flux, nspecies: int) -> float:
    f = (ctypes.c_double * 3)(*[float(v) for v in list(flux)[:3]] +
                              [0.0] * (3 - min(3, len(list(flux)))))
    eps = ctypes.c_double()
    _check(load().lbm_efficiency(f, nspecies, ctypes.byref(eps)))
    return eps.value


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
class Geometry:
    """Host raster (lbm_geometry_create) plus its device copy."""

    def __init__(self, nx: int, ny: int, fibers, k1: float, k2: float):
        lib = load()
        fib = np.ascontiguousarray(np.asarray(fibers, dtype=np.float64)
                                   .reshape(-1, 6))
        self._fib = fib
        h = ctypes.c_void_p()
        _check(lib.lbm_geometry_create(nx, ny, fib.ctypes.data_as(_P),
                                       fib.shape[0], k1, k2, ctypes.byref(h)))
        self.handle = h
        self.nx, self.ny = nx, ny
        pad = ctypes.c_int32()
        nsol = ctypes.c_int64()
        _check(lib.lbm_geometry_info(h, ctypes.byref(pad), ctypes.byref(nsol)))
        self.nx_pad = pad.value
        self.n_solid = nsol.value
        self.ws = None

    def fields(self):
        """Host solid mask (uint8 [ny, nx]) and rates k_AB, k_BC."""
        solid = np.zeros((self.ny, self.nx), np.uint8)
        kab = np.zeros((self.ny, self.nx))
        kbc = np.zeros((self.ny, self.nx))
        _check(load().lbm_geometry_fields(self.handle,
                                          solid.ctypes.data_as(_P),
                                          kab.ctypes.data_as(_P),
                                          kbc.ctypes.data_as(_P)))
        return solid, kab, kbc

    def ws_bytes(self) -> int:
        return int(load().lbm_geometry_ws_bytes(self.handle))

    def set_rates(self, kab=None, kbc=None):
        """lbm_geometry_set_rates: per-node rate fields ([ny, nx] float64,
        zero on fluid nodes; None keeps that rate).  Call upload() again
        before the next solve (it rewrites the same device buffer)."""
        arrs = []
        for f in (kab, kbc):
            arrs.append(None if f is None else np.ascontiguousarray(
                np.asarray(f, dtype=np.float64).reshape(self.ny, self.nx)))
        _check(load().lbm_geometry_set_rates(
            self.handle, *[a.ctypes.data_as(_P) if a is not None else None
                           for a in arrs]))
        return self

    def set_periodic(self, flags: int):
        """lbm_geometry_set_periodic: LBM_PERIODIC_X | LBM_PERIODIC_Y joins
        those edges (0: inlet, outlet and walls).  Call upload() again
        before the next solve."""
        _check(load().lbm_geometry_set_periodic(self.handle, int(flags)))
        return self

    def upload(self, device="cuda", stream=None):
        import torch
        nbytes = self.ws_bytes()
        dev = torch.device(device)
        if dev.type == "cuda" and dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        if not (self.ws is not None and self.ws.numel() == nbytes and
                self.ws.device == dev):
            self.ws = _device_bytes(nbytes, dev)
        _check(load().lbm_geometry_upload(self.handle,
                                          ctypes.c_void_p(self.ws.data_ptr()),
                                          self.ws.numel(),
                                          _stream_ptr(stream)))
        return self

    def close(self):
        if self.handle:
            load().lbm_geometry_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _field_dtype(precision: int):
    import torch
    return torch.float64 if precision == LBM_F64 else torch.float32


def lbm_flow_solve(geom: Geometry, tau: float, u0: float, max_steps: int,
                   tol: float = 0.0, check_every: int = 100,
                   precision: int = LBM_F64, stream=None, u_out=None,
                   raise_not_converged: bool = False):
    """Run the flow lattice; returns (u [2, ny, nx_pad] on the device, info).
    LBM_ENOTCONVERGED is reported in info (converged = False) unless
    ``raise_not_converged``."""
    import torch
    lib = load()
    p = lbm_flow_params(tau, u0, int(max_steps), tol, int(check_every),
                        precision)
    ws = _device_bytes(lib.lbm_flow_ws_bytes(geom.handle, precision),
                       geom.ws.device)
    if u_out is None:
        u_out = torch.zeros((2, geom.ny, geom.nx_pad),
                            dtype=_field_dtype(precision),
                            device=geom.ws.device)
    info = lbm_solve_info()
    st = lib.lbm_flow_solve(geom.handle, ctypes.byref(p),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                            ctypes.c_void_p(u_out.data_ptr()),
                            _stream_ptr(stream), ctypes.byref(info))
    if st != LBM_OK and not (st == LBM_ENOTCONVERGED and
                             not raise_not_converged):
        _check(st)
    return u_out, info.as_dict()


def adr_params(nspecies: int, tau, c_in=(1.0, 0.0, 0.0),
               precision: int = LBM_F64, max_steps: int = 0, tol: float = 0.0,
               check_every: int = 100, x_plane: int = -1,
               flags: int = 0, neg_tol: float = 0.0,
               eps_tol: float = 0.0) -> lbm_adr_params:
    """ADR settings; neg_tol 0 keeps the library's default (LBM_EUNSTABLE
    below -0.1 max(1, c_in)), < 0 turns the negative-concentration test
    off; eps_tol > 0 adds the efficiency test to the steady-state
    criterion of lbm_adr_solve and Batch.solve (see include/lbm.h)."""
    taus = list(tau) if hasattr(tau, "__len__") else [tau] * nspecies
    taus = (taus + [1.0] * 3)[:3]
    cin = (list(c_in) + [0.0] * 3)[:3]
    return lbm_adr_params(nspecies, precision, (ctypes.c_double * 3)(*taus),
                          (ctypes.c_double * 3)(*cin), int(max_steps), tol,
                          int(check_every), x_plane, flags, float(neg_tol),
                          float(eps_tol))


class ADRSolver:
    """lbm_adr_create / init / run / conc over a torch workspace."""

    def __init__(self, geom: Geometry, params: lbm_adr_params, u):
        lib = load()
        self.geom, self.params, self.u = geom, params, u
        self.ws = _device_bytes(lib.lbm_adr_ws_bytes(geom.handle,
                                                     ctypes.byref(params)),
                                geom.ws.device)
        h = ctypes.c_void_p()
        _check(lib.lbm_adr_create(geom.handle, ctypes.byref(params),
                                  ctypes.c_void_p(u.data_ptr()),
                                  ctypes.c_void_p(self.ws.data_ptr()),
                                  self.ws.numel(), ctypes.byref(h)))
        self.handle = h

    def init(self, stream=None):
        _check(load().lbm_adr_init(self.handle, _stream_ptr(stream)))
        return self

    def run(self, nsteps: int, stream=None, check: bool = True):
        """Advance nsteps; with check=True returns the info dict (syncs)."""
        if not check:
            _check(load().lbm_adr_run(self.handle, int(nsteps),
                                      _stream_ptr(stream), None))
            return None
        info = lbm_solve_info()
        _check(load().lbm_adr_run(self.handle, int(nsteps),
                                  _stream_ptr(stream), ctypes.byref(info)))
        return info.as_dict()

    def conc(self, stream=None):
        import torch
        c = torch.empty((self.params.nspecies, self.geom.ny,
                         self.geom.nx_pad),
                        dtype=_field_dtype(self.params.precision),
                        device=self.geom.ws.device)
        _check(load().lbm_adr_conc(self.handle, ctypes.c_void_p(c.data_ptr()),
                                   _stream_ptr(stream)))
        return c

    def adjoint(self, max_steps: int, tol: float = 0.0,
                check_every: int = 100, nfibers: int = 0, stream=None,
                raise_not_converged: bool = False):
        """lbm_adr_adjoint at the current state; returns (dkab, dkbc, dw,
        info) with dkab/dkbc [ny, nx_pad] float64 on the device and dw
        [nfibers] (None if nfibers == 0)."""
        import torch
        lib = load()
        dev = self.geom.ws.device
        ws = _device_bytes(lib.lbm_adr_adjoint_ws_bytes(
            self.geom.handle, ctypes.byref(self.params)), dev)
        shape = (self.geom.ny, self.geom.nx_pad)
        dkab = torch.empty(shape, dtype=torch.float64, device=dev)
        dkbc = torch.empty(shape, dtype=torch.float64, device=dev)
        dw = (torch.empty(nfibers, dtype=torch.float64, device=dev)
              if nfibers > 0 else None)
        info = lbm_solve_info()
        st = lib.lbm_adr_adjoint(self.handle, int(max_steps), tol,
                                 int(check_every),
                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                 ctypes.c_void_p(dkab.data_ptr()),
                                 ctypes.c_void_p(dkbc.data_ptr()),
                                 ctypes.c_void_p(dw.data_ptr())
                                 if dw is not None else None,
                                 _stream_ptr(stream), ctypes.byref(info))
        if st != LBM_OK and not (st == LBM_ENOTCONVERGED and
                                 not raise_not_converged):
            _check(st)
        return dkab, dkbc, dw, info.as_dict()

    def state_save(self, stream=None) -> np.ndarray:
        """lbm_adr_state_save into a new host byte array (the checkpoint)."""
        lib = load()
        n = int(lib.lbm_adr_state_bytes(self.handle))
        buf = np.empty(n, dtype=np.uint8)
        _check(lib.lbm_adr_state_save(self.handle, buf.ctypes.data_as(_P), n,
                                      _stream_ptr(stream)))
        return buf

    def state_load(self, buf, stream=None):
        """lbm_adr_state_load from a checkpoint made by state_save."""
        b = np.ascontiguousarray(np.asarray(buf, dtype=np.uint8))
        _check(load().lbm_adr_state_load(self.handle, b.ctypes.data_as(_P),
                                         b.size, _stream_ptr(stream)))
        return self

    def solve(self, tol: float, check_every: int, max_steps: int,
              stream=None):
        """Run in chunks of check_every until the residual is below tol (or
        max_steps); returns the last info (converged flag inside)."""
        info = None
        done = 0
        while done < max_steps:
            n = min(check_every, max_steps - done)
            info = self.run(max(n, 2), stream=stream)
            done += max(n, 2)
            if info["residual"] < tol:
                info["converged"] = True
                break
        return info

    def close(self):
        if self.handle:
            load().lbm_adr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_adr_outflux_noalloc(solver: "ADRSolver", x_plane: int = -1,
                            stream=None):
    """Outfluxes N_A, N_B, N_C of the solver's current state on a plane,
    computed without any device allocation (for callers that cannot
    allocate; see include/lbm.h for the shared fixed scratch it uses)."""
    out = (ctypes.c_double * 3)()
    _check(load().lbm_adr_outflux_noalloc(solver.handle, int(x_plane),
                                          _stream_ptr(stream), out))
    return [float(v) for v in out]


def lbm_adr_solve(geom: Geometry, params: lbm_adr_params, u, stream=None,
                  want_conc: bool = True,
                  raise_not_converged: bool = False):
    """One-shot ADR solve; returns (conc or None, info)."""
    import torch
    lib = load()
    ws = _device_bytes(lib.lbm_adr_ws_bytes(geom.handle, ctypes.byref(params)),
                       geom.ws.device)
    conc = None
    if want_conc:
        conc = torch.empty((params.nspecies, geom.ny, geom.nx_pad),
                           dtype=_field_dtype(params.precision),
                           device=geom.ws.device)
    info = lbm_solve_info()
    st = lib.lbm_adr_solve(geom.handle, ctypes.byref(params),
                           ctypes.c_void_p(u.data_ptr()),
                           ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                           ctypes.c_void_p(conc.data_ptr()) if want_conc
                           else None, _stream_ptr(stream), ctypes.byref(info))
    if st != LBM_OK and not (st == LBM_ENOTCONVERGED and
                             not raise_not_converged):
        _check(st)
    return conc, info.as_dict()


# ---------------------------------------------------------------------------
# batched solves
# ---------------------------------------------------------------------------
class Batch:
    """lbm_batch_create / tune / solve over uploaded geometries, their ADR
    parameters and device velocities (all lattices share nspecies and the
    precision)."""

    def __init__(self, geoms, params, us, device="cuda"):
        lib = load()
        self.geoms, self.us = list(geoms), list(us)
        n = len(self.geoms)
        self.count = n
        self._g = (ctypes.c_void_p * n)(*[g.handle.value for g in self.geoms])
        self._p = (lbm_adr_params * n)(*params)
        self._u = (ctypes.c_void_p * n)(*[u.data_ptr() for u in self.us])
        nbytes = lib.lbm_batch_ws_bytes(n, self._g, self._p)
        if nbytes == 0:
            raise LBMError(LBM_EINVAL, "lbm_batch_ws_bytes: invalid batch")
        self.ws = _device_bytes(nbytes, device)
        h = ctypes.c_void_p()
        _check(lib.lbm_batch_create(n, self._g, self._p, self._u,
                                    ctypes.c_void_p(self.ws.data_ptr()),
                                    self.ws.numel(), ctypes.byref(h)))
        self.handle = h

    def tune(self, stream=None):
        tile, grid = ctypes.c_int32(), ctypes.c_int32()
        _check(load().lbm_batch_tune(self.handle, _stream_ptr(stream),
                                     ctypes.byref(tile), ctypes.byref(grid)))
        return tile.value, grid.value

    def conc(self, index: int, stream=None):
        """lbm_batch_conc: concentrations [nspecies, ny, nx_pad] of lattice
        ``index`` at its last checked step (its final state after solve)."""
        import torch
        g = self.geoms[index]
        prec = self._p[0].precision
        c = torch.empty((self._p[0].nspecies, g.ny, g.nx_pad),
                        dtype=_field_dtype(prec), device=self.ws.device)
        _check(load().lbm_batch_conc(self.handle, int(index),
                                     ctypes.c_void_p(c.data_ptr()),
                                     _stream_ptr(stream)))
        return c

    def tuning(self):
        tile, grid = ctypes.c_int32(), ctypes.c_int32()
        ms = (ctypes.c_float * 8)()
        _check(load().lbm_batch_tuning(self.handle, ctypes.byref(tile),
                                       ctypes.byref(grid), ms))
        return dict(tile=tile.value, grid=grid.value,
                    ms_per_step=[float(v) for v in ms])

    def solve(self, stream=None, strict: bool = False):
        """Solve every lattice; returns one info dict per lattice.  A lattice
        that stopped at its step cap (converged False) or went non-finite
        (residual NaN) is reported in its info; strict=True raises instead."""
        infos = (lbm_solve_info * self.count)()
        st = load().lbm_batch_solve(self.handle, _stream_ptr(stream), infos)
        if st != LBM_OK and (strict or st not in (LBM_ENOTCONVERGED,
                                                  LBM_EUNSTABLE)):
            _check(st)
        return [i.as_dict() for i in infos]

    def close(self):
        if self.handle:
            load().lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# random walk particle tracking
# ---------------------------------------------------------------------------
class RWPT:
    """lbm_rwpt_create / init / run over a torch workspace: particles in an
    nx x ny channel with the fibers of a 6-column table, rates k1, k2 per
    unit time, the device velocity u ([2, ny, nx_pad] float64, or None)."""

    def __init__(self, nx: int, ny: int, fibers, k1: float, k2: float,
                 u=None, D: float = 0.1, dt: float = 0.5,
                 delta: float = 0.2, density: float = 10.0,
                 radius_offset: float = 0.5, seed: int = 0,
                 nspecies: int = 2, flags: int = 0, capacity: int = 1 << 20,
                 device="cuda"):
        lib = load()
        fib = np.ascontiguousarray(np.asarray(fibers, dtype=np.float64)
                                   .reshape(-1, 6))
        self._fib = fib
        self.params = lbm_rwpt_params(D, dt, delta, density, radius_offset,
                                      int(seed), int(nspecies), int(flags))
        self.u = u
        self.capacity = int(capacity)
        self.ws = _device_bytes(lib.lbm_rwpt_ws_bytes(self.capacity,
                                                      fib.shape[0]), device)
        h = ctypes.c_void_p()
        _check(lib.lbm_rwpt_create(
            nx, ny, fib.ctypes.data_as(_P), fib.shape[0], k1, k2,
            ctypes.byref(self.params),
            ctypes.c_void_p(u.data_ptr()) if u is not None else None,
            self.capacity, ctypes.c_void_p(self.ws.data_ptr()),
            self.ws.numel(), ctypes.byref(h)))
        self.handle = h

    def init(self, stream=None):
        _check(load().lbm_rwpt_init(self.handle, _stream_ptr(stream)))
        return self

    def run(self, nsteps: int, stream=None, report: bool = True):
        if not report:
            _check(load().lbm_rwpt_run(self.handle, int(nsteps),
                                       _stream_ptr(stream), None))
            return None
        info = lbm_rwpt_info()
        _check(load().lbm_rwpt_run(self.handle, int(nsteps),
                                   _stream_ptr(stream), ctypes.byref(info)))
        return info.as_dict()

    def reset_counts(self, stream=None):
        _check(load().lbm_rwpt_reset_counts(self.handle,
                                            _stream_ptr(stream)))
        return self

    def particles(self, stream=None):
        """Host copies (x, y, species, id), sorted by id."""
        n = self.capacity
        x = np.empty(n)
        y = np.empty(n)
        s = np.empty(n, np.int32)
        ids = np.empty(n, np.uint64)
        cnt = ctypes.c_int64()
        _check(load().lbm_rwpt_particles(
            self.handle, _stream_ptr(stream), n, ctypes.byref(cnt),
            x.ctypes.data_as(_P), y.ctypes.data_as(_P), s.ctypes.data_as(_P),
            ids.ctypes.data_as(_P)))
        m = cnt.value
        o = np.argsort(ids[:m], kind="stable")
        return x[:m][o], y[:m][o], s[:m][o], ids[:m][o]

    def close(self):
        if self.handle:
            load().lbm_rwpt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
