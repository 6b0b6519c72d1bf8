"""Plain FP64 CPU oracle for the membrane LBM flow + ADR method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library never imports, links or runs it, and it imports nothing from the
product package: both sides meet only in the seeded input generators
(``paper_2109_04455_gb300.inputs``), which carry no arithmetic of the method.

The numerics live in ``lbm_oracle.c`` (gcc, ``-O2 -ffp-contract=off``); this
module compiles it on demand and wraps it with numpy.  What follows which
passage of the paper (Sitaru & Gekle, arXiv 2109.04455):

* ``raster``         -- fibers as discs of the 2D cross-section (Sec. II.B/C,
                        side-by-side fibers Sec. II.C), node solid iff
                        ``(x-cx)^2 + (y-cy)^2 <= R^2``.
* ``flow_*``         -- D2Q9 BGK flow with bounce-back fibers/walls, velocity
                        inlet and pressure outlet (stands in for the D3Q19
                        MRT flow of Sec. III.A.1, Eq. LBE).
* ``adr_*``          -- ADR lattice of Sec. III.A.2 (Eqs. LBE_ADE, BGK, the
                        second-order equilibrium, Diffusion_LBM, C = sum g,
                        source_lbm applied to populations streaming into a
                        reactive node) with the boundary rules of Sec.
                        III.A.3 (Eq. BC).
* ``adr_flux``       -- outflux on the plane two nodes before the outlet
                        (Sec. III.A.3).
* ``efficiency``     -- Eq. (A-B).
* ``residual``       -- relative L1 change of C per step (the paper gives no
                        steady-state criterion; this is the reading used).

Pinned by ``tests/test_oracle_pins.py`` (closed forms, exact moment
recurrences, conservation invariants, independent pull-form flow and ADR
steps on tiny domains, the dense one-step matrix built from the latter with
its steady solve and, by implicit differentiation, the exact rate gradient
the adjoint must reproduce, the paper's worked Da/k numbers).  The channel ADR efficiency of the full configurations has no
printed value in the paper: parity there is pinned only through those
invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# boundary-mode flags (mirror of the #defines in lbm_oracle.c)
PX = 1            # periodic in x
PY = 2            # periodic in y
ALLPOP = 4        # every population reacts with the node's own rates
INLET_ABB_ALL = 8  # every species gets the inlet anti-bounce-back
NODEWISE = 16     # a node with a catalytic link reacts on all populations

Q = 9
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def build_command(out=_LIB):
    return ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
            "-fopenmp", _SRC, "-o", out, "-lm"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (idempotent)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(build_command(tmp), check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            L = ctypes.c_long
            lib.orc_raster.argtypes = [I, I, I, P, D, D, P, P, P]
            lib.orc_raster.restype = I
            lib.orc_flow_init_fields.argtypes = [I, I, P, P, P, P, P]
            lib.orc_flow_init_channel.argtypes = [I, I, P, D, P]
            lib.orc_flow_moments.argtypes = [I, I, P, P, P, P, P]
            lib.orc_flow_steps.argtypes = [I, I, P, D, D, I, L, P, P]
            lib.orc_flow_steps.restype = I
            lib.orc_adr_init.argtypes = [I, I, I, P, P, P, P, P]
            lib.orc_adr_conc.argtypes = [I, I, I, P, P, P]
            lib.orc_adr_steps.argtypes = [I, I, I, P, P, P, P, P, P, P, I, L,
                                          P, P]
            lib.orc_adr_steps.restype = I
            lib.orc_adr_flux.argtypes = [I, I, I, P, P, P, P, P, P, I, P, I,
                                         P]
            lib.orc_adr_adjoint_steps.argtypes = [I, I, I, P, P, P, P, P, P, I,
                                                  P, I, L, P, P]
            lib.orc_adr_adjoint_steps.restype = I
            lib.orc_adr_gradient.argtypes = [I, I, I, P, P, P, P, P, P, I, P,
                                             I, P, P, P, P]
            lib.orc_fiber_ids.argtypes = [I, I, I, P, P]
            lib.orc_num_threads.restype = I
            _lib = lib
    return _lib


def num_threads() -> int:
    """Threads the oracle's time steps run on."""
    return int(_load().orc_num_threads())


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------
def raster(nx: int, ny: int, fibers, k1: float, k2: float):
    """Solid mask (uint8 [ny, nx]) and per-node rates k_AB, k_BC ([ny, nx]).

    ``fibers`` is an (n, 6) table: cx, cy, r, cat, janus_angle, weight.
    """
    lib = _load()
    fib = _f64(np.asarray(fibers, dtype=np.float64).reshape(-1, 6))
    solid = np.zeros((ny, nx), dtype=np.uint8)
    kab = np.zeros((ny, nx))
    kbc = np.zeros((ny, nx))
    rc = lib.orc_raster(nx, ny, fib.shape[0], _p(fib), k1, k2, _p(solid),
                        _p(kab), _p(kbc))
    if rc:
        raise ValueError("orc_raster: bad arguments")
    return solid, kab, kbc


# --------------------------------------------------------------------------
# flow
# --------------------------------------------------------------------------
def flow_init_channel(solid: np.ndarray, u0: float) -> np.ndarray:
    lib = _load()
    ny, nx = solid.shape
    f = np.zeros((ny, nx, Q))
    lib.orc_flow_init_channel(nx, ny, _p(solid), u0, _p(f))
    return f


def flow_init_fields(solid, rho, ux, uy) -> np.ndarray:
    lib = _load()
    ny, nx = solid.shape
    f = np.zeros((ny, nx, Q))
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    lib.orc_flow_init_fields(nx, ny, _p(solid), _p(rho), _p(ux), _p(uy), _p(f))
    return f


def flow_steps(f: np.ndarray, solid, tau: float, u0: float, nsteps: int,
               flags: int = 0) -> np.ndarray:
    """Advance ``f`` (in place) by ``nsteps`` BGK steps; returns ``f``."""
    lib = _load()
    ny, nx = solid.shape
    tmp = np.empty_like(f)
    rc = lib.orc_flow_steps(nx, ny, _p(solid), tau, u0, flags, int(nsteps),
                            _p(f), _p(tmp))
    if rc:
        raise ValueError("orc_flow_steps: tau must exceed 1/2")
    return f


def flow_moments(f: np.ndarray, solid):
    lib = _load()
    ny, nx = solid.shape
    rho = np.zeros((ny, nx))
    ux = np.zeros((ny, nx))
    uy = np.zeros((ny, nx))
    lib.orc_flow_moments(nx, ny, _p(solid), _p(f), _p(rho), _p(ux), _p(uy))
    return rho, ux, uy


def flow_run(solid, tau: float, u0: float, nsteps: int, flags: int = 0):
    """Channel flow from the parabolic start; returns rho, ux, uy after
    ``nsteps`` steps and the per-step residual between the last two steps."""
    f = flow_init_channel(solid, u0)
    if nsteps >= 1:
        flow_steps(f, solid, tau, u0, nsteps - 1, flags)
    _, ux0, uy0 = flow_moments(f, solid)
    if nsteps >= 1:
        flow_steps(f, solid, tau, u0, 1, flags)
    rho, ux, uy = flow_moments(f, solid)
    return rho, ux, uy, flow_residual(ux0, uy0, ux, uy)


def flow_residual(ux0, uy0, ux1, uy1) -> float:
    """sum |u(t) - u(t-1)|_1 / sum |u(t)|_1 over all nodes (0 if flat zero)."""
    num = np.abs(ux1 - ux0).sum() + np.abs(uy1 - uy0).sum()
    den = np.abs(ux1).sum() + np.abs(uy1).sum()
    return float(num / den) if den > 0 else 0.0


# --------------------------------------------------------------------------
# ADR
# --------------------------------------------------------------------------
def adr_init(solid, ux, uy, c0) -> np.ndarray:
    """g = g^eq(c0, u); ``c0`` is [ns, ny, nx]."""
    lib = _load()
    ny, nx = solid.shape
    c0 = _f64(c0)
    ns = c0.shape[0]
    g = np.zeros((ns, ny, nx, Q))
    lib.orc_adr_init(nx, ny, ns, _p(solid), _p(_f64(ux)), _p(_f64(uy)),
                     _p(c0), _p(g))
    return g


def adr_initial_conc(solid, ns: int) -> np.ndarray:
    """C_A = 1 on fluid nodes, every other species 0."""
    c0 = np.zeros((ns,) + solid.shape)
    c0[0] = (solid == 0).astype(np.float64)
    return c0


class ADRProblem:
    """Everything the ADR lattice needs besides its populations."""

    def __init__(self, solid, kab, kbc, ux, uy, tau, cin, flags: int = 0):
        self.solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.kab, self.kbc = _f64(kab), _f64(kbc)
        self.ux, self.uy = _f64(ux), _f64(uy)
        self.tau = _f64(tau)
        self.cin = _f64(cin)
        self.ns = self.tau.shape[0]
        self.flags = flags

    def init(self, c0=None) -> np.ndarray:
        if c0 is None:
            c0 = adr_initial_conc(self.solid, self.ns)
        return adr_init(self.solid, self.ux, self.uy, c0)

    def steps(self, g: np.ndarray, nsteps: int) -> np.ndarray:
        lib = _load()
        ny, nx = self.solid.shape
        tmp = np.empty_like(g)
        rc = lib.orc_adr_steps(nx, ny, self.ns, _p(self.solid), _p(self.kab),
                               _p(self.kbc), _p(self.ux), _p(self.uy),
                               _p(self.tau), _p(self.cin), self.flags,
                               int(nsteps), _p(g), _p(tmp))
        if rc:
            raise ValueError("orc_adr_steps: bad arguments")
        return g

    def conc(self, g: np.ndarray) -> np.ndarray:
        lib = _load()
        ny, nx = self.solid.shape
        c = np.zeros((self.ns, ny, nx))
        lib.orc_adr_conc(nx, ny, self.ns, _p(self.solid), _p(g), _p(c))
        return c

    def flux(self, g: np.ndarray, xp: int | None = None) -> np.ndarray:
        lib = _load()
        ny, nx = self.solid.shape
        if xp is None:
            xp = nx - 3
        out = np.zeros(3)
        lib.orc_adr_flux(nx, ny, self.ns, _p(self.solid), _p(self.kab),
                         _p(self.kbc), _p(self.ux), _p(self.uy), _p(self.tau),
                         self.flags, _p(g), int(xp), _p(out))
        return out

    def run(self, nsteps: int, g: np.ndarray | None = None, xp=None):
        """``nsteps`` steps from the initial state (or from ``g``); returns
        dict(g, conc, flux, eps, residual) at the final step."""
        if g is None:
            g = self.init()
        if nsteps >= 1:
            self.steps(g, nsteps - 1)
        c_prev = self.conc(g)
        if nsteps >= 1:
            self.steps(g, 1)
        c = self.conc(g)
        flux = self.flux(g, xp)
        eps = efficiency(flux, self.ns) if self.ns >= 2 else None
        return dict(g=g, conc=c, flux=flux, eps=eps,
                    residual=residual(c_prev, c))

    def solve(self, tol: float, check_every: int, max_steps: int, xp=None):
        """Step in chunks of ``check_every`` until the per-step residual at
        the end of a chunk is below ``tol`` or ``max_steps`` is reached."""
        g = self.init()
        done = 0
        while True:
            out = self.run(check_every, g, xp)
            g = out["g"]
            done += check_every
            if out["residual"] < tol or done >= max_steps:
                out["steps"] = done
                out["converged"] = out["residual"] < tol
                return out


def efficiency_sensitivity(flux, ns: int) -> np.ndarray:
    """d eps / d N_s of Eq. (A-B) (zeros for absent species)."""
    f = [float(v) for v in flux]
    d = np.zeros(3)
    if ns == 2:
        tot = f[0] + f[1]
        d[0] = -f[1] / tot**2
        d[1] = f[0] / tot**2
    elif ns == 3:
        tot = f[0] + f[1] + f[2]
        d[0] = d[1] = -f[2] / tot**2
        d[2] = (f[0] + f[1]) / tot**2
    else:
        raise ValueError("efficiency needs 2 or 3 species")
    return d


def fiber_ids(nx: int, ny: int, fibers) -> np.ndarray:
    """Owning fiber of each node (first in list order), -1 on fluid."""
    lib = _load()
    fib = _f64(np.asarray(fibers, dtype=np.float64).reshape(-1, 6))
    ids = np.zeros((ny, nx), dtype=np.int32)
    lib.orc_fiber_ids(nx, ny, fib.shape[0], _p(fib), _p(ids))
    return ids


def adjoint(prob: "ADRProblem", g_steady: np.ndarray, nsteps: int,
            xp: int | None = None, nu: np.ndarray | None = None):
    """Discrete adjoint of the ADR lattice at the state ``g_steady``
    (pre-collision): ``nsteps`` iterations nu <- K^T (P^T nu + l) from
    ``nu`` (zero by default), then the rate gradients.  Returns
    dict(nu, dkab, dkbc, dNds, eps)."""
    lib = _load()
    ny, nx = prob.solid.shape
    if xp is None:
        xp = nx - 3
    flux = prob.flux(g_steady, xp)
    dnds = _f64(efficiency_sensitivity(flux, prob.ns))
    if nu is None:
        nu = np.zeros_like(g_steady)
    tmp = np.empty_like(nu)
    rc = lib.orc_adr_adjoint_steps(nx, ny, prob.ns, _p(prob.solid),
                                   _p(prob.kab), _p(prob.kbc), _p(prob.ux),
                                   _p(prob.uy), _p(prob.tau), prob.flags,
                                   _p(dnds), int(xp), int(nsteps), _p(nu),
                                   _p(tmp))
    if rc:
        raise ValueError("orc_adr_adjoint_steps: bad arguments")
    dkab = np.zeros((ny, nx))
    dkbc = np.zeros((ny, nx))
    lib.orc_adr_gradient(nx, ny, prob.ns, _p(prob.solid), _p(prob.kab),
                         _p(prob.kbc), _p(prob.ux), _p(prob.uy), _p(prob.tau),
                         prob.flags, _p(dnds), int(xp), _p(g_steady), _p(nu),
                         _p(dkab), _p(dkbc))
    return dict(nu=nu, dkab=dkab, dkbc=dkbc, dNds=dnds,
                eps=efficiency(flux, prob.ns))


def fiber_weight_gradient(ids: np.ndarray, dkab: np.ndarray,
                          dkbc: np.ndarray, k1: float, k2: float,
                          nfib: int) -> np.ndarray:
    """d eps / d w_f for relaxed weights (k_AB = w k1, k_BC = (1-w) k2 on
    every node of fiber f): sum over its nodes of k1 dk_AB - k2 dk_BC."""
    out = np.zeros(nfib)
    m = ids >= 0
    np.add.at(out, ids[m], k1 * dkab[m] - k2 * dkbc[m])
    return out


def residual(c_prev: np.ndarray, c: np.ndarray) -> float:
    """max over species of sum_x |C_s(t) - C_s(t-1)| / sum_x |C_s(t)|; a
    species with zero concentration everywhere contributes 0."""
    r = 0.0
    for s in range(c.shape[0]):
        den = np.abs(c[s]).sum()
        if den > 0:
            r = max(r, float(np.abs(c[s] - c_prev[s]).sum() / den))
    return r


def efficiency(flux, ns: int) -> float:
    """Eq. (A-B): eps = N_B/(N_A+N_B) for A->B, N_C/(N_A+N_B+N_C) for the
    cascade."""
    f = [float(v) for v in flux]
    if ns == 2:
        return f[1] / (f[0] + f[1])
    if ns == 3:
        return f[2] / (f[0] + f[1] + f[2])
    raise ValueError("efficiency needs 2 or 3 species")
