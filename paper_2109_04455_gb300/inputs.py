"""Seeded synthetic inputs: fiber tables and run parameters.

This module is shared by the GPU path and by the CPU oracle used in the tests.
It holds no arithmetic of the lattice method itself: only the random
placement of fibers, the workload sizes and the conversion of the paper's
dimensionless numbers into lattice parameters.

Fiber table format (float64, one row per fiber, 6 columns):
    cx, cy, r, cat, janus_angle, weight
cat 0 inert, 1 catalyses A->B, 2 catalyses B->C, 3 side-by-side (both
catalysts, split by the line through the centre normal to
(cos janus_angle, sin janus_angle)).  weight in [0, 1] marks a relaxed
catalyst assignment (rates weight*k1 and (1-weight)*k2); -1 means none.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so that the
same seed gives the same fibers on any machine.  Doubles are the top 53 bits
scaled by 2^-53.

Parameter conversion follows Sec. II.A of the paper: Pe = u0 R / D and
Da = k R^2 / D, with D = c_s^2 (tau - 1/2) (Eq. Diffusion_LBM, c_s^2 = 1/3),
so D = u0 R / Pe, tau = 3 D + 1/2 and k = Da D / R^2 (k per time step).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream (state advanced by the golden-ratio increment)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))


# ---------------------------------------------------------------------------
# parameters (Sec. II.A)
# ---------------------------------------------------------------------------
def diffusivity_from_pe(u0: float, r: float, pe: float) -> float:
    """D = u0 R / Pe."""
    return u0 * r / pe


def tau_from_diffusivity(d: float) -> float:
    """Inverse of D = c_s^2 (tau - 1/2) with c_s^2 = 1/3."""
    return 3.0 * d + 0.5


def rate_from_da(da: float, d: float, r: float) -> float:
    """k = Da D / R^2 (per time step)."""
    return da * d / (r * r)


def da_from_rate(k: float, d: float, r: float) -> float:
    return k * r * r / d


# ---------------------------------------------------------------------------
# fiber placement
# ---------------------------------------------------------------------------
def place_fibers(rng: SplitMix64, x0: float, x1: float, ny: int, count: int,
                 r_lo: int, r_hi: int, gap: float, cat_fn,
                 existing=None, max_tries: int = 200000) -> list:
    """Sequential rejection sampling of ``count`` discs in the band
    x in [x0, x1] of a channel of height ``ny``.

    Radius: integer uniform in [r_lo, r_hi].  Centre: uniform real in
    [x0 + R, x1 - R] x [R + gap, ny - 1 - R - gap] (no disc touches a wall).
    A candidate is rejected if its surface gap to any placed disc is below
    ``gap``.  ``cat_fn(rng)`` returns (cat, janus_angle) for an accepted disc.
    """
    placed = list(existing or [])
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(
                f"could not place {count} fibers in band [{x0},{x1}] "
                f"(placed {len(out)})")
        r = rng.randint(r_lo, r_hi) if r_hi > r_lo else r_lo
        cx = rng.uniform_range(x0 + r, x1 - r)
        cy = rng.uniform_range(r + gap, ny - 1 - r - gap)
        ok = True
        for (px, py, pr) in placed:
            if math.hypot(cx - px, cy - py) < r + pr + gap:
                ok = False
                break
        if not ok:
            continue
        cat, ang = cat_fn(rng)
        placed.append((cx, cy, r))
        out.append([cx, cy, float(r), float(cat), ang, -1.0])
    return out


def fiber_table(rows) -> np.ndarray:
    a = np.asarray(rows, dtype=np.float64).reshape(-1, 6)
    return np.ascontiguousarray(a)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    """One lattice problem: geometry + flow + ADR parameters."""
    name: str
    nx: int
    ny: int
    fibers: np.ndarray          # (n, 6) fiber table
    nspecies: int               # 2: A->B, 3: A->B->C
    u0: float = 0.05            # inflow centreline velocity
    tau_flow: float = 0.8       # flow relaxation time
    pe: float = 10.0
    da1: float = 1.0
    da2: float = 1.0
    r_ref: float = 8.0          # radius used in Pe and Da
    c_in: tuple = (1.0, 0.0, 0.0)
    flow_steps: int = 20000
    adr_steps: int = 20000

    @property
    def diffusivity(self) -> float:
        return diffusivity_from_pe(self.u0, self.r_ref, self.pe)

    @property
    def tau_c(self) -> float:
        return tau_from_diffusivity(self.diffusivity)

    @property
    def k1(self) -> float:
        return rate_from_da(self.da1, self.diffusivity, self.r_ref)

    @property
    def k2(self) -> float:
        return rate_from_da(self.da2, self.diffusivity, self.r_ref)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny


def single_fiber(nx: int = 200, ny: int = 100, cx: float = 60.0,
                 cy: float = 50.0, r: float = 8.0, pe: float = 10.0,
                 da: float = 1.0, flow_steps: int = 20000,
                 adr_steps: int = 20000) -> Workload:
    """One A->B catalyst cylinder in a channel (2D analogue of Sec. II.B):
    200x100 channel, R = 8 at (60, 50), u0 = 0.05, tau = 0.8, Pe = 10,
    Da = 1, 20000 flow and 20000 ADR steps."""
    fib = fiber_table([[cx, cy, r, 1.0, 0.0, -1.0]])
    return Workload("single_fiber_AB", nx, ny, fib, 2, pe=pe, da1=da, da2=da,
                    r_ref=r, flow_steps=flow_steps, adr_steps=adr_steps)


def isolated_fiber(pe: float, da: float, nx: int = 300, ny: int = 300,
                   r: float = 5.0) -> Workload:
    """Isolated A->B cylinder of Sec. II.B in the 2D channel: R = 5 in the
    middle of a 300 x 300 box, species A and B."""
    fib = fiber_table([[nx / 2.0, ny / 2.0, r, 1.0, 0.0, -1.0]])
    return Workload(f"isolated_fiber_pe{pe:g}_da{da:g}", nx, ny, fib, 2,
                    pe=pe, da1=da, da2=da, r_ref=r)


def fiber_pair(xi: float, pe: float, da: float = 150.0, nx: int = 1000,
               ny: int = 300, r: float = 5.0, x1: float = 300.0) -> Workload:
    """Cascade on two single-catalyst cylinders of Sec. II.C: R = 5, an A->B
    fiber at (x1, ny/2) and a B->C fiber downstream on the same streamline,
    their surfaces xi apart (centres 2R + xi apart), 1000 x 300 box."""
    x2 = x1 + 2.0 * r + xi
    fib = fiber_table([[x1, ny / 2.0, r, 1.0, 0.0, -1.0],
                       [x2, ny / 2.0, r, 2.0, 0.0, -1.0]])
    return Workload(f"fiber_pair_xi{xi:g}_pe{pe:g}_da{da:g}", nx, ny, fib, 3,
                    pe=pe, da1=da, da2=da, r_ref=r)


def side_by_side_fiber(pe: float, da: float = 150.0, nx: int = 1000,
                       ny: int = 300, r: float = 10.0,
                       x1: float = 300.0) -> Workload:
    """Side-by-side morphology of Sec. II.C: one R = 10 cylinder carrying
    both catalysts, A->B on its upstream half and B->C on its downstream half
    (interface across the flow), 1000 x 300 box."""
    fib = fiber_table([[x1, ny / 2.0, r, 3.0, math.pi, -1.0]])
    return Workload(f"side_by_side_pe{pe:g}_da{da:g}", nx, ny, fib, 3,
                    pe=pe, da1=da, da2=da, r_ref=r)


def fiber_membrane(pe: float, da: float = 150.0, seed: int = 0,
                   cascade: bool = False, n: int = 6, nx: int = 1000,
                   ny: int = 300, r: int = 5, gap: float = 4.0) -> Workload:
    """2D analogue of the membranes of Sec. IV (n randomly placed R = 5
    fibers, seeded): one A->B membrane in the band x in [300, 400], and for
    the cascade a B->C membrane in [450, 550] behind it; 1000 x 300 box."""
    rng = SplitMix64(1000 + seed)
    rows = place_fibers(rng, 300, 400, ny, n, r, r, gap, lambda _r: (1, 0.0))
    ns = 2
    if cascade:
        rows += place_fibers(rng, 450, 550, ny, n, r, r, gap,
                             lambda _r: (2, 0.0),
                             [(f[0], f[1], f[2]) for f in rows])
        ns = 3
    kind = "cascade" if cascade else "AB"
    return Workload(f"membrane_{kind}_seed{seed}_pe{pe:g}_da{da:g}", nx, ny,
                    fiber_table(rows), ns, pe=pe, da1=da, da2=da,
                    r_ref=float(r))


def two_membrane_cascade(seed: int = 0, pe: float = 10.0, nx: int = 2048,
                         ny: int = 512, bands=((400, 700), (1000, 1300)),
                         per_band: int = 40, r: int = 8,
                         gap: float = 4.0) -> Workload:
    """A->B->C through two random membranes (2D analogue of Sec. II.C):
    membrane 1 fibers catalyse A->B, membrane 2 fibers B->C."""
    rng = SplitMix64(seed)
    rows = []
    existing = []
    for b, (x0, x1) in enumerate(bands):
        cat = 1 if b % 2 == 0 else 2
        got = place_fibers(rng, x0, x1, ny, per_band, r, r, gap,
                           lambda _r, c=cat: (c, 0.0), existing)
        existing += [(f[0], f[1], f[2]) for f in got]
        rows += got
    return Workload(f"cascade_{nx}x{ny}_seed{seed}_pe{pe:g}", nx, ny,
                    fiber_table(rows), 3, pe=pe, r_ref=float(r))


def large_membrane(seed: int = 0, nx: int = 16384, ny: int = 4096,
                   per_band: int = 500, r: int = 8, gap: float = 4.0,
                   pe: float = 50.0, da: float = 0.5) -> Workload:
    """Large throughput lattice: four membranes in the bands
    [(2m+1)W/9, (2m+2)W/9), m = 0..3, catalysts alternating k1/k2/k1/k2."""
    rng = SplitMix64(seed)
    rows = []
    existing = []
    for m in range(4):
        x0 = (2 * m + 1) * nx / 9.0
        x1 = (2 * m + 2) * nx / 9.0
        cat = 1 if m % 2 == 0 else 2
        got = place_fibers(rng, x0, x1, ny, per_band, r, r, gap,
                           lambda _r, c=cat: (c, 0.0), existing)
        existing += [(f[0], f[1], f[2]) for f in got]
        rows += got
    return Workload(f"large_membrane_{nx}x{ny}_{4 * per_band}fibers", nx, ny,
                    fiber_table(rows), 3, pe=pe, da1=da, da2=da,
                    r_ref=float(r))


def sweep_instance(i: int, n_pe: int = 8, n_da: int = 8) -> Workload:
    """Instance ``i`` of the Pe x Da sweep: Pe = logspace(-1, 2, 8),
    Da = logspace(-2, 2, 8); width uniform in [512, 2048] and height in
    [256, 512] (multiples of 32); 20-120 fibers of R = 6..10 in one or two
    membranes, about half of them side-by-side."""
    rng = SplitMix64(0x5EED0000 + i)
    pes = np.logspace(-1, 2, n_pe)
    das = np.logspace(-2, 2, n_da)
    pe = float(pes[i // n_da % n_pe])
    da = float(das[i % n_da])
    nx = 32 * rng.randint(16, 64)
    ny = 32 * rng.randint(8, 16)
    nfib = rng.randint(20, 120)
    two = rng.uniform() < 0.5
    if two:
        bands = [(0.2 * nx, 0.45 * nx), (0.55 * nx, 0.8 * nx)]
    else:
        bands = [(0.25 * nx, 0.5 * nx)]

    def cat_fn(rr, band):
        if rr.uniform() < 0.5:
            return 3, rr.uniform_range(0.0, 2.0 * math.pi)
        return (1 if band == 0 or not two else 2), 0.0

    rows = []
    existing = []
    per = [nfib // len(bands) + (1 if b < nfib % len(bands) else 0)
           for b in range(len(bands))]
    for b, (x0, x1) in enumerate(bands):
        # cap the count to what fits comfortably in the band
        area = (x1 - x0) * (ny - 28.0)
        cap = max(1, int(area / (math.pi * 16.0 ** 2) * 0.6))
        got = place_fibers(rng, x0, x1, ny, min(per[b], cap), 6, 10, 4.0,
                           lambda rr, bb=b: cat_fn(rr, bb), existing)
        existing += [(f[0], f[1], f[2]) for f in got]
        rows += got
    return Workload(f"sweep_{i}", nx, ny, fiber_table(rows), 3, pe=pe,
                    da1=da, da2=da, r_ref=8.0)


def noflow_box(kind: str, da: float, n: int = 300, xi: float = 100.0,
               tau: float = 1.0) -> Workload:
    """Pure-diffusion cascade of Sec. IV.B: an n x n box, periodic in both
    directions, filled with A, no flow.  kind "pair": an A->B and a B->C
    fiber of R = 5 on the box's centre line, their surfaces xi apart;
    kind "side_by_side": one R = 10 fiber carrying both catalysts (A->B on
    the half facing -x, B->C on the other), the same total surface.  With no
    flow Pe is not defined: D follows from tau (the paper's tau = 1,
    D = 1/6) and k = Da D / R^2 from each geometry's own R."""
    d = (tau - 0.5) / 3.0
    if kind == "pair":
        r = 5.0
        x1 = n / 2.0 - r - xi / 2.0
        fib = fiber_table([[x1, n / 2.0, r, 1.0, 0.0, -1.0],
                           [x1 + 2.0 * r + xi, n / 2.0, r, 2.0, 0.0, -1.0]])
    elif kind == "side_by_side":
        r = 10.0
        fib = fiber_table([[n / 2.0, n / 2.0, r, 3.0, math.pi, -1.0]])
    else:
        raise ValueError(kind)
    pe = 0.05 * r / d          # placeholder u0 = 0.05: only D matters here
    return Workload(f"noflow_{kind}_da{da:g}", n, n, fib, 3, pe=pe, da1=da,
                    da2=da, r_ref=r)


def empty_channel(nx: int, ny: int) -> np.ndarray:
    return np.zeros((0, 6), dtype=np.float64)
