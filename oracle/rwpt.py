"""Plain CPU restatement of the random walk particle tracking (RWPT) of
Sec. III.B of the paper (Sitaru & Gekle, arXiv 2109.04455).

TEST INFRASTRUCTURE ONLY: used by ``tests/`` (and nothing in the product);
it imports nothing from the product package and shares no code with the
CUDA particle kernels.

Per time step dt every particle
  1. is advected: x += dt u(x), u bilinear in the LBM velocity field
     (nodes at integer positions, node indices clamped to the lattice);
  2. diffuses: x += sqrt(4 D dt) e, e a uniformly random unit vector (drawn
     by rejection from the unit disc: candidate (2 a - 1, 2 b - 1), accepted
     when 0 < |v|^2 <= 1, then normalised);
  3. reflects elastically off the channel walls y = -1/2, ny - 1/2 and off
     the fibers (discs of radius R + offset: a point at distance d < r from
     the centre goes to distance 2 r - d on the same ray);
  4. reacts with probability k dt when it lies in the shell
     r <= d < r + delta of a fiber whose catalyst acts on its species
     (A -> B at k_AB, B -> C at k_BC; side-by-side fibers by side);
  5. leaves through the outlet x >= nx - 1/2 (counted per species), or, as
     A, through the inlet x < -1/2 (back to the reservoir; B and C reflect
     there); A left in the entrance strip x < 1/2 is removed, and the strip is
     seeded anew with A at the given density.
Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a
counter-based generator.  Draw k of particle `id` at step t is output
64 t + k + 1 of the stream seeded by output id + 1 of the stream of the run's
seed; a double is the top 53 bits times 2^-53.  Every arithmetic step below
is one IEEE operation in float64 (numpy does not fuse), in the order written.
"""
from __future__ import annotations

import math

import numpy as np

U64 = np.uint64
GAMMA = U64(0x9E3779B97F4A7C15)
MUL1 = U64(0xBF58476D1CE4E5B9)
MUL2 = U64(0x94D049BB133111EB)
DRAWS = 64
TRIES = 16
REACT_DRAW = 40
SPAWN_DRAW = 48
REFLECTIONS = 4


def _round_half_up(v: float) -> int:
    """Nearest integer, halves away from zero (v >= 0)."""
    return int(math.floor(v + 0.5))


def mix64(z):
    """SplitMix64's output function (wrapping 64-bit arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.asarray(z, dtype=np.uint64)
        z = (z ^ (z >> U64(30))) * MUL1
        z = (z ^ (z >> U64(27))) * MUL2
        return z ^ (z >> U64(31))


def particle_seed(seed: int, ids):
    with np.errstate(over="ignore"):
        return mix64(U64(seed) + (np.asarray(ids, np.uint64) + U64(1)) * GAMMA)


def draw(ps, t: int, k: int):
    """Uniform doubles in [0, 1): draw k at step t of the streams ps."""
    c = U64(((t % 2**64) * DRAWS + k + 1) % 2**64)
    with np.errstate(over="ignore"):
        v = mix64(ps + c * GAMMA)
    return (v >> U64(11)).astype(np.float64) * 2.0**-53


class Particles:
    """The particle set (unordered): positions, species, ids."""

    def __init__(self):
        self.x = np.zeros(0)
        self.y = np.zeros(0)
        self.s = np.zeros(0, np.int32)
        self.id = np.zeros(0, np.uint64)

    def keep(self, m):
        self.x, self.y, self.s, self.id = (self.x[m], self.y[m], self.s[m],
                                           self.id[m])

    def append(self, x, y, s, ids):
        self.x = np.concatenate([self.x, x])
        self.y = np.concatenate([self.y, y])
        self.s = np.concatenate([self.s, s.astype(np.int32)])
        self.id = np.concatenate([self.id, ids.astype(np.uint64)])

    def sorted(self):
        o = np.argsort(self.id, kind="stable")
        return self.x[o], self.y[o], self.s[o], self.id[o]


class RWPT:
    """RWPT in an nx x ny channel with the fibers of a 6-column table
    (cx, cy, r, cat, janus_angle, weight) and rates k1, k2 per unit time;
    u is (ux, uy) on the nodes ([ny, nx] each) or None."""

    def __init__(self, nx, ny, fibers, k1, k2, u, D, dt=0.5, delta=0.2,
                 density=10.0, radius_offset=0.5, seed=0, nspecies=2,
                 periodic=False, homogeneous=False):
        self.nx, self.ny = nx, ny
        self.fib = []
        for row in np.asarray(fibers, dtype=np.float64).reshape(-1, 6):
            cx, cy, r, cat, ang, w = row
            cat = int(cat)
            kab = kbc = 0.0
            split = False
            nxv = nyv = 0.0
            if cat != 0 and w >= 0.0:
                kab, kbc = w * k1, (1.0 - w) * k2
            elif cat == 1:
                kab = k1
            elif cat == 2:
                kbc = k2
            elif cat == 3:
                kab, kbc, split = k1, k2, True
                nxv, nyv = np.cos(ang), np.sin(ang)
            self.fib.append((cx, cy, r + radius_offset, kab, kbc, split, nxv,
                             nyv))
        self.k1, self.k2 = k1, k2
        self.u = None if u is None else (np.asarray(u[0], np.float64),
                                         np.asarray(u[1], np.float64))
        self.dt = dt
        self.len = float(np.sqrt(4.0 * D * dt))
        self.delta = delta
        self.density = density
        self.seed = seed
        self.ns = nspecies
        self.periodic = periodic
        self.homogeneous = homogeneous
        self.seed_count = 0 if periodic else _round_half_up(density * ny)
        self.p = Particles()
        self.t = 0
        self.next_id = 0
        self.out = np.zeros(3, np.int64)

    # -- pieces of a step -------------------------------------------------
    def _velocity(self, x, y):
        ux_f, uy_f = self.u
        fx0, fy0 = np.floor(x), np.floor(y)
        fx, fy = x - fx0, y - fy0
        i0 = np.clip(fx0.astype(np.int64), 0, self.nx - 1)
        i1 = np.clip(fx0.astype(np.int64) + 1, 0, self.nx - 1)
        j0 = np.clip(fy0.astype(np.int64), 0, self.ny - 1)
        j1 = np.clip(fy0.astype(np.int64) + 1, 0, self.ny - 1)
        gx, gy = 1.0 - fx, 1.0 - fy
        w00, w10, w01, w11 = gx * gy, fx * gy, gx * fy, fx * fy
        ux = w00 * ux_f[j0, i0] + w10 * ux_f[j0, i1] + w01 * ux_f[j1, i0] \
            + w11 * ux_f[j1, i1]
        uy = w00 * uy_f[j0, i0] + w10 * uy_f[j0, i1] + w01 * uy_f[j1, i0] \
            + w11 * uy_f[j1, i1]
        return ux, uy

    def _direction(self, ps, t):
        n = ps.shape[0]
        v1 = np.ones(n)
        v2 = np.zeros(n)
        q = np.ones(n)
        done = np.zeros(n, bool)
        for k in range(TRIES):
            c1 = 2.0 * draw(ps, t, 2 * k) - 1.0
            c2 = 2.0 * draw(ps, t, 2 * k + 1) - 1.0
            q2 = c1 * c1 + c2 * c2
            ok = (~done) & (q2 > 0.0) & (q2 <= 1.0)
            v1[ok], v2[ok], q[ok] = c1[ok], c2[ok], q2[ok]
            done |= ok
        return v1, v2, q

    def _reflect(self, x, y):
        ytop = self.ny - 0.5
        for _ in range(REFLECTIONS):   # a pass without a hit changes nothing
            if self.periodic:
                x = np.where(x < -0.5, x + self.nx,
                             np.where(~(x < -0.5 + self.nx), x - self.nx, x))
                y = np.where(y < -0.5, y + self.ny,
                             np.where(~(y < -0.5 + self.ny), y - self.ny, y))
            else:
                lo, hi = y < -0.5, y > ytop
                y = np.where(lo, -1.0 - y, np.where(hi, 2.0 * ytop - y, y))
            for (cx, cy, rp, *_rest) in self.fib:
                dx, dy = x - cx, y - cy
                d2 = dx * dx + dy * dy
                inside = d2 < rp * rp
                if not inside.any():
                    continue
                at_c = inside & (d2 == 0.0)
                mv = inside & ~at_c
                d = np.sqrt(np.where(mv, d2, 1.0))
                qf = (2.0 * rp - d) / d
                x = np.where(mv, cx + qf * dx, np.where(at_c, cx + rp, x))
                y = np.where(mv, cy + qf * dy, y)
        return x, y

    def _rates(self, s, x, y):
        if self.homogeneous:
            return np.where(s == 0, self.k1, np.where(s == 1, self.k2, 0.0))
        k = np.zeros(x.shape[0])
        found = np.zeros(x.shape[0], bool)
        for (cx, cy, rp, kab, kbc, split, nxv, nyv) in self.fib:
            dx, dy = x - cx, y - cy
            d2 = dx * dx + dy * dy
            ro = rp + self.delta
            inside = (d2 >= rp * rp) & (d2 < ro * ro)
            if split:
                first = (dx * nxv + dy * nyv) >= 0.0
                ka = np.where(first, kab, 0.0)
                kb = np.where(first, 0.0, kbc)
            else:
                ka = np.full(x.shape[0], kab)
                kb = np.full(x.shape[0], kbc)
            kf = np.where(s == 0, ka, np.where(s == 1, kb, 0.0))
            take = inside & ~found & (kf > 0.0)
            k = np.where(take, kf, k)
            found |= take
        return k

    def _spawn(self, t, id0, m, x0, wx):
        if m <= 0:
            return
        ids = np.arange(m, dtype=np.uint64) + U64(id0)
        ps = particle_seed(self.seed, ids)
        x = x0 + wx * draw(ps, t, SPAWN_DRAW)
        y = -0.5 + float(self.ny) * draw(ps, t, SPAWN_DRAW + 1)
        keep = np.ones(m, bool)
        for (cx, cy, rp, *_rest) in self.fib:
            dx, dy = x - cx, y - cy
            keep &= ~((dx * dx + dy * dy) < rp * rp)
        self.p.append(x[keep], y[keep], np.zeros(int(keep.sum()), np.int32),
                      ids[keep])

    # -- public -------------------------------------------------------------
    def init(self):
        """A at the density over the whole box (none inside a fiber)."""
        self.p = Particles()
        self.t = 0
        self.out[:] = 0
        m = _round_half_up(self.density * self.nx * self.ny)
        self._spawn(-1, 0, m, -0.5, float(self.nx))
        self.next_id = m
        return self

    def step(self):
        p, t = self.p, self.t
        x, y, s = p.x.copy(), p.y.copy(), p.s.copy()
        ps = particle_seed(self.seed, p.id)
        if self.u is not None:
            ux, uy = self._velocity(x, y)
            x = x + self.dt * ux
            y = y + self.dt * uy
        if self.len > 0.0:
            v1, v2, q = self._direction(ps, t)
            r = np.sqrt(q)
            x = x + (self.len * v1) / r
            y = y + (self.len * v2) / r
        x, y = self._reflect(x, y)
        react = s < self.ns - 1
        if react.any():
            k = self._rates(s, x, y)
            hit = react & (k > 0.0) & (draw(ps, t, REACT_DRAW) < k * self.dt)
            s = np.where(hit, s + 1, s).astype(np.int32)
        keep = np.ones(x.shape[0], bool)
        if not self.periodic:
            out = ~(x < self.nx - 0.5)
            for sp in range(3):
                self.out[sp] += int((out & (s == sp)).sum())
            inl = (~out) & (x < -0.5)
            keep = ~out & ~(inl & (s == 0))
            x = np.where(inl & (s != 0), -1.0 - x, x)
            keep &= ~((s == 0) & (x < 0.5))
        p.x, p.y, p.s = x, y, s
        p.keep(keep)
        self._spawn(t, self.next_id, self.seed_count, -0.5, 1.0)
        self.next_id += self.seed_count
        self.t += 1

    def run(self, n):
        for _ in range(n):
            self.step()
        return self

    def efficiency(self):
        f = self.out.astype(np.float64)
        if self.ns == 2:
            return f[1] / (f[0] + f[1])
        return f[2] / f.sum()
