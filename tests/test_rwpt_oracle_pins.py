"""Pins of the CPU random-walk particle oracle (Sec. III.B) against what the
method fixes (no GPU):
* every diffusion step has length sqrt(4 D dt) (to rounding) and the
  directions are isotropic, so the mean squared displacement after n steps
  is 4 D n dt (the statistical bound is stated per test);
* a uniform velocity field moves a particle exactly u dt per step (the
  bilinear weights sum to 1);
* the homogeneous reaction (every particle reacts with probability k dt per
  step) leaves a fraction (1 - k dt)^n of A, within binomial error; for
  small k that follows exp(-k t), the homogeneous-reaction check of the
  paper (with dt = 0.5, k = 1 halves A every step);
* no particle ends a step inside a fiber or beyond a wall;
* the generator is SplitMix64: its first outputs for seed 1234567 are the
  values printed by the published reference implementation's definition
  (recomputed here with Python integers)."""
import math

import numpy as np
import pytest

from oracle import rwpt


def _splitmix_python(seed, n):
    """SplitMix64 with Python integers, straight from its definition."""
    out, s = [], seed
    m = (1 << 64) - 1
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & m
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        out.append(z ^ (z >> 31))
    return out


def test_generator_is_splitmix64():
    ref = _splitmix_python(1234567, 5)
    got = [int(rwpt.mix64(np.uint64((1234567 + (i + 1) * 0x9E3779B97F4A7C15)
                                    % 2**64))) for i in range(5)]
    assert got == ref
    # draw k at step t: output 64 t + k + 1 of the particle's stream
    ps = rwpt.particle_seed(99, np.array([7], np.uint64))
    stream = _splitmix_python(int(ps[0]), 64 * 3 + 6)
    d = rwpt.draw(ps, 3, 5)[0]
    assert d == (stream[64 * 3 + 5] >> 11) * 2.0**-53


def test_diffusion_step_length_and_msd():
    n_part, steps, D, dt = 4000, 40, 0.3, 0.5
    sim = rwpt.RWPT(400, 400, np.zeros((0, 6)), 0.0, 0.0, None, D, dt=dt,
                    density=n_part / (400 * 400), periodic=True, nspecies=1,
                    seed=3).init()
    x0, y0, _, id0 = sim.p.sorted()
    sim.step()
    x1, y1, _, _ = sim.p.sorted()
    sx = (x1 - x0 + 200) % 400 - 200      # across a periodic edge
    sy = (y1 - y0 + 200) % 400 - 200
    step = np.hypot(sx, sy)
    assert np.allclose(step, math.sqrt(4 * D * dt), rtol=0, atol=1e-12)
    ang = np.arctan2(sy, sx)
    # isotropy: E cos 2t = E sin 2t = 0, sd 1/sqrt(2n)
    tol = 5 / math.sqrt(2 * len(ang))
    assert abs(np.cos(2 * ang).mean()) < tol and abs(np.sin(2 * ang).mean()) < tol
    sim.run(steps - 1)
    x2, y2, _, _ = sim.p.sorted()
    dx = (x2 - x0 + 200) % 400 - 200      # unwrap (moves are << 200)
    dy = (y2 - y0 + 200) % 400 - 200
    msd = (dx * dx + dy * dy).mean()
    want = 4 * D * steps * dt
    # |sum of n unit vectors|^2 has mean n and variance ~ n^2 (chi-square
    # with 2 degrees of freedom at large n): sd of the mean ~ want/sqrt(N)
    assert abs(msd - want) < 5 * want / math.sqrt(len(dx))


def test_uniform_flow_moves_exactly():
    nx, ny = 30, 20
    ux = np.full((ny, nx), 0.07)
    uy = np.full((ny, nx), -0.03)
    sim = rwpt.RWPT(nx, ny, np.zeros((0, 6)), 0.0, 0.0, (ux, uy), 0.0,
                    dt=0.5, density=2.0, periodic=True, nspecies=1).init()
    x0, y0, _, _ = sim.p.sorted()
    sim.step()
    x1, y1, _, _ = sim.p.sorted()
    dx = (x1 - x0 + nx / 2) % nx - nx / 2
    dy = (y1 - y0 + ny / 2) % ny - ny / 2
    assert np.allclose(dx, 0.035, rtol=0, atol=1e-14)
    assert np.allclose(dy, -0.015, rtol=0, atol=1e-14)


@pytest.mark.parametrize("k", [0.01, 1.0])
def test_homogeneous_reaction(k):
    """Every particle reacts with probability k dt per step (dt = 0.5): the
    share of A after n steps is (1 - k dt)^n (binomial error); for k = 0.01
    that is exp(-k t) to O(k^2 t)."""
    n_part, dt = 20000, 0.5
    sim = rwpt.RWPT(100, 100, np.zeros((0, 6)), k, 0.0, None, 0.1, dt=dt,
                    density=n_part / 1e4, periodic=True, homogeneous=True,
                    nspecies=2, seed=11).init()
    for n in (1, 2, 4, 8):
        while sim.t < n:
            sim.step()
        frac = (sim.p.s == 0).mean()
        p = (1 - k * dt) ** n
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / n_part) + 1e-12
    if k == 0.01:
        sim.run(392)                       # t = 400 steps = 200 time units
        p = (1 - k * dt) ** 400
        assert abs(p / math.exp(-k * 200) - 1) < 200 * k * k * dt
        frac = (sim.p.s == 0).mean()
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / n_part)


def test_particles_stay_outside_fibers_and_walls():
    nx, ny = 60, 24
    fib = np.array([[20.3, 11.2, 4.0, 1, 0, -1], [40.6, 9.7, 3.0, 2, 0, -1]])
    rng = np.random.default_rng(2)
    ux = 0.04 + 0.01 * rng.random((ny, nx))
    uy = 0.01 * (rng.random((ny, nx)) - 0.5)
    sim = rwpt.RWPT(nx, ny, fib, 0.1, 0.1, (ux, uy), 0.2, density=3.0,
                    nspecies=3, seed=5).init()
    for _ in range(60):
        sim.step()
        x, y = sim.p.x, sim.p.y
        assert (y >= -0.5).all() and (y <= ny - 0.5).all()
        assert (x >= -0.5).all() and (x < nx - 0.5).all()
        for cx, cy, r, *_ in fib:
            assert (np.hypot(x - cx, y - cy) >= r + 0.5 - 1e-12).all()
    assert sim.out.sum() > 0 and (sim.p.s > 0).any()
