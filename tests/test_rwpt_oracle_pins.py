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


@pytest.mark.parametrize("cat", [1, 2, 3])
def test_reactive_shell_with_particles_at_rest(cat):
    """Step 4 of Sec. III.B with D = 0 and no flow, so particles stay where
    the fill put them: a particle reacts only inside the shell
    r <= d < r + delta around the fiber, r = R + 1/2 (reading R24), only
    for the species the catalyst acts on (A on an A->B fiber; nothing for
    A on a B->C fiber; A only on the k1 half of a side-by-side fiber, where
    (p - c).(cos t, sin t) >= 0), and there with probability k dt per step:
    the shell's A fraction after n steps is (1 - k dt)^n (binomial error).
    Particles outside it never change species."""
    nx = ny = 40
    R, delta, k, dt, th = 6.0, 0.8, 0.6, 0.5, 0.9
    fib = np.array([[20.3, 19.6, R, cat, th, -1]])
    sim = rwpt.RWPT(nx, ny, fib, k, k, None, 0.0, dt=dt, delta=delta,
                    density=200.0, periodic=True, nspecies=2,
                    seed=17).init()
    x0, y0, s0, id0 = sim.p.sorted()
    assert (s0 == 0).all()
    dx, dy = x0 - fib[0, 0], y0 - fib[0, 1]
    d = np.hypot(dx, dy)
    r = R + 0.5
    shell = (d >= r) & (d < r + delta)
    if cat == 2:
        active = np.zeros_like(shell)
    elif cat == 3:
        active = shell & (dx * math.cos(th) + dy * math.sin(th) >= 0.0)
    else:
        active = shell
    # the fill covers the shell at the density (Poisson count)
    area = math.pi * ((r + delta) ** 2 - r ** 2)
    assert abs(shell.sum() - 200.0 * area) < 5 * math.sqrt(200.0 * area)
    for n in (1, 3):
        while sim.t < n:
            sim.step()
        x, y, s, ids = sim.p.sorted()
        assert np.array_equal(ids, id0)
        assert np.array_equal(x, x0) and np.array_equal(y, y0)
        assert (s[~active] == 0).all()
        if active.any():
            m = int(active.sum())
            p = (1 - k * dt) ** n
            frac = (s[active] == 0).mean()
            assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / m)
            assert (s[active] <= 1).all()          # B does not react on
    if cat == 3:
        assert active.sum() > 0.3 * shell.sum()     # about half the shell
