"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics of the scheme (no GPU needed).

Each test names the passage it pins and the kind of pin: a closed form, an
exact moment recurrence, a conservation invariant, an independent brute-force
implementation on a tiny domain, or a number printed in the paper.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2109_04455_gb300 import inputs
from tests.conftest import read_golden

CX = oracle.CX
CY = oracle.CY
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]


# ---------------------------------------------------------------------------
# p8: parameter conventions against the paper's worked numbers
# ---------------------------------------------------------------------------
def test_da_k_and_tau_d_worked_numbers():
    """Sec. IV.A (Fig. singleAB caption): R = 5, Da = 150 <-> k = 1 and
    Da = 1.5 <-> k = 0.01; Appendix C: tau = 1 <-> D = 0.1666."""
    g = read_golden("paper_worked_numbers.txt")
    d = (g["gauss_tau"] - 0.5) / 3.0
    assert abs(d - g["gauss_D"]) < 1e-4
    assert inputs.tau_from_diffusivity(d) == pytest.approx(g["gauss_tau"],
                                                           abs=1e-15)
    for da, k in ((g["single_Da_a"], g["single_k_a"]),
                  (g["single_Da_b"], g["single_k_b"])):
        assert inputs.rate_from_da(da, d, g["single_R"]) == pytest.approx(
            k, rel=1e-12)
        assert inputs.da_from_rate(k, d, g["single_R"]) == pytest.approx(
            da, rel=1e-12)
    # Pe = u0 R / D round trip
    assert inputs.diffusivity_from_pe(0.05, 8.0, 10.0) == pytest.approx(0.04)


# ---------------------------------------------------------------------------
# raster: Gauss circle counts and side-by-side split
# ---------------------------------------------------------------------------
def test_raster_gauss_circle_counts():
    """Node solid iff (x-cx)^2+(y-cy)^2 <= R^2: an integer-centred disc of
    radius r holds exactly the Gauss-circle count of nodes (OEIS A000328)."""
    rows = read_golden("gauss_circle.txt")[1:]
    for r_s, n_s in rows:
        r = int(r_s)
        fib = [[15.0, 14.0, float(r), 1.0, 0.0, -1.0]]
        solid, kab, kbc = oracle.raster(31, 29, fib, 0.3, 0.7)
        assert int(solid.sum()) == int(n_s)
        assert np.all(kab[solid == 1] == 0.3) and np.all(kbc == 0.0)


def test_raster_janus_and_relaxed_weight():
    """Side-by-side fiber (Sec. II.C): A->B on the half (p-c).n >= 0, B->C on
    the other; relaxed weight w gives w*k1 and (1-w)*k2 on every node."""
    fib = [[15.0, 14.0, 8.0, 3.0, 0.0, -1.0]]     # split line x = 15
    solid, kab, kbc = oracle.raster(31, 29, fib, 0.3, 0.7)
    ys, xs = np.nonzero(solid)
    assert np.all(kab[ys, xs][xs >= 15] == 0.3)
    assert np.all(kbc[ys, xs][xs < 15] == 0.7)
    assert np.all((kab[ys, xs] > 0) ^ (kbc[ys, xs] > 0))
    # disc of 197 nodes, column x = 15 holds 17 of them, halves are 90 each
    assert int((kab > 0).sum()) == 90 + 17 and int((kbc > 0).sum()) == 90
    fib = [[15.0, 14.0, 8.0, 1.0, 0.0, 0.25]]
    solid, kab, kbc = oracle.raster(31, 29, fib, 0.4, 0.8)
    assert np.allclose(kab[solid == 1], 0.1) and np.allclose(
        kbc[solid == 1], 0.6)


# ---------------------------------------------------------------------------
# p1: homogeneous first-order reaction (Appendix C, Eq. source_lbm)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k1,k2", [(0.01, 0.03), (0.2, 0.05), (1.0, 0.5)])
def test_homogeneous_cascade_closed_form(k1, k2):
    """Periodic, u = 0, every population reacts: the discrete law is
    C_A(t) = (1-k1)^t, C_B(t) = k1/(k2-k1) [(1-k1)^t - (1-k2)^t],
    C_C = 1 - C_A - C_B; with k1 = 1 A vanishes after one step, as the
    homogeneous-reaction check of Appendix C states for k = 1."""
    nx, ny = 6, 5
    solid = np.zeros((ny, nx), np.uint8)
    z = np.zeros((ny, nx))
    prob = oracle.ADRProblem(solid, np.full((ny, nx), k1),
                             np.full((ny, nx), k2), z, z, [0.7] * 3,
                             [0, 0, 0], flags=oracle.PX | oracle.PY |
                             oracle.ALLPOP)
    g = prob.init()
    for t in range(1, 41):
        prob.steps(g, 1)
        c = prob.conc(g)
        a = (1 - k1) ** t
        b = k1 / (k2 - k1) * ((1 - k1) ** t - (1 - k2) ** t)
        assert np.allclose(c[0], a, rtol=1e-12, atol=1e-15)
        assert np.allclose(c[1], b, rtol=1e-12, atol=1e-16)
        assert np.allclose(c[2], 1 - a - b, rtol=1e-12, atol=1e-15)
    if k1 == 1.0:
        g = prob.init()
        prob.steps(g, 1)
        # zero up to the rounding of sum_i w_i = 1
        assert np.abs(prob.conc(g)[0]).max() < 1e-15


@pytest.mark.parametrize("k1,k2", [(0.05, 0.02), (0.3, 0.6)])
def test_nodewise_reactive_lattice_closed_form(k1, k2):
    """Node-wise variant (every population of a node with catalytic links
    reacts, with the mean rates of those links): periodic lattice with an
    isolated catalytic solid node at every (odd x, odd y), so every fluid
    node has catalytic links, all with the same rates.  With u = 0 the fluid
    state stays uniform (bounce-back returns w_i C like a uniform neighbour)
    and follows the homogeneous law C_A = (1-k1)^t,
    C_B = k1/(k2-k1) [(1-k1)^t - (1-k2)^t].  The link-wise source on the
    same lattice reacts less per step (fewer than nine links react)."""
    nx, ny = 8, 6
    solid = np.zeros((ny, nx), np.uint8)
    solid[1::2, 1::2] = 1
    kab = np.where(solid == 1, k1, 0.0)
    kbc = np.where(solid == 1, k2, 0.0)
    z = np.zeros((ny, nx))
    fluid = solid == 0
    prob = oracle.ADRProblem(solid, kab, kbc, z, z, [0.9] * 3, [0, 0, 0],
                             flags=oracle.PX | oracle.PY | oracle.NODEWISE)
    link = oracle.ADRProblem(solid, kab, kbc, z, z, [0.9] * 3, [0, 0, 0],
                             flags=oracle.PX | oracle.PY)
    g, gl = prob.init(), link.init()
    for t in range(1, 31):
        prob.steps(g, 1)
        link.steps(gl, 1)
        c = prob.conc(g)
        a = (1 - k1) ** t
        b = k1 / (k2 - k1) * ((1 - k1) ** t - (1 - k2) ** t)
        assert np.allclose(c[0][fluid], a, rtol=1e-12, atol=1e-15)
        assert np.allclose(c[1][fluid], b, rtol=1e-12, atol=1e-16)
        assert np.allclose(c[2][fluid], 1 - a - b, rtol=1e-12, atol=1e-15)
    assert link.conc(gl)[0][fluid].mean() > a * 1.01


def test_homogeneous_decay_vs_exponential_small_k():
    """Appendix C: for small k the lattice law follows exp(-k t); the gap is
    (1-k)^t / exp(-kt) = exp(t (ln(1-k) + k)) = 1 - t k^2/2 + ..."""
    k, t = 0.01, 100
    nx, ny = 4, 4
    solid = np.zeros((ny, nx), np.uint8)
    z = np.zeros((ny, nx))
    prob = oracle.ADRProblem(solid, np.full((ny, nx), k), z, z, z, [1.0, 1.0],
                             [0, 0], flags=oracle.PX | oracle.PY |
                             oracle.ALLPOP)
    g = prob.init()
    prob.steps(g, t)
    ca = prob.conc(g)[0, 0, 0]
    assert abs(ca / math.exp(-k * t) - 1) < t * k * k / 2 * 1.05


# ---------------------------------------------------------------------------
# p2/p3: Gaussian hill (Appendix C)
# ---------------------------------------------------------------------------
def _gauss_problem(n, sigma0, tau, u):
    solid = np.zeros((n, n), np.uint8)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    x0 = y0 = n / 2
    c = np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (2 * sigma0 ** 2))
    ux = np.full((n, n), u[0])
    uy = np.full((n, n), u[1])
    z = np.zeros((n, n))
    prob = oracle.ADRProblem(solid, z, z, ux, uy, [tau], [0.0],
                             flags=oracle.PX | oracle.PY)
    return prob, c, x, y


def _moments(c, x, y):
    m = c.sum()
    mx, my = (c * x).sum() / m, (c * y).sum() / m
    vx = (c * (x - mx) ** 2).sum() / m
    vy = (c * (y - my) ** 2).sum() / m
    return m, mx, my, vx, vy


@pytest.mark.parametrize("tau", [1.0, 0.8, 1.3])
def test_gaussian_moment_recurrence_no_flow(tau):
    """u = 0, equilibrium start: mass is exact, the centroid stays, and with
    w = 1/tau the per-axis variance obeys the exact lattice recurrence
    var(T) = var(0) + 2 D T - (2/3)(1-w)(1-(1-w)^T)/w^2, D = (tau-1/2)/3
    (Eq. Diffusion_LBM), derived from the BGK relaxation of the first and
    second moments."""
    prob, c0, x, y = _gauss_problem(128, 2.0, tau, (0.0, 0.0))
    g = prob.init(c0[None])
    m0, mx0, my0, vx0, vy0 = _moments(c0, x, y)
    T = 60
    prob.steps(g, T)
    c = prob.conc(g)[0]
    m, mx, my, vx, vy = _moments(c, x, y)
    w = 1.0 / tau
    d = (tau - 0.5) / 3.0
    expect = vx0 + 2 * d * T - (2 / 3) * (1 - w) * (1 - (1 - w) ** T) / w**2
    assert m == pytest.approx(m0, rel=1e-13)
    assert mx == pytest.approx(mx0, abs=1e-10)
    assert my == pytest.approx(my0, abs=1e-10)
    assert vx == pytest.approx(expect, rel=1e-11)
    assert vy == pytest.approx(expect, rel=1e-11)


def test_gaussian_moment_recurrence_with_flow():
    """tau = 1, uniform u = (0.1, 0.1) (Appendix C): the centroid moves by
    exactly u per step and each variance grows by exactly 1/3 per step."""
    prob, c0, x, y = _gauss_problem(128, 2.0, 1.0, (0.1, 0.1))
    g = prob.init(c0[None])
    m0, mx0, my0, vx0, vy0 = _moments(c0, x, y)
    T = 50
    prob.steps(g, T)
    m, mx, my, vx, vy = _moments(prob.conc(g)[0], x, y)
    assert m == pytest.approx(m0, rel=1e-13)
    assert mx == pytest.approx(mx0 + 0.1 * T, abs=1e-10)
    assert my == pytest.approx(my0 + 0.1 * T, abs=1e-10)
    assert vx == pytest.approx(vx0 + T / 3, rel=1e-11)
    assert vy == pytest.approx(vy0 + T / 3, rel=1e-11)


@pytest.mark.parametrize("u,t", [((0.0, 0.0), 100), ((0.0, 0.0), 400),
                                 ((0.1, 0.1), 50), ((0.1, 0.1), 100)])
def test_gaussian_hill_vs_analytic_profile(u, t):
    """Appendix C: 100x100, sigma0 = 1, tau = 1 (D = 1/6); the lattice profile
    follows the continuum solution
    C = s0^2/(s0^2+2Dt) exp(-(x-x0-ut)^2 / (2(s0^2+2Dt))) up to a small
    shape difference (max error below 2% of the peak)."""
    n = 100
    prob, c0, x, y = _gauss_problem(n, 1.0, 1.0, u)
    g = prob.init(c0[None])
    prob.steps(g, t)
    c = prob.conc(g)[0]
    d = 1.0 / 6.0
    s2 = 1.0 + 2 * d * t
    # periodic images of the analytic hill
    ana = np.zeros_like(c)
    for ix in (-1, 0, 1):
        for iy in (-1, 0, 1):
            dx = x - n / 2 - u[0] * t + ix * n
            dy = y - n / 2 - u[1] * t + iy * n
            ana += (1.0 / s2) * np.exp(-(dx**2 + dy**2) / (2 * s2))
    err = np.abs(c - ana).max() / ana.max()
    assert err < 2e-2


@pytest.mark.parametrize("u,t", [((0.0, 0.0), 50), ((0.0, 0.0), 100),
                                 ((0.0, 0.0), 400), ((0.1, 0.1), 50),
                                 ((0.1, 0.1), 100), ((0.1, 0.1), 400)])
def test_gaussian_hill_sigma4_vs_analytic_profile(u, t):
    """Appendix C at sigma0 = 4 (a hill the lattice resolves): with tau = 1
    (D = 1/6) the profile follows the continuum solution
    C = s0^2/(s0^2 + 2Dt) exp(-|x - x0 - ut|^2 / (2(s0^2 + 2Dt))) to 1e-3
    of the peak."""
    n = 160
    prob, c0, x, y = _gauss_problem(n, 4.0, 1.0, u)
    g = prob.init(c0[None])
    prob.steps(g, t)
    c = prob.conc(g)[0]
    s2 = 16.0 + 2 * (1.0 / 6.0) * t
    ana = np.zeros_like(c)
    for ix in (-1, 0, 1):
        for iy in (-1, 0, 1):
            dx = x - n / 2 - u[0] * t + ix * n
            dy = y - n / 2 - u[1] * t + iy * n
            ana += (16.0 / s2) * np.exp(-(dx**2 + dy**2) / (2 * s2))
    assert np.abs(c - ana).max() / ana.max() < 1e-3


# ---------------------------------------------------------------------------
# p4: flow lattice
# ---------------------------------------------------------------------------
def _shear_wave_amplitude(ny, tau, t, u_amp=1e-4):
    nx = 2
    solid = np.zeros((ny, nx), np.uint8)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    kk = 2 * np.pi / ny
    ux = u_amp * np.sin(kk * y)
    f = oracle.flow_init_fields(solid, np.ones((ny, nx)), ux,
                                np.zeros((ny, nx)))
    oracle.flow_steps(f, solid, tau, 0.0, t, flags=oracle.PX | oracle.PY)
    _, ux_t, _ = oracle.flow_moments(f, solid)
    amp = 2 * (ux_t[:, 0] * np.sin(kk * y[:, 0])).sum() / ny
    return amp / u_amp, kk


def test_shear_wave_decay_rate_converges_second_order():
    """Fully periodic shear wave u_x = U sin(k y): decays as exp(-nu k^2 t)
    with nu = (tau - 1/2)/3 in the continuum limit; the lattice error of the
    decay exponent shrinks by ~4x when the wavelength doubles."""
    tau = 0.8
    nu = (tau - 0.5) / 3.0
    errs = []
    for ny in (32, 64):
        kk = 2 * np.pi / ny
        t = int(round(0.5 / (nu * kk * kk)))   # decay to ~exp(-0.5)
        a, kk = _shear_wave_amplitude(ny, tau, t)
        rate = -math.log(a) / t
        errs.append(abs(rate / (nu * kk * kk) - 1))
    assert errs[0] < 2e-2
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_flow_mass_conserved_closed_box_with_fiber():
    """Periodic in x, walls in y, a fiber: halfway bounce-back and BGK keep
    the total mass exactly (to rounding)."""
    nx, ny = 40, 24
    solid, _, _ = oracle.raster(nx, ny, [[20.3, 11.7, 4.0, 0, 0, -1]], 0, 0)
    rho = np.ones((ny, nx))
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    ux = 0.03 * np.sin(np.pi * (y + 0.5) / ny) * (solid == 0)
    f = oracle.flow_init_fields(solid, rho, ux, np.zeros((ny, nx)))
    m0 = f.sum()
    oracle.flow_steps(f, solid, 0.8, 0.0, 500, flags=oracle.PX)
    assert f.sum() == pytest.approx(m0, rel=1e-13)


def test_empty_channel_poiseuille_profile():
    """Inlet-outlet channel without fibers (velocity bounce-back inlet with
    the parabola 4 u0 (y+1/2)(ny-1/2-y)/ny^2, pressure anti-bounce-back
    outlet, halfway bounce-back walls):
    * at steady state the mass flux sum_y rho u_x through every column equals
      the imposed inflow sum_y u_in(y) (to the residual);
    * the profile shape in the middle of the channel is the parabola, with a
      lattice error that falls by 4x when ny doubles (second order)."""
    tau, u0 = 0.8, 0.01
    errs = []
    for ny, steps in ((12, 8000), (24, 12000)):
        nx = 6 * ny
        solid = np.zeros((ny, nx), np.uint8)
        rho, ux, uy, res = oracle.flow_run(solid, tau, u0, steps)
        assert res < 1e-4
        yy = np.arange(ny)
        para = 4 * u0 * (yy + 0.5) * (ny - 0.5 - yy) / ny**2
        q = (rho * ux).sum(axis=0)
        assert np.abs(q / para.sum() - 1).max() < 1e-5
        prof = ux[:, nx // 2]
        errs.append(np.linalg.norm(prof / prof.sum() - para / para.sum())
                    / np.linalg.norm(para / para.sum()))
        assert np.abs(uy[:, nx // 4:3 * nx // 4]).max() < 1e-4 * u0
    assert errs[1] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


# ---------------------------------------------------------------------------
# p5/p6: invariants of the channel ADR lattice
# ---------------------------------------------------------------------------
def _small_channel(nx=64, ny=24, steps=300):
    fib = [[20.2, 11.3, 4.0, 1, 0, -1], [38.7, 12.4, 4.0, 2, 0, -1],
           [29.1, 4.9, 2.0, 3, 1.0, -1]]
    solid, kab, kbc = oracle.raster(nx, ny, fib, 0.05, 0.08)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, steps)
    return solid, kab, kbc, ux, uy


@pytest.mark.parametrize("variant", [0, oracle.NODEWISE])
def test_species_sum_invariant_cascade(variant):
    """Eq. (source_lbm): the sources of A, B and C on each link add to zero,
    so with equal tau and the same anti-bounce-back inlet for every species
    (test mode, C_w = 1, 0, 0) the field C_A+C_B+C_C equals, at every node
    and step, that of one non-reacting species.  The same holds for the
    node-wise variant (its sources add to zero on every population)."""
    solid, kab, kbc, ux, uy = _small_channel()
    tau = 0.62
    p3 = oracle.ADRProblem(solid, kab, kbc, ux, uy, [tau] * 3, [1, 0, 0],
                           flags=oracle.INLET_ABB_ALL | variant)
    p1 = oracle.ADRProblem(solid, kab * 0, kbc * 0, ux, uy, [tau], [1.0],
                           flags=oracle.INLET_ABB_ALL)
    g3, g1 = p3.init(), p1.init()
    for _ in range(4):
        p3.steps(g3, 50)
        p1.steps(g1, 50)
        s = p3.conc(g3).sum(axis=0)
        one = p1.conc(g1)[0]
        assert np.allclose(s, one, rtol=1e-13, atol=1e-14)
        assert p3.flux(g3).sum() == pytest.approx(p1.flux(g1)[0], rel=1e-12)
    # and the reaction really happened
    c = p3.conc(g3)
    assert c[1].max() > 1e-3 and c[2].max() > 1e-4


# ---------------------------------------------------------------------------
# p6: the outflux of Sec. III.A.3 and steady flux conservation.  None of these
# pins calls the oracle's flux routine to make its expected value: they use
# the first moments of the BGK collision, the boundary rules of Eq. (BC)
# inverted on the pre-collision steady state, and the streaming map.
# ---------------------------------------------------------------------------
PLUS, MINUS = [1, 5, 8], [3, 6, 7]   # directions with c_ix = +1 and -1


def _source_x_moment(ns, kab, kbc, solid, c, xp, y):
    """sum_i c_ix Q_{s,i} at fluid node (xp, y) for the link-wise source of
    Eq. (source_lbm): links into a solid node t carry Q_A = -k_AB(t) w C_A,
    Q_B = +k_AB w C_A - k_BC w C_B, Q_C = +k_BC w C_B (walls carry none)."""
    ny, nx = solid.shape
    q = np.zeros(ns)
    for i in range(1, 9):
        tx, ty = xp + CX[i], y + CY[i]
        if not (0 <= ty < ny and 0 <= tx < nx) or not solid[ty, tx]:
            continue
        ra = kab[ty, tx] * W[i] * c[0]
        rb = kbc[ty, tx] * W[i] * c[1] if ns >= 3 else 0.0
        q[0] -= CX[i] * ra
        if ns >= 2:
            q[1] += CX[i] * (ra - rb)
        if ns >= 3:
            q[2] += CX[i] * rb
    return q


@pytest.mark.parametrize("ns", [2, 3])
def test_outflux_is_first_moment_of_post_collision_state(ns):
    """Sec. III.A.3: N_s = (1/ny) sum_y sum_i c_ix g*_{s,i}(x_p, y) over the
    post-collision populations.  The x-moment of the BGK update is
    (1 - w) j_s + w C_s u_x (the equilibrium's first moment is C u), plus
    the x-moment of the source on catalytic links, so on any state
    N_s = (1/ny) sum_y [(1 - w_s) j_s + w_s C_s u_x + sum_i c_ix Q_{s,i}].
    Random non-equilibrium states, planes cut by catalytic fibers of both
    kinds.  A pre-collision reading, a plane one node off, the opposite
    sign or a dropped source each miss by far more than the tolerance."""
    nx, ny = 26, 11
    fib = [[9.3, 4.6, 2.2, 1, 0, -1], [15.8, 6.1, 2.4, 2, 0, -1],
           [12.4, 9.7, 1.5, 3, 0.4, -1]]
    solid, kab, kbc = oracle.raster(nx, ny, fib, 0.3, 0.45)
    rng = np.random.default_rng(11 + ns)
    ux = (0.03 + 0.04 * rng.random((ny, nx))) * (solid == 0)
    uy = 0.03 * (rng.random((ny, nx)) - 0.5) * (solid == 0)
    tau = [0.9, 0.66, 1.4][:ns]
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, tau, [1, 0, 0][:ns])
    g = rng.random((ns, ny, nx, 9)) * (solid == 0)[None, :, :, None]
    checked_source = 0
    for xp in (7, 11, 12, 14, nx - 3):
        want = np.zeros(ns)
        pre = np.zeros(ns)
        nosrc = np.zeros(ns)
        for y in range(ny):
            if solid[y, xp]:
                continue
            gi = g[:, y, xp, :]
            c = gi.sum(axis=1)
            j = (gi * CX).sum(axis=1)
            om = 1.0 / np.asarray(tau)
            q = _source_x_moment(ns, kab, kbc, solid, c, xp, y)
            want += (1 - om) * j + om * c * ux[y, xp] + q
            nosrc += (1 - om) * j + om * c * ux[y, xp]
            pre += j
        want /= ny
        got = prob.flux(g, xp)[:ns]
        scale = np.abs(want).max()
        assert np.allclose(got, want, rtol=0, atol=1e-14 * max(scale, 1))
        # the plausible misreadings are far away
        assert np.abs(pre / ny - got).max() > 1e-3 * scale
        assert np.abs(-want - got).max() > 1e-3 * scale
        other = prob.flux(g, xp + 1)[:ns]
        assert np.abs(other - got).max() > 1e-3 * scale
        if np.abs(nosrc / ny - want).max() > 1e-3 * scale:
            checked_source += 1
    assert checked_source >= 2


def test_outflux_of_equilibrium_state_in_poiseuille_flow():
    """At an equilibrium state g = g^eq(C, u) with no catalyst, collision
    changes nothing and the first moment of g^eq is C u_x, so
    N_s = (1/ny) sum_y C_s(y) u_x(x_p, y) exactly.  With C = 1 on the steady
    empty channel this is the plane-mean of u_x: the parabola's mean
    (2/3) u0 (1 + 1/(2 ny^2)) divided by the density on the plane."""
    nx, ny, u0 = 48, 14, 0.05
    solid = np.zeros((ny, nx), np.uint8)
    rho, ux, uy, res = oracle.flow_run(solid, 0.8, u0, 6000)
    assert res < 1e-8
    z = np.zeros((ny, nx))
    prob = oracle.ADRProblem(solid, z, z, ux, uy, [0.7, 0.8, 1.1], [1, 0, 0])
    yy = np.arange(ny, dtype=float)
    c0 = np.stack([np.ones((ny, nx)),
                   np.broadcast_to((0.2 + 0.05 * yy)[:, None], (ny, nx)),
                   np.broadcast_to(np.cos(0.3 * yy)[:, None] ** 2, (ny, nx))])
    g = prob.init(c0)
    xp = nx - 3
    got = prob.flux(g, xp)
    want = (c0[:, :, xp] * ux[None, :, xp]).sum(axis=1) / ny
    assert np.allclose(got, want, rtol=1e-13, atol=0)
    # the flow carries the parabola's mass flux, rho u_x, through every
    # column; rho varies along x with the pressure drop but barely across
    # the plane, so the plane-mean of u_x is the parabola's mean over rho
    mean_para = (2.0 / 3.0) * u0 * (1 + 1 / (2 * ny * ny))
    rp = rho[:, xp]
    assert rp.max() - rp.min() < 2e-3
    assert got[0] == pytest.approx(mean_para / rp.mean(), rel=1e-3)


def _face_fluxes(g, solid, cin):
    """Net flux of the species sum through every face x = -1/2 .. nx - 1/2
    of the pre-collision steady state g (the step maps it to itself), per
    Eq. (BC): the inlet face from the anti-bounce-back of species A
    (g_i(0) = -g*_opp + 2 w_i c_in, so the face carries
    sum_y [2 sum_{c_ix>0} g_i(0, y) - c_in/3]; B and C bounce back and carry
    nothing); the outlet face from g_opp(nx-1) = -g*_i + 2 w_i C_b, i.e.
    sum_y [C_b/3 - 2 sum_{c_ix<0} g_i(nx-1, y)]; an interior face from the
    populations that streamed across it (bounced ones stay)."""
    ns, ny, nx, _ = g.shape
    fl = solid == 0
    out = np.zeros(nx + 1)
    for s in range(ns):
        if cin[s] != 0 or s == 0:
            out[0] += (2 * g[s][:, 0, PLUS].sum(axis=1) - cin[s] / 3)[fl[:, 0]].sum()
        for x in range(nx - 1):
            f = 0.0
            for y in range(ny):
                for i in PLUS:      # arrived at (x+1, y) from (x, y - c_iy)
                    sy = y - CY[i]
                    if fl[y, x + 1] and 0 <= sy < ny and fl[sy, x]:
                        f += g[s, y, x + 1, i]
                for i in MINUS:     # arrived at (x, y) from (x+1, y - c_iy)
                    sy = y - CY[i]
                    if fl[y, x] and 0 <= sy < ny and fl[sy, x + 1]:
                        f -= g[s, y, x, i]
            out[x + 1] += f
        cb = g[s][:, nx - 1, :].sum(axis=1)
        out[nx] += (cb / 3 - 2 * g[s][:, nx - 1, MINUS].sum(axis=1))[
            fl[:, nx - 1]].sum()
    return out


def _landed_flux(g, solid, xp):
    """ny N_s rebuilt from the streaming map: at a steady state each
    post-collision population g*_i(x_p, y) is found in the next pre-collision
    state at its neighbour (x_p + c_i) when that is a fluid node, else bounced
    back in place as g_opp(x_p, y)."""
    ns, ny, nx, _ = g.shape
    fl = solid == 0
    out = np.zeros(ns)
    for y in range(ny):
        if not fl[y, xp]:
            continue
        for i in PLUS + MINUS:
            tx, ty = xp + CX[i], y + CY[i]
            if 0 <= ty < ny and fl[ty, tx]:
                out += CX[i] * g[:, ty, tx, i]
            else:
                out += CX[i] * g[:, y, xp, OPP[i]]
    return out


@pytest.mark.parametrize("k", [1.0, 0.0])
def test_steady_flux_conservation_and_outflux(k):
    """p6 (Sec. III.A.3; the sources of Eq. source_lbm add to zero, collision
    and bounce-back keep mass): at the steady state of a cascade channel
    (per-step residual < 1e-13) the A injected through the inlet leaves as
    A + B + C, and the same net flux crosses every face.  The outflux N_s on
    a plane is the post-collision first moment, which the streaming map
    returns exactly.  The paper's node-centred N at x_p = nx - 3 differs
    from the conserved face flux by a lattice-spacing effect near the outlet
    (0.6-0.8% on this 60 x 16 lattice); it must stay within 1%.  With k = 0
    no B or C exists anywhere."""
    nx, ny = 60, 16
    fib = [[20.2, 8.3, 3.0, 1, 0, -1], [35.5, 7.1, 3.0, 2, 0, -1],
           [27.6, 1.2, 2.0, 3, 0.5, -1]]
    solid, kab, kbc = oracle.raster(nx, ny, fib, 0.05, 0.08)
    _, ux, uy, fres = oracle.flow_run(solid, 0.8, 0.05, 6000)
    assert fres < 1e-8
    cin = [1.0, 0.0, 0.0]
    prob = oracle.ADRProblem(solid, kab * k, kbc * k, ux, uy,
                             [0.62, 0.7, 0.8], cin)
    out = prob.solve(1e-13, 500, 200000)
    assert out["converged"]
    g = out["g"]
    faces = _face_fluxes(g, solid, cin)
    f_in = faces[0]
    assert f_in > 0.3
    assert np.abs(faces - f_in).max() < 1e-9 * f_in
    for xp in (nx - 3, 21, 28, 36, 45):
        n = prob.flux(g, xp)
        assert np.allclose(n * ny, _landed_flux(g, solid, xp), rtol=0,
                           atol=1e-11 * f_in)
    n = out["flux"]
    assert abs(n.sum() * ny - f_in) < 1e-2 * f_in
    if k == 0.0:
        assert n[1] == 0.0 and n[2] == 0.0
    else:
        assert n[1] > 1e-3 and n[2] > 1e-3


def test_no_reaction_no_product():
    """k = 0: B and C start at zero and nothing produces them, so their
    concentrations and outfluxes stay exactly zero."""
    solid, kab, kbc, ux, uy = _small_channel()
    p = oracle.ADRProblem(solid, kab * 0, kbc * 0, ux, uy, [0.62] * 3,
                          [1, 0, 0])
    out = p.run(200)
    assert np.all(out["conc"][1:] == 0.0)
    assert out["flux"][1] == 0.0 and out["flux"][2] == 0.0
    assert out["flux"][0] > 0 and out["eps"] == 0.0


def test_efficiency_definition():
    """Eq. (A-B)."""
    assert oracle.efficiency([3.0, 1.0, 0.0], 2) == pytest.approx(0.25)
    assert oracle.efficiency([1.0, 1.0, 2.0], 3) == pytest.approx(0.5)


def test_pe_trend_single_fiber():
    """Sec. IV.A: the efficiency falls as Pe rises (shorter contact time),
    checked on a small single-fiber channel near steady state."""
    nx, ny, r = 96, 48, 5.0
    solid, kab, kbc = oracle.raster(nx, ny, [[30.0, 24.0, r, 1, 0, -1]], 1, 0)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, 3000)
    eps = []
    for pe in (2.0, 10.0, 50.0):
        d = inputs.diffusivity_from_pe(0.05, r, pe)
        tau = inputs.tau_from_diffusivity(d)
        k = inputs.rate_from_da(1.0, d, r)
        p = oracle.ADRProblem(solid, kab * k, kbc, ux, uy, [tau, tau],
                              [1, 0])
        eps.append(p.run(3000)["eps"])
    assert eps[0] > eps[1] > eps[2] > 0


def test_da_trend_single_fiber():
    """Sec. IV.A: at fixed Pe the efficiency rises with Da (a faster surface
    reaction), in proportion to Da while the reaction limits the rate, and
    saturating once diffusion to the surface does (the shape of the paper's
    efficiency-against-Da figure)."""
    nx, ny, r, pe = 96, 48, 5.0, 5.0
    solid, kab, kbc = oracle.raster(nx, ny, [[30.0, 24.0, r, 1, 0, -1]], 1, 0)
    _, ux, uy, _ = oracle.flow_run(solid, 0.8, 0.05, 3000)
    d = inputs.diffusivity_from_pe(0.05, r, pe)
    tau = inputs.tau_from_diffusivity(d)
    eps = []
    das = (0.01, 0.1, 30.0, 300.0)
    for da in das:
        k = inputs.rate_from_da(da, d, r)
        assert k < 1.0
        p = oracle.ADRProblem(solid, kab * k, kbc, ux, uy, [tau, tau],
                              [1, 0])
        eps.append(p.run(3000)["eps"])
    assert 0 < eps[0] < eps[1] < eps[2] < eps[3]
    # reaction-limited: ten times the rate gives nearly ten times eps
    assert 9.0 < eps[1] / eps[0] < 10.0
    # diffusion-limited: ten times the rate gives much less than that
    assert eps[3] / eps[2] < 2.5


# ---------------------------------------------------------------------------
# p7: brute force -- an independent pull-form implementation on tiny domains
# ---------------------------------------------------------------------------
def _collide(gb, solid, kab, kbc, ux, uy, tau, ns):
    """BGK collision plus the link-wise source at every fluid node, batched
    over the first axis: gb[b, s, y, x, i] (pre-collision) -> post-collision
    g* (zero on solid nodes)."""
    ny, nx = solid.shape
    gs = np.zeros_like(gb)
    # collision + source at every fluid node
    for y in range(ny):
        for x in range(nx):
            if solid[y, x]:
                continue
            c = gb[:, :, y, x, :].sum(axis=2)            # [b, s]
            cu = CX * ux[y, x] + CY * uy[y, x]
            uu = ux[y, x] ** 2 + uy[y, x] ** 2
            e = W * (1 + 3 * cu + 4.5 * cu**2 - 1.5 * uu)  # [i]
            for s in range(ns):
                gi = gb[:, s, y, x, :]
                gs[:, s, y, x, :] = gi + (c[:, s:s + 1] * e - gi) / tau[s]
            for i in range(1, 9):
                tx, ty = x + CX[i], y + CY[i]
                if not (0 <= tx < nx and 0 <= ty < ny) or not solid[ty, tx]:
                    continue
                ra = kab[ty, tx] * W[i] * c[:, 0]
                rb = kbc[ty, tx] * W[i] * c[:, 1] if ns >= 3 else 0.0
                gs[:, 0, y, x, i] -= ra
                if ns >= 2:
                    gs[:, 1, y, x, i] += ra - rb
                if ns >= 3:
                    gs[:, 2, y, x, i] += rb
    return gs


def _pull_step(gb, solid, kab, kbc, ux, uy, tau, cin, ns):
    """Naive pull-form ADR step written from the rules, batched over the
    first axis: gb[b, s, y, x, i] (pre-collision) -> next pre-collision."""
    ny, nx = solid.shape
    gs = _collide(gb, solid, kab, kbc, ux, uy, tau, ns)
    out = np.zeros_like(gb)
    # pull streaming with boundary rules
    for y in range(ny):
        for x in range(nx):
            if solid[y, x]:
                continue
            for s in range(ns):
                cb = gs[:, s, y, x, :].sum(axis=1)
                for i in range(9):
                    sx, sy = x - CX[i], y - CY[i]
                    o = OPP[i]
                    if sx < 0:          # came in through the inlet
                        if s == 0:
                            v = -gs[:, s, y, x, o] + 2 * W[i] * cin[s]
                        else:
                            v = gs[:, s, y, x, o]
                    elif sx >= nx:      # came in through the outlet
                        v = -gs[:, s, y, x, o] + 2 * W[i] * cb
                    elif sy < 0 or sy >= ny or solid[sy, sx]:
                        v = gs[:, s, y, x, o]
                    else:
                        v = gs[:, s, sy, sx, i]
                    out[:, s, y, x, i] = v
    return out


def _tiny_case(ns):
    nx, ny = 9, 6
    fib = [[3.2, 2.6, 1.2, 1, 0, -1], [6.1, 3.4, 1.0, 2, 0, -1]]
    solid, kab, kbc = oracle.raster(nx, ny, fib, 0.15, 0.25)
    rng = np.random.default_rng(7)
    ux = 0.04 + 0.02 * rng.random((ny, nx))
    uy = 0.02 * (rng.random((ny, nx)) - 0.5)
    ux[solid == 1] = 0
    uy[solid == 1] = 0
    tau = [0.9, 0.7, 0.8][:ns]
    cin = [1.0, 0.0, 0.0][:ns]
    return solid, kab, kbc, ux, uy, tau, cin


@pytest.mark.parametrize("ns", [2, 3])
def test_one_step_matches_independent_pull_implementation(ns):
    """Every link type (inlet, outlet, wall, corner, catalytic fiber of both
    kinds, plain fluid) on a 9x6 lattice: one oracle step (push form) equals
    the naive pull-form step on random states."""
    solid, kab, kbc, ux, uy, tau, cin = _tiny_case(ns)
    assert solid.sum() >= 4
    ny, nx = solid.shape
    rng = np.random.default_rng(1)
    g = rng.random((ns, ny, nx, 9)) * (solid == 0)[None, :, :, None]
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, tau, cin)
    want = _pull_step(g[None].copy(), solid, kab, kbc, ux, uy, tau, cin,
                      ns)[0]
    got = prob.steps(g.copy(), 1)
    assert np.allclose(got, want, rtol=0, atol=1e-14)


def test_steady_state_matches_dense_linear_solve():
    """The ADR step is affine in g (frozen u): g' = M g + b.  The steady state
    solves (I - M) g = b exactly; the oracle's long run must converge to it,
    and the steady efficiency follows from it."""
    ns = 3
    solid, kab, kbc, ux, uy, tau, cin = _tiny_case(ns)
    ny, nx = solid.shape
    fluid = (solid == 0)
    idx = [(s, y, x, i) for s in range(ns) for y in range(ny)
           for x in range(nx) if fluid[y, x] for i in range(9)]
    n = len(idx)
    basis = np.zeros((n + 1, ns, ny, nx, 9))
    for j, (s, y, x, i) in enumerate(idx):
        basis[j + 1, s, y, x, i] = 1.0
    img = _pull_step(basis, solid, kab, kbc, ux, uy, tau, cin, ns)
    flat = lambda a: np.array([a[s, y, x, i] for (s, y, x, i) in idx])
    b = flat(img[0])
    m = np.stack([flat(img[j + 1]) - b for j in range(n)], axis=1)
    gss = np.linalg.solve(np.eye(n) - m, b)
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, tau, cin)
    out = prob.run(6000)
    got = flat(out["g"])
    assert np.abs(got - gss).max() < 1e-11
    gfull = np.zeros((ns, ny, nx, 9))
    for v, (s, y, x, i) in zip(gss, idx):
        gfull[s, y, x, i] = v
    eps_exact = oracle.efficiency(prob.flux(gfull), ns)
    assert out["eps"] == pytest.approx(eps_exact, abs=1e-11)
    assert 0 < eps_exact < 1


# ---------------------------------------------------------------------------
# discrete adjoint of the oracle: pinned by central finite differences of
# the oracle's own steady state (itself pinned to the dense solve above)
# ---------------------------------------------------------------------------
def _steady_eps(prob, steps):
    return prob.run(steps)["eps"]


@pytest.mark.parametrize("ns", [2, 3])
def test_adjoint_rate_gradient_matches_finite_differences(ns):
    """d eps / d k at every solid node from the adjoint equals the central
    difference of the steady efficiency (h = 1e-5 relative)."""
    solid, kab, kbc, ux, uy, tau, cin = _tiny_case(ns)
    steps = 6000
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, tau, cin)
    fwd = prob.run(steps)
    adj = oracle.adjoint(prob, fwd["g"], steps)
    assert adj["eps"] == pytest.approx(fwd["eps"], abs=1e-15)
    ys, xs = np.nonzero(solid)
    checked = 0
    for y, x in zip(ys, xs):
        for field, grad in ((kab, adj["dkab"]), (kbc, adj["dkbc"])):
            if ns < 3 and field is kbc:
                continue
            base = field[y, x] if field[y, x] > 0 else 0.1
            h = 1e-5 * base
            vals = []
            for sgn in (1, -1):
                f2 = field.copy()
                f2[y, x] = field[y, x] + sgn * h
                ka = f2 if field is kab else kab
                kb = f2 if field is kbc else kbc
                p2 = oracle.ADRProblem(solid, ka, kb, ux, uy, tau, cin)
                vals.append(_steady_eps(p2, steps))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert grad[y, x] == pytest.approx(fd, rel=1e-5, abs=1e-12)
            checked += abs(fd) > 1e-8
    assert checked >= 3


def test_adjoint_fiber_weight_gradient_matches_finite_differences():
    """Relaxed catalyst weights (k_AB = w k1, k_BC = (1-w) k2): d eps/d w_f
    = sum over the fiber's nodes of k1 d eps/dk_AB - k2 d eps/dk_BC."""
    nx, ny = 12, 7
    k1, k2 = 0.2, 0.3
    fib = np.array([[3.6, 3.1, 1.3, 1, 0, 0.7], [8.2, 3.8, 1.4, 1, 0, 0.25]])
    rng = np.random.default_rng(3)
    solid, kab, kbc = oracle.raster(nx, ny, fib, k1, k2)
    ux = (0.05 + 0.01 * rng.random((ny, nx))) * (solid == 0)
    uy = 0.01 * (rng.random((ny, nx)) - 0.5) * (solid == 0)
    tau = [0.8, 0.75, 0.9]
    steps = 6000
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, tau, [1, 0, 0])
    fwd = prob.run(steps)
    adj = oracle.adjoint(prob, fwd["g"], steps)
    ids = oracle.fiber_ids(nx, ny, fib)
    dw = oracle.fiber_weight_gradient(ids, adj["dkab"], adj["dkbc"], k1, k2, 2)
    h = 1e-5
    for f in range(2):
        vals = []
        for sgn in (1, -1):
            fb = fib.copy()
            fb[f, 5] += sgn * h
            s2, a2, b2 = oracle.raster(nx, ny, fb, k1, k2)
            p2 = oracle.ADRProblem(s2, a2, b2, ux, uy, tau, [1, 0, 0])
            vals.append(p2.run(steps)["eps"])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd) > 1e-6
        assert dw[f] == pytest.approx(fd, rel=1e-5)


@pytest.mark.parametrize("ns", [2, 3])
def test_adjoint_matches_dense_implicit_derivative(ns):
    """p7 for the adjoint: d eps / d k at every solid node by dense linear
    algebra, without the adjoint and without a difference step.  With the
    flow frozen, one step is g' = M(k) g + b (the independent pull-form step
    above); the source is linear in each rate, so M(k + e_n) g - M(k) g is
    the exact k_n-derivative of the map at g.  The steady state solves
    (I - M) g = b, so dg/dk_n = (I - M)^-1 (M(k + e_n) - M(k)) g.  The
    outflux is the first moment of the post-collision state on x_p = nx - 3
    (Sec. III.A.3), and eps of Eq. (A-B) is differentiated by a complex
    step, exact for a rational function.  The oracle's adjoint, iterated to
    convergence at that steady state, must give the same gradient."""
    import scipy.linalg as sla

    solid, kab, kbc, ux, uy, tau, cin = _tiny_case(ns)
    ny, nx = solid.shape
    xp = nx - 3
    fluid = solid == 0
    nfl = int(fluid.sum())
    n = ns * nfl * 9

    def flat(a):
        return a[:, fluid, :].reshape(-1)

    def full(v):
        g = np.zeros((ns, ny, nx, 9), dtype=v.dtype)
        g[:, fluid, :] = v.reshape(ns, nfl, 9)
        return g

    def step(g, ka, kb):
        return flat(_pull_step(g[None], solid, ka, kb, ux, uy, tau, cin,
                               ns)[0])

    def outflux(g, ka, kb):
        gs = _collide(g[None], solid, ka, kb, ux, uy, tau, ns)[0]
        col = gs[:, fluid[:, xp], xp, :]            # [s, fluid rows, i]
        return (col * CX).sum(axis=(1, 2)) / ny

    def eps(nf):
        return nf[ns - 1] / nf[:ns].sum()

    basis = np.zeros((n + 1, ns, ny, nx, 9))
    basis[1:, :, fluid, :] = np.eye(n).reshape(n, ns, nfl, 9)
    img = _pull_step(basis, solid, kab, kbc, ux, uy, tau, cin, ns)
    b = flat(img[0])
    m = np.stack([flat(img[j + 1]) - b for j in range(n)], axis=1)
    lu = sla.lu_factor(np.eye(n) - m)
    g = full(sla.lu_solve(lu, b))
    nf = outflux(g, kab, kbc)
    assert np.abs(step(g, kab, kbc) - flat(g)).max() < 1e-13   # steady

    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, tau, cin)
    adj = oracle.adjoint(prob, g, 8000)
    assert adj["eps"] == pytest.approx(eps(nf), rel=1e-12)

    fields = [(kab, "dkab")] + ([(kbc, "dkbc")] if ns == 3 else [])
    nonzero = 0
    for y, x in zip(*np.nonzero(solid)):
        for field, key in fields:
            f2 = field.copy()
            f2[y, x] += 1.0
            ka = f2 if key == "dkab" else kab
            kb = f2 if key == "dkbc" else kbc
            dg = full(sla.lu_solve(lu, step(g, ka, kb) - step(g, kab, kbc)))
            dn = outflux(dg, kab, kbc) + (outflux(g, ka, kb) - nf)
            h = 1e-30
            want = eps(nf + 1j * h * dn).imag / h
            got = adj[key][y, x]
            assert got == pytest.approx(want, rel=1e-11, abs=1e-15), (y, x, key)
            nonzero += abs(want) > 1e-6
        if ns == 2:
            assert adj["dkbc"][y, x] == 0.0
    assert nonzero >= 4


# ---------------------------------------------------------------------------
# Eq. (BC): the inlet's anti-bounce-back imposes its concentration
# ---------------------------------------------------------------------------
def test_inlet_anti_bounce_back_fixes_the_concentration_without_flow():
    """Sec. III.A.3, Eq. (BC): with u = 0 and no reaction, the anti-bounce-
    back inlet (incoming g_i = -g*_opp + 2 w_i C_w) is a Dirichlet condition,
    the outlet's (C_w = C of the boundary node) a zero-gradient one, and the
    walls and the inert fiber bounce back: from C = 0 everywhere the lattice
    must fill up to C = C_w at every fluid node.  A stays the only species
    the default inlet feeds; with every species on anti-bounce-back (test
    mode) B and C fill up to their own inlet values."""
    nx, ny = 14, 7
    solid, kab, kbc = oracle.raster(nx, ny, [[7.2, 3.3, 1.6, 0, 0, -1]],
                                    0.0, 0.0)
    assert solid.sum() > 0
    z = np.zeros((ny, nx))
    fl = solid == 0
    for flags, cin, want in ((0, [1.0, 0.4, 0.9], [1.0, 0.0, 0.0]),
                             (oracle.INLET_ABB_ALL, [1.0, 0.3, 0.7],
                              [1.0, 0.3, 0.7])):
        prob = oracle.ADRProblem(solid, kab, kbc, z, z, [1.0, 0.8, 1.3], cin,
                                 flags=flags)
        g = prob.init(np.zeros((3, ny, nx)))
        prob.steps(g, 40000)
        c = prob.conc(g)
        for s in range(3):
            assert np.abs(c[s][fl] - want[s]).max() < 1e-10, (flags, s)


# ---------------------------------------------------------------------------
# p7 for the flow lattice: an independent pull-form flow step on a tiny domain
# ---------------------------------------------------------------------------
def _flow_pull_step(f, solid, tau, u0):
    """One D2Q9 BGK flow step written from the rules (reading R1): BGK at
    every fluid node; pull streaming; halfway bounce-back from walls and
    solid nodes; at the inlet velocity bounce-back, f_i = f*_opp + 6 w_i
    rho_w c_i.u_w with rho_w = 1 and u_w = (u_in(y), 0) of the node's row;
    at the outlet pressure anti-bounce-back, f_i = -f*_opp + 2 w_i rho_w
    (1 + 4.5 (c_i.u_w)^2 - 1.5 u_w^2) with rho_w = 1 and u_w the node's own
    velocity at time t; the x-edge rule wins on corner links (R7)."""
    ny, nx = solid.shape
    fs = np.zeros_like(f)
    ux = np.zeros((ny, nx))
    uy = np.zeros((ny, nx))
    for y in range(ny):
        for x in range(nx):
            if solid[y, x]:
                continue
            fi = f[y, x]
            rho = fi.sum()
            ux[y, x] = (fi * CX).sum() / rho
            uy[y, x] = (fi * CY).sum() / rho
            cu = CX * ux[y, x] + CY * uy[y, x]
            uu = ux[y, x] ** 2 + uy[y, x] ** 2
            feq = W * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu)
            fs[y, x] = fi - (fi - feq) / tau
    out = np.zeros_like(f)
    for y in range(ny):
        for x in range(nx):
            if solid[y, x]:
                continue
            for i in range(9):
                sx, sy = x - CX[i], y - CY[i]
                o = OPP[i]
                if sx < 0:
                    uin = 4 * u0 * (y + 0.5) * (ny - 0.5 - y) / ny ** 2
                    v = fs[y, x, o] + 6 * W[i] * CX[i] * uin
                elif sx >= nx:
                    cu = CX[i] * ux[y, x] + CY[i] * uy[y, x]
                    uu = ux[y, x] ** 2 + uy[y, x] ** 2
                    v = -fs[y, x, o] + 2 * W[i] * (1 + 4.5 * cu ** 2
                                                   - 1.5 * uu)
                elif sy < 0 or sy >= ny or solid[sy, sx]:
                    v = fs[y, x, o]
                else:
                    v = fs[sy, sx, i]
                out[y, x, i] = v
    return out


@pytest.mark.parametrize("tau", [0.8, 1.3])
def test_flow_step_matches_independent_pull_implementation(tau):
    """Every flow link type (inlet and outlet with their corners, walls, a
    fiber, a fiber touching a wall, plain fluid) on an 11x7 lattice: one
    oracle flow step equals the naive pull-form step on random states near
    equilibrium (1e-14)."""
    nx, ny, u0 = 11, 7, 0.05
    solid, _, _ = oracle.raster(nx, ny, [[4.3, 3.2, 1.4, 0, 0, -1],
                                         [8.0, 1.0, 1.0, 0, 0, -1]], 0, 0)
    assert solid[0].any() and solid.sum() >= 8
    fl = solid == 0
    rng = np.random.default_rng(4)
    for _ in range(3):
        f = W * (1 + 0.3 * (rng.random((ny, nx, 9)) - 0.5)) * fl[:, :, None]
        want = _flow_pull_step(f, solid, tau, u0)
        got = oracle.flow_steps(f.copy(), solid, tau, u0, 1)
        assert np.abs(got[fl] - want[fl]).max() < 1e-14


def test_initial_states_have_the_prescribed_moments():
    """Reading R13: the flow starts at equilibrium with rho = 1 and
    u = (u_in(y), 0) on every fluid node (zero on solid nodes); an ADR
    species starts at the second-order equilibrium of (C, u), whose zeroth,
    first and second moments are C, C u and C (I/3 + u u) exactly."""
    nx, ny, u0 = 13, 9, 0.05
    solid, _, _ = oracle.raster(nx, ny, [[6.2, 4.1, 2.0, 0, 0, -1]], 0, 0)
    fl = solid == 0
    f = oracle.flow_init_channel(solid, u0)
    rho, ux, uy = oracle.flow_moments(f, solid)
    yy = np.arange(ny)[:, None] * np.ones((1, nx))
    uin = 4 * u0 * (yy + 0.5) * (ny - 0.5 - yy) / ny ** 2
    assert np.abs(rho[fl] - 1).max() < 1e-15
    assert np.abs(ux[fl] - uin[fl]).max() < 1e-16
    assert np.abs(uy[fl]).max() < 1e-17
    assert not f[~fl].any()
    rng = np.random.default_rng(9)
    vx = 0.08 * (rng.random((ny, nx)) - 0.5) * fl
    vy = 0.08 * (rng.random((ny, nx)) - 0.5) * fl
    c0 = rng.random((3, ny, nx)) * fl
    g = oracle.adr_init(solid, vx, vy, c0)
    assert np.abs(g.sum(axis=3) - c0).max() < 1e-15
    assert np.abs((g * CX).sum(axis=3) - c0 * vx).max() < 1e-16
    assert np.abs((g * CY).sum(axis=3) - c0 * vy).max() < 1e-16
    # second moments of the D2Q9 equilibrium: C (I/3 + u u)
    assert np.abs((g * CX * CX).sum(axis=3) - c0 * (1 / 3 + vx * vx)).max() < 1e-15
    assert np.abs((g * CX * CY).sum(axis=3) - c0 * vx * vy).max() < 1e-16
    assert np.abs((g * CY * CY).sum(axis=3) - c0 * (1 / 3 + vy * vy)).max() < 1e-15
