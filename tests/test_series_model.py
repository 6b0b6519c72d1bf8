"""Pins of the collision-zone model of Sec. IV.A (host arithmetic of
paper_2109_04455_gb300.series): the zone width solves Eq. (d), the limits
of Eq. (eps), and the reading of the printed eps_coll."""
import math

import pytest

from paper_2109_04455_gb300 import series


@pytest.mark.parametrize("pe,r", [(0.5, 5.0), (7.0, 5.0), (100.0, 10.0)])
def test_collision_zone_solves_quadratic(pe, r):
    # Eq. (d) with explicit u0 and D = u0 R / Pe
    u0 = 0.05
    d_coef = u0 * r / pe
    d = series.collision_zone(pe, r)
    resid = d * d / (2 * d_coef) - math.pi / u0 * d - math.pi * r / u0
    assert abs(resid) < 1e-9 * (math.pi * r / u0)
    assert d > 0
    # the other root is negative
    other = 2 * d_coef * math.pi / u0 - d
    assert other < 0


def test_collision_zone_large_pe_scaling():
    # d -> R sqrt(2 pi / Pe) for Pe -> infinity
    for pe in (1e4, 1e6):
        assert series.collision_zone(pe, 5.0) / (5.0 * math.sqrt(
            2 * math.pi / pe)) == pytest.approx(1.0, rel=2 * math.sqrt(
                math.pi / (2 * pe)))


def test_model_limits():
    pe, r, l = 10.0, 5.0, 300.0
    d = series.collision_zone(pe, r)
    # every molecule of the zone that reaches the fiber reacts: eps_coll
    assert series.model_efficiency(pe, 1e9, r, l) == pytest.approx(
        0.5 * d / l, rel=1e-12)
    # no reaction
    assert series.model_efficiency(pe, 0.0, r, l) == 0.0
    # small Da: linear in Da with slope eps_coll alpha d^2 / (2 R^2)
    alpha = ((r + 0.5) ** 2 - r * r) / ((r + d) ** 2 - r * r)
    slope = 0.5 * d / l * alpha * d * d / (2 * r * r)
    assert series.model_efficiency(pe, 1e-6, r, l) == pytest.approx(
        slope * 1e-6, rel=1e-5)
    # efficiency falls with Pe (Sec. IV.A)
    vals = [series.model_efficiency(p, 150.0, r, l) for p in (1, 3, 10, 30)]
    assert all(a > b for a, b in zip(vals, vals[1:]))


def test_printed_eps_coll_differs_from_derived():
    # the printed closed form carries pi/(2 Pe) under the root; solving
    # Eq. (d) gives 2 pi / Pe (the model uses the derived form)
    pe, r, l = 7.0, 5.0, 300.0
    printed = 0.5 * (math.pi / pe + math.sqrt(math.pi ** 2 / pe ** 2 +
                                              math.pi / (2 * pe))) * r / l
    derived = 0.5 * series.collision_zone(pe, r) / l
    assert derived > printed * 1.2


def test_production_rate_is_outflux_times_width():
    assert series.production_rate([0.9, 0.08, 0.02], 300, 3) == \
        pytest.approx(6.0)
    assert series.production_rate([0.9, 0.1, 0.0], 300, 2) == \
        pytest.approx(30.0)


@pytest.mark.parametrize("n", [1, 6, 40])
def test_membrane_model_is_the_fiber_by_fiber_sum(n):
    # Eq. (eff_memb1): fiber i converts eps of what fibers 1..i-1 left
    pe, da, r, l = 7.0, 150.0, 5.0, 300.0
    e = series.model_efficiency(pe, da, r, l)
    left, total = 1.0, 0.0
    for _ in range(n):
        total += e * left
        left *= 1.0 - e
    assert series.membrane_model(pe, da, r, l, n) == pytest.approx(
        total, rel=1e-12)
    if n == 1:
        assert series.membrane_model(pe, da, r, l, 1) == pytest.approx(e)
