"""Pins of the oracle's level-set energy (eq. scfunc / rcfunc) against facts that do not retype
its formula: the co-area formula for the length term, region variances for the fitting terms,
and the closed forms of the distance and area terms of a sharp level set."""
import numpy as np
import pytest

import oracle as O


def _params(**kw):
    base = dict(mu=0.0, lambda1=0.0, lambda2=0.0, theta=0.0, nu=0.0)
    base.update(kw)
    return O.params(64, 64, **base)


def test_straight_contour_length_by_coarea():
    # phi = x - x0 with w = 1: sum delta(phi) |grad phi| approximates the length n of the
    # vertical zero line (the integral of the Cauchy-shaped delta is 1; its tails beyond the
    # grid and the sampling error stay below 1.5%)
    n, m = 80, 201
    x = np.arange(m, dtype=float)
    phi = np.tile(x - 100.3, (n, 1))
    p = _params(mu=1.7)
    ones, zeros = np.ones((n, m)), np.zeros((n, m))
    E = O.energy(phi, zeros, ones, zeros, 0.0, 0.0, 0.0, p)
    assert abs(E / (1.7 * n) - 1.0) < 0.015


def test_circle_length_by_coarea():
    n = m = 160
    yy, xx = np.mgrid[0:n, 0:m].astype(float)
    r0 = 37.0
    phi = r0 - np.hypot(xx - 80.2, yy - 79.6)          # signed distance, positive inside
    p = _params(mu=1.0)
    ones, zeros = np.ones((n, m)), np.zeros((n, m))
    E = O.energy(phi, zeros, ones, zeros, 0.0, 0.0, 0.0, p)
    assert abs(E / (2 * np.pi * r0) - 1.0) < 0.02


def test_length_term_uses_the_weight():
    # halving w halves the length term; Rada-Chen uses w as given (the caller's d g)
    n, m = 40, 120
    phi = np.tile(np.arange(m) - 60.5, (n, 1)).astype(float)
    zeros = np.zeros((n, m))
    for model in (0, 1):
        p = O.params(n, m, mu=1.0, lambda1=0.0, lambda2=0.0, theta=0.0, nu=0.0, model=model)
        e1 = O.energy(phi, zeros, np.ones((n, m)), zeros, 0, 0, 0, p)
        e2 = O.energy(phi, zeros, 0.5 * np.ones((n, m)), zeros, 0, 0, 0, p)
        assert abs(e2 / e1 - 0.5) < 1e-12


def _sharp_disc(n, m, eps_small=1e-9):
    yy, xx = np.mgrid[0:n, 0:m].astype(float)
    inside = np.hypot(xx - 0.4 * m, yy - 0.55 * n) < 0.3 * min(n, m)
    phi = np.where(inside, 1.0, -1.0)
    return phi, inside


def test_fitting_terms_equal_region_variances():
    n, m = 50, 70
    rng = np.random.default_rng(4)
    z = rng.uniform(0, 1, (n, m))
    phi, inside = _sharp_disc(n, m)
    c1, c2 = 0.31, 0.77
    p = _params(lambda1=2.0, lambda2=3.0, eps=1e-9)
    E = O.energy(phi, z, np.ones((n, m)), np.zeros((n, m)), c1, c2, 0.0, p)
    zi, zo = z[inside], z[~inside]
    expect = 2.0 * zi.size * (np.var(zi) + (np.mean(zi) - c1) ** 2) \
        + 3.0 * zo.size * (np.var(zo) + (np.mean(zo) - c2) ** 2)
    assert abs(E - expect) <= 1e-7 * expect


def test_distance_term_of_a_sharp_level_set():
    n, m = 48, 52
    rng = np.random.default_rng(5)
    d = rng.uniform(0, 1, (n, m))
    phi, inside = _sharp_disc(n, m)
    p = _params(theta=1.5, eps=1e-9)
    E = O.energy(phi, np.zeros((n, m)), np.ones((n, m)), d, 0, 0, 0, p)
    assert abs(E - 1.5 * d[inside].sum()) <= 1e-7 * E
    # Rada-Chen has no standalone distance term
    p1 = O.params(n, m, mu=0.0, lambda1=0.0, lambda2=0.0, theta=1.5, nu=0.0, eps=1e-9, model=1)
    assert abs(O.energy(phi, np.zeros((n, m)), np.ones((n, m)), d, 0, 0, 0, p1)) < 1e-6


@pytest.mark.parametrize("A1", [0.0, 300.0, 1234.5])
def test_area_term_of_a_sharp_level_set(A1):
    n, m = 40, 60
    phi, inside = _sharp_disc(n, m)
    p = O.params(n, m, mu=0.0, lambda1=0.0, lambda2=0.0, theta=0.0, nu=2.5, eps=1e-9, model=1)
    E = O.energy(phi, np.zeros((n, m)), np.ones((n, m)), np.zeros((n, m)), 0, 0, A1, p)
    K = inside.sum()
    assert abs(E - 2.5 * (K - A1) ** 2 / (n * m)) <= 1e-6 * max(E, 1.0)


def test_solver_energy_is_finite_and_falls_over_steps():
    # a pseudo-time step lowers the energy of the two-region test image from its initial contour
    from paper_1807_02137_gb300 import synth
    W = synth.workload("disc128")
    p = O.params(128, 128, levels=W.levels)
    s = O.Solver(W.image, W.markers, p)
    e0 = s.energy()
    s.solve_step(1e-8, 40)
    e1 = s.energy()
    s.end_step()
    assert np.isfinite(e0) and np.isfinite(e1) and e1 < e0
    s.close()
