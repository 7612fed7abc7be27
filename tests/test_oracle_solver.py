"""Pins of the coarsest solve, the FAS V-cycle (Algorithm 1) and the driver invariants."""
import numpy as np
import pytest
from scipy.linalg import lu_factor, lu_solve

import oracle as O
from paper_1807_02137_gb300 import synth


def small_problem(n, seed=0, model=0):
    img, mk, _ = synth.disc_square(n, 0.05, seed)
    p = O.params(n, n, levels=1, model=model)
    s = O.Solver(img, mk, p)
    s.begin_step()
    return s, p


def dense_picard(phi, w, Fn, rhs, h, p, iters=200):
    """Picard on the frozen coefficients with dense LU (scipy), rows divided by delta."""
    n, m = phi.shape
    N = n * m
    for _ in range(iters):
        k = O.frozen_coeffs(phi, w, Fn, rhs, h, p)
        dl = k["delta"]
        K = np.zeros((N, N))
        b = -(k["f"] / dl).ravel()
        for i in range(n):
            for j in range(m):
                q = i * m + j
                K[q, q] = (k["A"][i, j] + k["B"][i, j] + k["C"][i, j] + k["D"][i, j]) / dl[i, j] + p.inv_tau
                if i + 1 < n: K[q, q + m] = -k["A"][i, j] / dl[i, j]
                if i > 0: K[q, q - m] = -k["B"][i, j] / dl[i, j]
                if j + 1 < m: K[q, q + 1] = -k["C"][i, j] / dl[i, j]
                if j > 0: K[q, q - 1] = -k["D"][i, j] / dl[i, j]
        new = lu_solve(lu_factor(K), b).reshape(n, m)
        if np.max(np.abs(new - phi)) <= 1e-14 * max(1.0, np.max(np.abs(new))):
            return new
        phi = new
    return phi


@pytest.mark.parametrize("n", [16, 32])
def test_coarse_solve_matches_dense_lu_picard(n):
    s, p = small_problem(n)
    phi0, w, Fn = s.phi, s.level(0, "w"), s.level(0, "Fn")
    rhs = np.random.default_rng(1).normal(0, 0.1, (n, n))
    p.coarse_maxit, p.coarse_tol = 500, 1e-15
    got, it = O.coarse_solve(phi0, w, Fn, rhs, 2.0, p)
    ref = dense_picard(phi0, w, Fn, rhs, 2.0, p)
    assert it > 0
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    # the fixed point solves the nonlinear equation L(phi) = rhs
    res = rhs - O.apply_L(got, w, Fn, 2.0, p)
    assert np.linalg.norm(res) <= 1e-8 * np.linalg.norm(rhs - O.apply_L(phi0, w, Fn, 2.0, p))


@pytest.mark.parametrize("n,levels", [(16, 3), (32, 4), (37, 3)])
def test_fas_vcycles_converge_to_the_direct_solution(n, levels):
    img, mk, _ = synth.disc_square(n, 0.05, 3)
    p = O.params(n, n, levels=levels)
    s = O.Solver(img, mk, p)
    s.begin_step()
    phin, w, Fn = s.phi, s.level(0, "w"), s.level(0, "Fn")
    for _ in range(60):
        r = s.vcycle()
        if r < 1e-12:
            break
    assert r < 1e-11
    ref = dense_picard(phin, w, Fn, np.zeros((n, n)), 1.0, p)
    assert np.max(np.abs(s.phi - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_first_step_residual_decreases_every_cycle():
    W = synth.workload("disc128")
    p = O.params(128, 128, levels=W.levels)
    s = O.Solver(W.image, W.markers, p)
    hist = s.solve_step(W.tol, 40)
    assert hist[-1] <= W.tol
    assert all(b < a for a, b in zip(hist, hist[1:]))


def test_two_region_image_gives_the_exact_region_mask():
    # A clean two-valued image (a disc on a background) with markers inside the disc: after a
    # few pseudo-time steps sign(phi) is the disc exactly.
    n = 64
    i, j = np.mgrid[0:n, 0:n].astype(float)
    disc = (i - 30) ** 2 + (j - 34) ** 2 <= 15 ** 2
    img = np.where(disc, 0.8, 0.2)
    ang = np.linspace(0, 2 * np.pi, 8, endpoint=False)
    mk = np.stack([34 + 10 * np.cos(ang), 30 + 10 * np.sin(ang)], 1).round()
    s = O.Solver(img, mk, O.params(n, n, levels=4))
    for _ in range(14):
        s.solve_step(1e-10, 60)
        s.end_step()
    assert np.array_equal(s.phi > 0, disc)


def test_rada_chen_area_term():
    # The Rada-Chen bracket adds 2 nu (h^2 sum H / |Omega| - A1 / |Omega|) to the fitting term
    # (eqs. rcabcd and gslexrc); with w and the fitting field equal, the two models' operators
    # differ by exactly that scalar.
    n = 12
    rng = np.random.default_rng(4)
    phi, w, Fn = rng.normal(0, 2, (n, n)), rng.uniform(0.5, 1, (n, n)), rng.normal(size=(n, n))
    psc = O.params(n, n, model=0)
    prc = O.params(n, n, model=1, nu=0.7)
    A1 = 30.0
    d = O.apply_L(phi, w, Fn, 2.0, prc, n0m0=4.0 * n * n, A1=A1) - O.apply_L(phi, w, Fn, 2.0, psc)
    H = 0.5 + np.arctan(phi) / np.pi
    ref = -2 * 0.7 * (4.0 * H.sum() / (4.0 * n * n) - A1 / (4.0 * n * n))
    assert np.allclose(d, ref, atol=1e-13)


def test_rada_chen_fas_converges():
    img, mk, _ = synth.disc_square(64, 0.05, 5)
    s = O.Solver(img, mk, O.params(64, 64, levels=4, model=1))
    hist = s.solve_step(1e-8, 60)
    assert hist[-1] <= 1e-8


def test_paper_orderings_converge_too():
    # Both orderings of Hybrid Smoother 2 (Algorithm 3), of GSLINE-I (Algorithm 1) and of Hybrid
    # Smoother 1 (Algorithm 2) drive the same first step to the same solution.
    img, mk, _ = synth.disc_square(64, 0.05, 6)
    sols = []
    for sm in (0, 1, 2, 3, 4, 5):
        s = O.Solver(img, mk, O.params(64, 64, levels=4, smoother=sm))
        hist = s.solve_step(1e-10, 80)
        assert hist[-1] <= 1e-10
        sols.append(s.phi)
    for x in sols[1:]:
        assert np.allclose(sols[0], x, atol=1e-8)


def _ellipse_solver(n, seed, tau=1.0):
    img, mk, _ = synth.ellipses(n, n, 12, (20 * n / 256, 200 * n / 256), 8, 0.05, seed, dtype=np.float64)
    lev = 1
    s = n
    while s // 2 >= 4:
        s //= 2
        lev += 1
    return O.Solver(img, mk, O.params(n, n, levels=lev, tau=tau)), img, mk, lev


def test_step_control_rejects_a_stalled_attempt_and_restarts_from_phi_n():
    # 64^2 ellipses, seed 1: the first step's attempt with tau = 1 stalls (two V-cycles gain less
    # than a factor 1 / 0.6); the step is retried from phi^n with tau = 1/2 and converges
    o, img, mk, lev = _ellipse_solver(64, 1)
    phin = o.phi
    tau, att = o.solve_step_controlled(1.0, 1e-6, stall_ratio=0.6)
    assert len(att) >= 2 and tau == 0.5 ** (len(att) - 1)
    for k, (t, h) in enumerate(att[:-1]):
        assert t == 0.5 ** k
        stalled = len(h) >= 4 and h[-1] > 0.6 * h[-3]
        assert stalled or len(h) == 40 or not np.isfinite(h[-1]) or h[-1] > 1e3
        assert h[-1] > 1e-6
    assert att[-1][1][-1] <= 1e-6
    got = o.phi
    # the accepted attempt started from phi^n: the same step solved directly with the accepted
    # tau gives the same phi, bitwise
    o2, *_ = _ellipse_solver(64, 1, tau=tau)
    assert np.array_equal(o2.phi, phin)
    h2 = o2.solve_step(1e-6, 40)
    assert h2 == att[-1][1]
    assert np.array_equal(o2.phi, got)


@pytest.mark.parametrize("n,seed", [(48, 2), (64, 3)])
def test_every_controlled_step_reaches_the_tolerance(n, seed):
    # with tau fixed at 1, the later steps of these images stall (rho ~ 1e-3); under the step
    # control every step reaches rho <= 1e-6 and tau never grows
    o, *_ = _ellipse_solver(n, seed)
    tau, taus = 1.0, []
    for _ in range(3):
        tau, att = o.solve_step_controlled(tau, 1e-6)
        o.end_step()
        assert att[-1][1][-1] <= 1e-6
        taus.append(tau)
    assert all(b <= a for a, b in zip(taus, taus[1:]))


def test_all_core_build_gives_bitwise_the_serial_results():
    # the -fopenmp build (the all-core timing baseline) runs the independent loops in parallel;
    # every V-cycle equals the serial checker's bitwise
    img, mk, _ = synth.ellipses(96, 80, 8, (10, 50), 6, 0.05, 4, dtype=np.float64)
    out = []
    for omp in (False, True):
        s = O.Solver(img, mk, O.params(96, 80, levels=5), openmp=omp)
        s.begin_step()
        rhos = [s.vcycle() for _ in range(3)]
        out.append((rhos, s.phi))
        s.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])
