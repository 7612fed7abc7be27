"""Pins of the oracle's AOS time marching (additive operator splitting of the artificial
evolution d phi / ds = L(phi) - rhs): consistency with the operator L, the closed form of the
reaction-only problem, and the behaviour of its fixed point."""
import numpy as np
import pytest

import oracle as O


def _problem(n, m, seed, model=0):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:n, 0:m].astype(float)
    phi = 12.0 - np.hypot(xx - 0.45 * m, yy - 0.5 * n) + 0.3 * rng.normal(size=(n, m))
    w = 0.2 + rng.uniform(0, 1, (n, m))
    Fn = rng.normal(0, 1, (n, m)) - phi          # fitting field minus phi^n / tau (tau = 1)
    rhs = 0.1 * rng.normal(size=(n, m))
    p = O.params(n, m, model=model, nu=0.5)
    return phi, w, Fn, rhs, p


def _L(phi, w, Fn, p, A1=0.0):
    n, m = phi.shape
    return O.apply_L(phi, w, Fn, h=1.0, p=p, n0m0=float(n * m), A1=A1)


@pytest.mark.parametrize("model", [0, 1])
def test_aos_step_is_consistent_with_L(model):
    # (phi_new - phi) / dt -> L(phi) - rhs as dt -> 0, with an error of order dt
    phi, w, Fn, rhs, p = _problem(20, 24, 1, model)
    target = _L(phi, w, Fn, p, A1=60.0) - rhs
    errs = []
    for dt in (1e-4, 5e-5, 2.5e-5):
        new = O.aos_iteration(phi, w, Fn, rhs, p=p, A1=60.0, dt=dt)
        errs.append(np.max(np.abs((new - phi) / dt - target)))
    scale = np.max(np.abs(target))
    assert errs[-1] < 1e-3 * scale
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def test_reaction_only_problem_has_the_closed_form_step():
    # mu = 0: both directions reduce to (1 + dt / tau) y = phi + dt c, c = -(Fn + rhs), so the
    # step and its fixed point c tau are known exactly
    phi, w, Fn, rhs, p = _problem(9, 13, 2)
    p.mu = 0.0
    dt = 0.7
    new = O.aos_iteration(phi, w, Fn, rhs, p=p, dt=dt)
    c = -(Fn + rhs)
    assert np.allclose(new, (phi + dt * c) / (1 + dt), rtol=0, atol=1e-13)
    x = phi.copy()
    for _ in range(200):
        x = O.aos_iteration(x, w, Fn, rhs, p=p, dt=dt)
    assert np.allclose(x, c, atol=1e-12)
    assert np.max(np.abs(_L(x, w, Fn, p) - rhs)) < 1e-10


def test_fixed_point_residual_shrinks_with_dt():
    # on a linear problem (beta large: G does not depend on phi) AOS converges to a fixed point
    # that solves L(phi) = rhs up to a splitting error proportional to dt
    n = m = 16
    rng = np.random.default_rng(3)
    yy, xx = np.mgrid[0:n, 0:m].astype(float)
    phi = 0.8 * xx - 0.5 * yy + 2 * np.sin(xx / 3) * np.cos(yy / 4)
    w = 0.5 + 0.5 * rng.uniform(0, 1, (n, m))
    Fn = rng.normal(0, 1, (n, m)) - phi
    rhs = 0.1 * rng.normal(size=(n, m))
    p = O.params(n, m, mu=50.0, beta=1e6)
    r0 = np.linalg.norm(_L(phi, w, Fn, p) - rhs)
    res = []
    for dt in (0.1, 0.05):
        x = phi.copy()
        for _ in range(600):
            x = O.aos_iteration(x, w, Fn, rhs, p=p, dt=dt)
        step = O.aos_iteration(x, w, Fn, rhs, p=p, dt=dt)
        assert np.max(np.abs(step - x)) < 1e-12 * np.max(np.abs(x))     # converged
        res.append(np.linalg.norm(_L(x, w, Fn, p) - rhs))
    assert res[1] < 1e-3 * r0
    assert 1.7 < res[0] / res[1] < 2.3


def test_vcycles_with_aos_coarsest_solver_converge():
    from paper_1807_02137_gb300 import synth
    W = synth.workload("disc128")
    s = O.Solver(W.image, W.markers, O.params(128, 128, levels=5, coarse_solver=1, aos_dt=10.0))
    hist = s.solve_step(1e-8, 60)
    assert hist[-1] <= 1e-8
    assert all(b < a for a, b in zip(hist, hist[1:]))
    s.close()


def test_finest_grid_aos_reduces_the_residual():
    from paper_1807_02137_gb300 import synth
    W = synth.workload("disc128")
    s = O.Solver(W.image, W.markers, O.params(128, 128, levels=5))
    s.begin_step()
    it, rho = s.aos(0.5, 400, 1e-6)
    assert it > 10 and rho < 0.5
    s.close()
