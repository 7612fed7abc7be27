"""Pins of the fitting field (the data terms of eq. scel / rcel) and of the pseudo-time term.

The fitting field is the first variation of the energy's data terms (Sec. 2.2, eqs. scfunc /
rcfunc -> scel / rcel).  The energy (`or_energy`) is pinned on its own by closed forms
(tests/test_oracle_energy.py), so its central finite differences give the field independently
of `or_fitting`:  with mu = 0 (no length term) and tau = inf,
    L(phi)_ij * delta_eps(phi_ij) = -dE/dphi_ij,
and with a finite tau the step equation L(phi) = 0 decouples cell by cell into
    phi = phi^n - tau (dE/dphi_ij) / delta_eps(phi_ij),
which one V-cycle reaches exactly.  lambda1 != lambda2 and theta != 0 make a swapped fitting
term, a flipped distance term or a dropped phi^n / tau term fail.
"""
import numpy as np
import pytest

import oracle as O


def energy_gradient(phi, z, w, d, c1, c2, A1, p, h=1e-5):
    """Central differences of or_energy in every cell."""
    g = np.empty_like(phi)
    for q in np.ndindex(phi.shape):
        a, b = phi.copy(), phi.copy()
        a[q] += h
        b[q] -= h
        g[q] = (O.energy(a, z, w, d, c1, c2, A1, p) - O.energy(b, z, w, d, c1, c2, A1, p)) / (2 * h)
    return g


def case(seed, n=9, m=11):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(-2.5, 2.5, (n, m))
    z = rng.uniform(0, 1, (n, m))
    w = rng.uniform(0.2, 1, (n, m))
    d = rng.uniform(0, 1, (n, m))
    return phi, z, w, d


@pytest.mark.parametrize("model", [0, 1])
def test_fitting_field_is_the_first_variation_of_the_data_terms(model):
    phi, z, w, d = case(1 + model)
    n, m = phi.shape
    c1, c2, A1 = 0.71, 0.23, 30.0
    p = O.params(n, m, model=model, mu=0.0, lambda1=3.0, lambda2=7.0, theta=2.5, nu=4.0, tau=None)
    Fn = O.fitting(z, d, np.zeros_like(phi), c1, c2, p)
    L = O.apply_L(phi, w, Fn, 1.0, p, n0m0=float(n * m), A1=A1)
    delta = O.frozen_coeffs(phi, w, Fn, None, 1.0, p, n0m0=float(n * m), A1=A1)["delta"]
    grad = energy_gradient(phi, z, w, d, c1, c2, A1, p)
    scale = np.max(np.abs(grad))
    assert scale > 1e-2
    assert np.max(np.abs(L * delta + grad)) <= 1e-7 * scale


def test_pseudo_time_step_without_length_term_is_the_explicit_formula():
    from paper_1807_02137_gb300 import synth
    img, mk, _ = synth.ellipses(24, 20, 3, (6, 14), 4, 0.05, 5, dtype=np.float64)
    n, m = img.shape
    tau = 0.5
    p = O.params(n, m, mu=0.0, lambda1=3.0, lambda2=7.0, theta=2.5, tau=tau, levels=3)
    s = O.Solver(img, mk, p)
    phin = s.phi
    sc = s.scalars()
    z, w, d = s.level(0, "z"), s.level(0, "w"), s.level(0, "d")
    s.begin_step()
    rho = s.vcycle()
    assert rho <= 1e-12
    Fn = s.level(0, "Fn")
    delta = O.frozen_coeffs(phin, w, Fn, None, 1.0, p)["delta"]
    grad = energy_gradient(phin, z, w, d, sc["c1"], sc["c2"], sc["A1"], p)
    want = phin - tau * grad / delta
    assert np.max(np.abs(s.phi - want)) <= 1e-7 * np.max(np.abs(want))
    s.close()
