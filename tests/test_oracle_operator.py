"""Pins of the discretisation (Sec. 2.2, eqs. rcabcd / abcdrc and the Spencer-Chen analogue)."""
import numpy as np
import pytest

import oracle as O


def _rand(n, m, seed=0):
    rng = np.random.default_rng(seed)
    phi = rng.normal(0, 3, (n, m))
    w = rng.uniform(0.2, 1.0, (n, m))
    Fn = rng.normal(0, 1, (n, m))
    return phi, w, Fn


@pytest.mark.parametrize("n,m,h", [(9, 7, 1.0), (16, 16, 2.0), (1, 5, 1.0), (6, 1, 4.0)])
def test_flux_conservation(n, m, h):
    # Each interior face carries one flux G_f (phi_b - phi_a) / h^2 that enters the two cells with
    # opposite signs, and boundary faces carry none (Neumann), so the diffusion part of delta^-1 N
    # sums to zero over the grid for any phi.
    phi, w, Fn = _rand(n, m)
    p = O.params(n, m, tau=2.0)
    L = O.apply_L(phi, w, Fn, h, p)
    diff = L + Fn + p.inv_tau * phi
    assert abs(diff.sum()) < 1e-10 * np.abs(diff).sum() + 1e-14


def test_frozen_matrix_is_symmetric_after_row_scaling():
    # A_ij/delta_ij and B_{i+1,j}/delta_{i+1,j} are the same face coefficient mu G_{i+1/2,j}/h^2
    phi, w, Fn = _rand(11, 13, 1)
    k = O.frozen_coeffs(phi, w, Fn, None, 2.0, O.params(11, 13))
    A, B, C, D, dl = (k[x] / k["delta"] if x != "delta" else k[x] for x in "A B C D delta".split())
    assert np.allclose(A[:-1, :], B[1:, :], rtol=1e-14)
    assert np.allclose(C[:, :-1], D[:, 1:], rtol=1e-14)
    assert np.all(A[-1, :] == 0) and np.all(B[0, :] == 0) and np.all(C[:, -1] == 0) and np.all(D[:, 0] == 0)
    # S and f as in eq. gslexrc plus the pseudo-time terms
    p = O.params(11, 13)
    assert np.allclose(k["S"], k["A"] + k["B"] + k["C"] + k["D"] + k["delta"] * p.inv_tau)
    assert np.allclose(k["f"], k["delta"] * Fn)
    eps = 1.0
    assert np.allclose(k["delta"], eps / (np.pi * (eps ** 2 + phi ** 2)))


def test_linear_phi_with_constant_weight():
    # phi = a x + b y + c: |grad phi| is constant, so G is constant and the discrete divergence
    # vanishes in the interior: L = -Fn - phi / tau there.
    n, m = 12, 10
    i, j = np.mgrid[0:n, 0:m].astype(float)
    phi = 0.8 * j - 0.5 * i + 3
    Fn = np.random.default_rng(2).normal(size=(n, m))
    p = O.params(n, m, tau=3.0)
    L = O.apply_L(phi, np.ones((n, m)), Fn, 1.0, p)
    ref = -Fn - phi / 3.0
    assert np.allclose(L[2:-2, 2:-2], ref[2:-2, 2:-2], atol=1e-12)


def test_discrete_curvature_of_a_cone_converges():
    # phi = R - r: the diffusion part equals mu div(grad phi / |grad phi|) = -mu / r in the limit
    # (eq. scel); second-order convergence under refinement of the cone's own scale.
    errs = []
    for s in (1, 2, 4):
        n = 64 * s
        i, j = np.mgrid[0:n, 0:n].astype(float)
        c = (n - 1) / 2.0
        r = np.hypot(i - c, j - c)
        phi = 50.0 * s - r
        p = O.params(n, n, tau=float("inf"), beta=1e-12, mu=1.0)
        L = O.apply_L(phi, np.ones((n, n)), np.zeros((n, n)), 1.0, p)
        ring = (r > 12 * s) & (r < 24 * s)
        kappa_scaled = L[ring] * s          # curvature in units of the cone's scale
        errs.append(np.max(np.abs(kappa_scaled + s / r[ring])))
    assert errs[0] < 0.02
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3


def test_single_cell_and_strip():
    p = O.params(1, 1, tau=2.0)
    L = O.apply_L(np.array([[5.0]]), np.array([[1.0]]), np.array([[0.5]]), 1.0, p)
    assert abs(L[0, 0] - (-0.5 - 2.5)) < 1e-15


def test_classification_rule():
    # Sec. 4.1 (set D: max/min > Sigma) and Sec. 4.1.3 (lag the smallest coefficient)
    assert O.classify(202, 202, 137391, 35) == 3            # Table 2 worst pixel: D smallest
    assert O.classify(1, 1, 1, 1) == -1
    assert O.classify(1, 1.9, 1.5, 1.2) == -1                 # max/min = 1.9 <= 2
    assert O.classify(1, 2.1, 1.5, 1.2) == 0
    assert O.classify(5, 1, 1, 9) == 1                        # ties go to the earlier letter
    assert O.classify(0, 3, 1, 1, has=(0, 1, 1, 1)) == 2     # boundary face A excluded
    assert O.classify(0, 3, 0, 0, has=(0, 1, 0, 0)) == -1    # a single face: no jump
    assert O.classify(0.0, 1.0, 1.0, 1.0) == 0                # a zero face is a jump
