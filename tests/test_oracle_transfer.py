"""Pins of the grid transfers (Sec. 3.1, restriction and interpolation)."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("n,m", [(16, 16), (17, 12), (25, 31), (8, 5)])
def test_restriction_linear_and_constant(n, m):
    i, j = np.mgrid[0:n, 0:m].astype(float)
    a, b, c = 0.7, -1.3, 2.0
    r = O.restrict(a * j + b * i + c)
    nc, mc = n // 2, m // 2
    I, J = np.mgrid[0:nc, 0:mc].astype(float)
    exact = a * (2 * J + 1) + b * (2 * I + 1) + c          # coarse I sits on fine 2I+1
    inter_i = slice(0, nc if n % 2 else nc - 1)
    inter_j = slice(0, mc if m % 2 else mc - 1)
    assert np.allclose(r[inter_i, inter_j], exact[inter_i, inter_j], atol=1e-13)
    assert np.allclose(O.restrict(np.full((n, m), 3.25)), 3.25, atol=1e-15)


def test_restriction_is_the_papers_stencil():
    n = m = 12
    for (fi, fj) in [(5, 7), (4, 6), (5, 6)]:
        e = np.zeros((n, m)); e[fi, fj] = 1.0
        r = O.restrict(e)
        # the coarse cell (I, J) on fine (2I+1, 2J+1) weights fine offsets by [1 2 1]^T [1 2 1]/16
        for I in range(n // 2):
            for J in range(m // 2):
                di, dj = fi - (2 * I + 1), fj - (2 * J + 1)
                w = 0.0
                if abs(di) <= 1 and abs(dj) <= 1:
                    w = (2 - abs(di)) * (2 - abs(dj)) / 16.0
                assert abs(r[I, J] - w) < 1e-15


def test_restriction_boundary_rule_even_size():
    # even n: the last coarse cell takes (1/2, 1/2) of the last two fine cells along that axis
    f = np.arange(10 * 10, dtype=float).reshape(10, 10) ** 1.5
    r = O.restrict(f)
    w1 = np.array([0.25, 0.5, 0.25])
    wl = np.array([0.5, 0.5])
    ref = wl @ f[8:10, 4:7] @ w1
    assert abs(r[4, 2] - ref) < 1e-12
    ref = w1 @ f[2:5, 8:10] @ wl
    assert abs(r[1, 4] - ref) < 1e-12


@pytest.mark.parametrize("n,m", [(16, 16), (17, 13), (9, 24)])
def test_interpolation_linear_and_constant(n, m):
    nc, mc = n // 2, m // 2
    I, J = np.mgrid[0:nc, 0:mc].astype(float)
    a, b, c = -0.4, 0.9, 1.5
    e = a * (2 * J + 1) + b * (2 * I + 1) + c
    f = O.interpolate_add(e, np.zeros((n, m)))
    i, j = np.mgrid[0:n, 0:m].astype(float)
    exact = a * j + b * i + c
    ri = slice(1, n if n % 2 == 0 else n - 1)
    rj = slice(1, m if m % 2 == 0 else m - 1)
    assert np.allclose(f[ri, rj], exact[ri, rj], atol=1e-13)
    assert np.allclose(O.interpolate_add(np.full((nc, mc), 2.5), np.zeros((n, m))), 2.5)


def test_interpolation_is_the_papers_formula():
    # injection at (2i, 2j) (1-based), halves on edges, quarters at centres
    nc = mc = 5
    e = np.zeros((nc, mc)); e[2, 3] = 1.0
    f = O.interpolate_add(e, np.zeros((10, 10)))
    assert f[5, 7] == 1.0                                     # fine (2I+1, 2J+1)
    assert f[6, 7] == 0.5 and f[4, 7] == 0.5 and f[5, 8] == 0.5 and f[5, 6] == 0.5
    assert f[6, 8] == 0.25 and f[4, 6] == 0.25
    assert f.sum() == 4.0


def test_interpolation_is_four_times_restriction_transpose_inside():
    n = m = 14
    nc, mc = 7, 7
    R = np.zeros((nc * mc, n * m)); P = np.zeros((n * m, nc * mc))
    for q in range(n * m):
        e = np.zeros(n * m); e[q] = 1
        R[:, q] = O.restrict(e.reshape(n, m)).ravel()
    for q in range(nc * mc):
        e = np.zeros(nc * mc); e[q] = 1
        P[:, q] = O.interpolate_add(e.reshape(nc, mc), np.zeros((n, m))).ravel()
    fi, fj = np.mgrid[0:n, 0:m]
    inner_f = ((fi >= 1) & (fi <= n - 3) & (fj >= 1) & (fj <= m - 3)).ravel()
    ci, cj = np.mgrid[0:nc, 0:mc]
    inner_c = ((ci >= 1) & (ci <= nc - 2) & (cj >= 1) & (cj <= mc - 2)).ravel()
    assert np.allclose(P[np.ix_(inner_f, inner_c)], 4 * R.T[np.ix_(inner_f, inner_c)])
