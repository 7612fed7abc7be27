"""Pins of the oracle's image-derived data (Sec. 2.2) and initialisation (Sec. 5)."""
import numpy as np

import oracle as O


def test_blur_preserves_constants_and_linear_functions():
    z = np.full((20, 17), 0.37)
    assert np.allclose(O.gauss_blur(z, 1.0), 0.37, atol=1e-15)
    i, j = np.mgrid[0:20, 0:17]
    lin = 0.3 * i - 0.2 * j + 1.0
    b = O.gauss_blur(lin, 1.0)
    # a symmetric normalised kernel reproduces linear functions away from the mirror boundary
    assert np.allclose(b[3:-3, 3:-3], lin[3:-3, 3:-3], atol=1e-13)


def test_blur_impulse_response_is_normalised_gaussian():
    z = np.zeros((21, 21))
    z[10, 10] = 1.0
    b = O.gauss_blur(z, 1.0)
    t = np.arange(-3, 4)
    g1 = np.exp(-t ** 2 / 2.0)
    g1 /= g1.sum()
    ref = np.zeros((21, 21))
    ref[7:14, 7:14] = np.outer(g1, g1)
    assert np.allclose(b, ref, atol=1e-15)
    assert abs(b.sum() - 1) < 1e-14


def test_edge_detector_closed_forms():
    assert np.allclose(O.edge_detector(np.full((8, 9), 2.0)), 1.0)
    i, j = np.mgrid[0:12, 0:10].astype(float)
    a, c = 0.3, -0.4
    g = O.edge_detector(a * j + c * i, 2.0)
    # central differences of a linear function are exact in the interior
    assert np.allclose(g[1:-1, 1:-1], 1.0 / (1.0 + 2.0 * (a * a + c * c)), atol=1e-15)
    # mirror boundary halves the one-sided difference at the edge column
    assert np.allclose(g[1:-1, 0], 1.0 / (1.0 + 2.0 * ((a / 2) ** 2 + c * c)), atol=1e-15)


def test_distance_function():
    d = O.distance(30, 40, [[10, 12]], 3.0)
    assert d[12, 10] == 0.0                        # zero at the marker
    assert d[0, 39] > 1 - 1e-12                      # one far away
    r2 = (np.arange(40)[None, :] - 10) ** 2 + (np.arange(30)[:, None] - 12) ** 2
    assert np.allclose(d, 1 - np.exp(-r2 / 18.0), atol=1e-15)
    d2 = O.distance(30, 40, [[10, 12], [30, 5]], 3.0)
    e = O.distance(30, 40, [[30, 5]], 3.0)
    assert np.allclose(d2, d * e, atol=1e-15)         # product over markers


def test_initial_phi_square_hull():
    mk = [[10, 10], [30, 10], [30, 30], [10, 30], [20, 20]]   # interior point is not on the hull
    phi, area, h = O.initial_phi(41, 41, mk)
    assert h == 4 and abs(area - 400.0) < 1e-12
    assert abs(phi[20, 20] - 10.0) < 1e-12           # centre: 10 px from every edge
    assert abs(phi[0, 20] + 10.0) < 1e-12            # above the top edge
    assert abs(phi[0, 0] + np.sqrt(200.0)) < 1e-12   # nearest point is a corner
    assert phi[10, 20] == 0.0 and phi[15, 15] > 0 and phi[5, 15] < 0


def test_initial_phi_degenerate_markers_fall_back_to_disc():
    for mk in ([[20, 20]], [[10, 20], [30, 20]], [[10, 10], [20, 20], [30, 30]]):
        phi, area, h = O.initial_phi(40, 40, mk, r0=5.0)
        cx = np.mean([p[0] for p in mk]); cy = np.mean([p[1] for p in mk])
        i, j = np.mgrid[0:40, 0:40]
        assert h == 0 and abs(area - np.pi * 25) < 1e-12
        assert np.allclose(phi, 5.0 - np.hypot(j - cx, i - cy))


def test_region_means():
    z = np.full((10, 10), 0.2)
    z[:, :5] = 0.9
    phi = np.where(z > 0.5, 1e6, -1e6)
    c1, c2 = O.region_means(phi, z)
    assert abs(c1 - 0.9) < 1e-6 and abs(c2 - 0.2) < 1e-6
    c1, c2 = O.region_means(np.random.default_rng(0).normal(size=(7, 9)), np.full((7, 9), 0.4))
    assert abs(c1 - 0.4) < 1e-15 and abs(c2 - 0.4) < 1e-15
