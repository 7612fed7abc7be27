"""Pins of the oracle's learned relaxation weights: convolution against a library routine, the
feature and rounding definitions by hand, the damped smoother against its block definition,
the loss gradient against finite differences, the first Adam step's closed form."""
import numpy as np
import pytest
from scipy.signal import correlate2d

import oracle as O
from oracle import learned as NL
from tests.test_oracle_smoother import assemble, block_matrix, parallel_phases, rand_coef


def test_conv3_is_zero_padded_cross_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 7, 9))
    W = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    y = NL.conv3(x, W, b)
    for o in range(2):
        ref = b[o] + sum(correlate2d(x[i], W[o, i], mode="same", boundary="fill") for i in range(3))
        assert np.allclose(y[o], ref, atol=1e-12)


def test_features_by_hand():
    cS, cN, cE, cW = (np.full((1, 1), v) for v in (1.0, 2.0, 3.0, 4.0))
    x = NL.features(cS, cN, cE, cW)[:, 0, 0]
    assert np.allclose(x[:4], [0.1, 0.2, 0.3, 0.4])
    assert np.isclose(x[4], np.log(4.0) / 8)
    # a boundary face (zero) takes no part in the max / min ratio
    x = NL.features(np.zeros((1, 1)), *(np.full((1, 1), v) for v in (2.0, 3.0, 6.0)))[:, 0, 0]
    assert np.allclose(x[:4], [0.0, 2 / 11, 3 / 11, 6 / 11]) and np.isclose(x[4], np.log(3.0) / 8)


def test_bf16_rounding():
    vals = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, 1 / 3, -2.5])
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, 0.333984375, -2.5])
    assert np.array_equal(NL.bf16_round(vals), want)


def _crop(n, m, seed):
    rng = np.random.default_rng(seed)
    c = np.exp(rng.normal(0, 1.2, (4, n, m)))
    c[0][-1], c[1][0], c[2][:, -1], c[3][:, 0] = 0, 0, 0, 0
    S = c.sum(axis=0) + 0.3
    f = rng.normal(size=(n, m))
    u = rng.normal(size=(n, m))
    return c, S, f, u


def test_damped_red_black_residual_identities():
    # plain GS zeroes the residual at the cells it updates; weight omega leaves (1 - omega) of it
    c, S, f, u = _crop(9, 11, 1)
    om = np.random.default_rng(2).uniform(0.3, 1.7, u.shape)
    n, m = u.shape
    ii, jj = np.mgrid[0:n, 0:m]
    inner = (ii >= 1) & (ii < n - 1) & (jj >= 1) & (jj < m - 1)
    red = inner & ((ii + jj) % 2 == 0)
    r0 = NL.residual(c, S, f, u)
    # red phase only: run with the black cells' weights set to zero
    u1 = NL.damped_rb(c, S, f, u, np.where(red, om, 0.0))
    r1 = NL.residual(c, S, f, u1)
    assert np.allclose(r1[red], (1 - om[red]) * r0[red], atol=1e-12)
    u1 = NL.damped_rb(c, S, f, u, np.where(red, 1.0, 0.0))
    assert np.allclose(NL.residual(c, S, f, u1)[red], 0.0, atol=1e-12)


@pytest.mark.parametrize("seed,loss", [(3, "full"), (4, "full"), (5, "hf"), (6, "hf")])
def test_loss_gradient_matches_finite_differences(seed, loss):
    rng = np.random.default_rng(seed)
    c, S, f, u = _crop(10, 12, seed)
    theta = rng.normal(0, 0.3, NL.NPARAM)
    value, g = NL.crop_loss_grad(theta, c, S, f, u, loss=loss)
    assert np.isclose(value, NL.crop_loss(theta, c, S, f, u, loss=loss), rtol=1e-13)
    idx = rng.choice(NL.NPARAM, 40, replace=False)
    idx = np.concatenate([idx, [NL.NPARAM - 1, 0, 720, 736]])   # b3, W1, b1, W2 first entries
    def fd(k, h):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        return (NL.crop_loss(tp, c, S, f, u, loss=loss) - NL.crop_loss(tm, c, S, f, u, loss=loss)) / (2 * h)

    for k in idx:
        if loss == "full":
            d = fd(k, 1e-6)
        else:
            # the high-pass loss is larger and more curved: Richardson extrapolation of two
            # central differences (error O(h^4)) at a step where rounding stays small
            d = (4.0 * fd(k, 5e-5) - fd(k, 1e-4)) / 3.0
        assert abs(d - g[k]) <= 1e-6 * max(1.0, abs(d)) + 1e-9, (k, d, g[k])


def test_high_pass_symbol():
    # h = 4 r - (sum of the neighbours): zero on constants and linear functions, 8 r on the
    # checkerboard mode, (4 - 2 cos t1 - 2 cos t2) r on a plane wave (interior cells)
    n = 12
    ii, jj = np.mgrid[0:n, 0:n].astype(float)
    inner = (slice(2, n - 2), slice(2, n - 2))
    assert np.allclose(NL.high_pass(np.full((n, n), 3.0))[inner], 0.0)
    assert np.allclose(NL.high_pass(2 * ii - jj + 1)[inner], 0.0)
    chk = (-1.0) ** (ii + jj)
    assert np.allclose(NL.high_pass(chk)[inner], 8.0 * chk[inner])
    t1, t2 = 0.7, 1.9
    wave = np.cos(t1 * ii + t2 * jj)
    assert np.allclose(NL.high_pass(wave)[inner], (4 - 2 * np.cos(t1) - 2 * np.cos(t2)) * wave[inner])


def test_first_adam_step_moves_by_lr_times_sign():
    rng = np.random.default_rng(5)
    theta = rng.normal(size=50)
    grad = rng.normal(size=50)
    state = (np.zeros(50), np.zeros(50), 0)
    t1, _ = NL.adam_step(theta, grad, state, 0.01)
    assert np.allclose(t1 - theta, -0.01 * np.sign(grad), rtol=1e-6)


def test_damped_hybrid_smoother_matches_block_definition():
    # point blocks take the weighted update e_c <- (1 - w_c) e_c + w_c (exact block value);
    # line groups are unchanged
    n, m = 7, 9
    K = rand_coef(n, m, 8)
    om = np.random.default_rng(9).uniform(0.4, 1.6, (n, m))
    N = n * m
    Kz = dict(K)
    Kz["f"] = np.zeros((n, m))
    T = np.zeros((N, N))
    for q in range(N):
        e = np.zeros(N)
        e[q] = 1
        T[:, q] = O.smooth_given_omega(Kz, om, e.reshape(n, m), 2.0, 0).ravel()
    M = assemble(K)
    Tref = np.eye(N)
    for blocks in parallel_phases(K):
        Tp = np.eye(N)
        for P in blocks:
            P = np.asarray(P)
            rest = np.setdiff1d(np.arange(N), P)
            exact = np.zeros((len(P), N))
            exact[:, rest] = -np.linalg.solve(M[np.ix_(P, P)], M[np.ix_(P, rest)])
            if len(P) == 1:
                w = om.ravel()[P[0]]
                row = w * exact[0]
                row[P[0]] += 1 - w
                Tp[P[0]] = row
            else:
                Tp[P] = exact
        Tref = Tp @ Tref
    # the point phases are the single-cell blocks; groups come from the line phases
    assert np.allclose(T, Tref, atol=1e-11)
    # omega = 1 is the plain smoother
    T1 = O.smooth_given_omega(Kz, np.ones((n, m)), np.arange(N, dtype=float).reshape(n, m), 2.0, 0)
    assert np.array_equal(T1, O.smooth_given(Kz, np.arange(N, dtype=float).reshape(n, m), 2.0, 0))
