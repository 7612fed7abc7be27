"""Pins of the smoothers (Sec. 3.2 GSLEX-I / GSLINE-I, Sec. 4.3 Hybrid Smoother 2).

The smoothers are linear stationary iterations once the coefficients are frozen, so each one
has an error-propagation matrix.  The tests build that matrix from the oracle (by smoothing unit
vectors with f = 0) and independently from its definition as a sequence of block updates of
the assembled matrix M (M e = A e_S + B e_N + C e_E + D e_W - S e): a block P of cells updated
together solves its own rows exactly, e_P <- -M_PP^{-1} M_{P,rest} e_rest, and the blocks of one
phase of the parallel ordering all read the values from the start of the phase.
"""
import numpy as np
import pytest
from scipy.linalg import solve

import oracle as O
from oracle import lfa


def rand_coef(n, m, seed, spread=3.0, extra=0.05):
    rng = np.random.default_rng(seed)
    K = {k: np.exp(rng.normal(0, spread / 2, (n, m))) for k in "ABCD"}
    K["A"][-1, :] = 0; K["B"][0, :] = 0; K["C"][:, -1] = 0; K["D"][:, 0] = 0
    K["S"] = K["A"] + K["B"] + K["C"] + K["D"] + extra
    K["f"] = rng.normal(size=(n, m))
    return K


def assemble(K):
    n, m = K["S"].shape
    N = n * m
    M = np.zeros((N, N))
    for i in range(n):
        for j in range(m):
            q = i * m + j
            M[q, q] = -K["S"][i, j]
            if i + 1 < n: M[q, q + m] = K["A"][i, j]
            if i > 0: M[q, q - m] = K["B"][i, j]
            if j + 1 < m: M[q, q + 1] = K["C"][i, j]
            if j > 0: M[q, q - 1] = K["D"][i, j]
    return M


def oracle_matrix(K, kind, Sigma=2.0):
    n, m = K["S"].shape
    N = n * m
    Kz = dict(K); Kz["f"] = np.zeros((n, m))
    T = np.zeros((N, N))
    for q in range(N):
        e = np.zeros(N); e[q] = 1
        T[:, q] = O.smooth_given(Kz, e.reshape(n, m), Sigma, kind).ravel()
    return T


def runs(flags):
    out, t = [], 0
    while t < len(flags):
        if flags[t]:
            a = t
            while t < len(flags) and flags[t]:
                t += 1
            out.append((a, t))
        else:
            t += 1
    return out


def block_matrix(M, phases, N):
    T = np.eye(N)
    for blocks in phases:
        Tp = np.eye(N)
        for P in blocks:
            P = np.asarray(P)
            rest = np.setdiff1d(np.arange(N), P)
            Tp[P, :] = 0
            Tp[np.ix_(P, rest)] = -solve(M[np.ix_(P, P)], M[np.ix_(P, rest)])
        T = Tp @ T
    return T


def parallel_phases(K, Sigma=2.0, chunk=32):
    n, m = K["S"].shape
    mem = O.members(K, Sigma, chunk)
    phases = []
    for k in range(4):
        rowwise, rev = k < 2, k % 2 == 1
        for c in ((1, 0) if rev else (0, 1)):
            phases.append([[i * m + j] for i in range(n) for j in range(m)
                           if (i + j) % 2 == c and not mem[k, i, j]])
        nl, ln = (n, m) if rowwise else (m, n)
        for par in ((1, 0) if rev else (0, 1)):
            blocks = []
            for l in range(par, nl, 2):
                for lo in range(0, ln, chunk):
                    hi = min(lo + chunk, ln)
                    fl = [mem[k, l, t] if rowwise else mem[k, t, l] for t in range(lo, hi)]
                    for a, b in runs(fl):
                        blocks.append([l * m + lo + t if rowwise else (lo + t) * m + l
                                       for t in range(a, b)])
            phases.append(blocks)
    return phases


def lex_phases(K, Sigma=2.0):
    n, m = K["S"].shape
    mem = O.members(K, Sigma, 0)
    phases = []
    for k in range(4):
        rowwise, rev = k < 2, k % 2 == 1
        nl, ln = (n, m) if rowwise else (m, n)
        done = set()
        for lc in range(nl):
            l = nl - 1 - lc if rev else lc
            fl = [mem[k, l, t] if rowwise else mem[k, t, l] for t in range(ln)]
            seg = {}
            for a, b in runs(fl):
                for t in range(a, b):
                    seg[t] = (a, b)
            for tc in range(ln):
                t = ln - 1 - tc if rev else tc
                q = l * m + t if rowwise else t * m + l
                if t in seg:
                    if (l,) + seg[t] in done:
                        continue
                    done.add((l,) + seg[t])
                    a, b = seg[t]
                    phases.append([[l * m + s if rowwise else s * m + l for s in range(a, b)]])
                else:
                    phases.append([[q]])
        done.clear()
    return phases


@pytest.mark.parametrize("n,m,seed", [(6, 70, 0), (70, 5, 1), (9, 11, 2)])
def test_parallel_hybrid_smoother_matches_block_definition(n, m, seed):
    K = rand_coef(n, m, seed)
    mem = O.members(K, 2.0, 32)
    assert mem.any(axis=(1, 2)).all()               # every sweep has groups
    T = oracle_matrix(K, 0)
    Tref = block_matrix(assemble(K), parallel_phases(K), n * m)
    assert np.allclose(T, Tref, atol=1e-12, rtol=0)


@pytest.mark.parametrize("n,m,seed", [(6, 40, 3), (9, 11, 4)])
def test_lexicographic_hybrid_smoother_matches_block_definition(n, m, seed):
    K = rand_coef(n, m, seed)
    T = oracle_matrix(K, 1)
    Tref = block_matrix(assemble(K), lex_phases(K), n * m)
    assert np.allclose(T, Tref, atol=1e-12, rtol=0)


def test_gsline_matches_block_definition():
    K = rand_coef(7, 6, 5)
    n, m = 7, 6
    T = oracle_matrix(K, 2)
    phases = [[[i * m + j for i in range(n)]] for j in range(m)]
    assert np.allclose(T, block_matrix(assemble(K), phases, n * m), atol=1e-12)


def _zebra_phases(n, m):
    return [[[i * m + j for i in range(n)] for j in range(par, m, 2)] for par in (0, 1)]


def _hs1_block(K, i, j, lag, Sigma=2.0):
    n, m = K["S"].shape
    cells = [i * m + j]
    for t, (di, dj) in enumerate(((1, 0), (-1, 0), (0, 1), (0, -1))):
        ii, jj = i + di, j + dj
        if t != lag and 0 <= ii < n and 0 <= jj < m:
            cells.append(ii * m + jj)
    return cells


def _cls(K, i, j, Sigma=2.0):
    n, m = K["S"].shape
    return O.classify(K["A"][i, j], K["B"][i, j], K["C"][i, j], K["D"][i, j],
                      (i + 1 < n, i > 0, j + 1 < m, j > 0), Sigma)


def test_gsline_zebra_matches_block_definition():
    n, m = 7, 9
    K = rand_coef(n, m, 15)
    T = oracle_matrix(K, 3)
    assert np.allclose(T, block_matrix(assemble(K), _zebra_phases(n, m), n * m), atol=1e-12)


@pytest.mark.parametrize("n,m,seed", [(7, 8, 16), (9, 6, 17)])
def test_hybrid_smoother_1_lexicographic_matches_block_definition(n, m, seed):
    K = rand_coef(n, m, seed)
    D = [(i, j, _cls(K, i, j)) for i in range(n) for j in range(m) if _cls(K, i, j) >= 0]
    assert len(D) > 5
    phases = [[[i * m + j for i in range(n)]] for j in range(m)]
    phases += [[_hs1_block(K, i, j, c)] for i, j, c in D]
    T = oracle_matrix(K, 4)
    assert np.allclose(T, block_matrix(assemble(K), phases, n * m), atol=1e-11)


@pytest.mark.parametrize("n,m,seed", [(9, 10, 18), (11, 7, 19)])
def test_hybrid_smoother_1_parallel_matches_block_definition(n, m, seed):
    K = rand_coef(n, m, seed)
    phases = _zebra_phases(n, m)
    for c in range(16):
        blocks = [_hs1_block(K, i, j, _cls(K, i, j)) for i in range(c // 4, n, 4)
                  for j in range(c % 4, m, 4) if _cls(K, i, j) >= 0]
        phases.append(blocks)
    assert sum(len(b) for b in phases[2:]) > 5
    T = oracle_matrix(K, 5)
    assert np.allclose(T, block_matrix(assemble(K), phases, n * m), atol=1e-11)


def test_smoothers_converge_to_the_direct_solution():
    K = rand_coef(12, 10, 6, spread=2.0, extra=0.5)
    M = assemble(K)
    x = solve(M, K["f"].ravel())                     # M phi = f
    for kind in (0, 1, 2, 3, 4, 5):
        phi = np.zeros((12, 10))
        for _ in range(200):
            phi = O.smooth_given(K, phi, 2.0, kind)
        assert np.allclose(phi.ravel(), x, atol=1e-10)


def test_member_groups_by_hand():
    # one row (the middle of 3) of 70 cells; starred for sweep A where A is the smallest by > 2x
    n, m = 3, 70
    K = {k: np.ones((n, m)) for k in "ABCD"}
    stars = [3, 10, 11, 12, 31, 32, 45, 69]
    for t in stars:
        K["A"][1, t] = 0.1
    K["A"][-1, :] = 0; K["B"][0, :] = 0; K["C"][:, -1] = 0; K["D"][:, 0] = 0
    mem = O.members(K, 2.0, 32)[0]
    got = set(np.nonzero(mem[1])[0])
    # singletons take the next cell, or the previous one at the end of a 32-cell piece / line
    assert got == {3, 4, 10, 11, 12, 30, 31, 32, 33, 45, 46, 68, 69}
    whole = set(np.nonzero(O.members(K, 2.0, 0)[0][1])[0])
    assert whole == {3, 4, 10, 11, 12, 31, 32, 45, 46, 68, 69}   # 31, 32 are one run on a whole line
    # boundary rows: B face missing on row 0, A face missing on row 2 -> those cells' own classes
    assert not mem[0].any() and not mem[2].any()


@pytest.mark.parametrize("alpha", [(0.9, 2.2), (np.pi / 2, 0.3), (-2.5, 1.7), (3.0, -0.4)])
def test_lexicographic_hybrid_smoother_amplifies_modes_as_lfa(alpha):
    # With equal coefficients there are no jumps and one outer iteration of the lexicographic
    # smoother is four lexicographic GS sweeps: two with B, D new (orders A and C) and two with
    # A, C new (orders B and D).  Far from the grid edges a Fourier mode is multiplied by the
    # product of the four LFA factors of Sec. 3.4.
    n = 120
    a1, a2 = alpha
    K = {k: np.ones((n, n)) for k in "ABCD"}
    K["A"][-1, :] = 0; K["B"][0, :] = 0; K["C"][:, -1] = 0; K["D"][:, 0] = 0
    K["S"] = np.full((n, n), 4.0)
    K["f"] = np.zeros((n, n))
    i, j = np.mgrid[0:n, 0:n].astype(float)
    ph = a1 * i + a2 * j
    re = O.smooth_given(K, np.cos(ph), 2.0, 1)
    im = O.smooth_given(K, np.sin(ph), 2.0, 1)
    ratio = (re + 1j * im) / np.exp(1j * ph)
    c = ratio[50:70, 50:70]
    gA = lfa.mode_factor((1, 1, 1, 1), "AC", np.array(a1), np.array(a2))
    gB = lfa.mode_factor((1, 1, 1, 1), "BD", np.array(a1), np.array(a2))
    assert np.allclose(c, gA ** 2 * gB ** 2, atol=1e-8)
