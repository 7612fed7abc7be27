"""Local Fourier Analysis smoothing rates (test infrastructure only).

Restates the smoothing-rate formulas of Sec. 3.4 of the paper ("Local Fourier Analysis of
Algorithm 1"): the error of a frozen-coefficient 5-point scheme is expanded in Fourier modes
exp(i (a1 i + a2 j)), and the smoothing rate of a pixel is the largest amplification over the
high frequencies [-pi, pi)^2 \\ [-pi/2, pi/2)^2.  Frequencies are sampled on the paper's
discrete grid a = 2 pi theta / n, theta = -n/2 .. n/2 - 1 (n = 1024 by default, which contains
a = +-pi/2 and -pi exactly).

Which neighbour terms sit on the "new" side of the error equation decides the scheme:
  * lexicographic GS (GSLEX, error form eq. errorformpixel): new = B (north), D (west);
  * column line GS (GSLINE, eq. errorform / gslinelfa): new = A, B, D, old = C;
  * the hybrid schemes that lag one coefficient k (Sec. 4.1.3 and 4.3): old = {k}, new = rest;
  * the adapted_1 schemes of Sec. 4.1 (e.g. eq. smratecase1): old = the lagged set.
"""
from __future__ import annotations

import numpy as np

__all__ = ["high_freq_grid", "rate", "rate_lex", "rate_line", "rate_lag", "rate_lagset",
           "mode_factor", "iterations_to_reduce"]

_NAMES = "ABCD"


def high_freq_grid(n: int = 1024):
    """(a1, a2) arrays of the high-frequency set on the paper's discrete theta grid."""
    th = np.arange(-n // 2, n // 2)
    a = 2 * np.pi * th / n
    a1, a2 = np.meshgrid(a, a, indexing="ij")
    low = (a1 >= -np.pi / 2) & (a1 < np.pi / 2) & (a2 >= -np.pi / 2) & (a2 < np.pi / 2)
    return a1[~low], a2[~low]


def _phases(a1, a2):
    # Mode value at each neighbour relative to the cell: A=(i+1,j), B=(i-1,j), C=(i,j+1), D=(i,j-1)
    return {"A": np.exp(1j * a1), "B": np.exp(-1j * a1), "C": np.exp(1j * a2), "D": np.exp(-1j * a2)}


def mode_factor(coef, old, a1, a2, S=None):
    """Complex amplification of mode (a1, a2) for a scheme whose `old` neighbours are lagged.

    The error equation sum_{k in new} K_k e_k^{new} - S e^{new} = - sum_{k in old} K_k e_k^{old}
    gives e^{new} / e^{old} = - sum_old K_k ph_k / (sum_new K_k ph_k - S).
    """
    A, B, C, D = coef
    K = dict(zip(_NAMES, (A, B, C, D)))
    S = A + B + C + D if S is None else S
    ph = _phases(a1, a2)
    num = sum(K[k] * ph[k] for k in old) if old else 0 * a1
    den = sum(K[k] * ph[k] for k in _NAMES if k not in old) - S
    return -num / den


def rate(coef, old, n: int = 1024, S=None):
    """Smoothing rate: max over the high-frequency grid of |mode_factor|."""
    a1, a2 = high_freq_grid(n)
    return float(np.max(np.abs(mode_factor(coef, old, a1, a2, S))))


def rate_lex(coef, n: int = 1024):
    """GSLEX-I / NEWT (Sec. 3.4, first smoothing-rate formula): old = A, C."""
    return rate(coef, "AC", n)


def rate_line(coef, n: int = 1024):
    """GSLINE-I (eq. gslinelfa): old = C."""
    return rate(coef, "C", n)


def rate_lag(coef, k: str, n: int = 1024):
    """Hybrid scheme lagging only coefficient k (Sec. 4.1.3, 'lag only the smallest')."""
    return rate(coef, k, n)


def rate_lagset(coef, lagged: str, n: int = 1024):
    """adapted_1 scheme lagging a set of coefficients (Sec. 4.1.1, e.g. eq. smratecase1)."""
    return rate(coef, lagged, n)


def iterations_to_reduce(mu: float, factor: float = 0.1) -> int:
    """Smallest k with mu^k <= factor (the paper's 'iterations to reduce high-frequency errors
    by 90%')."""
    return int(np.ceil(np.log(factor) / np.log(mu)))
