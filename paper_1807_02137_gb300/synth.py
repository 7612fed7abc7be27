"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

The paper evaluates on real photographs and clinical scans (Sec. 5, Fig. 6 "Problems 1-3",
and the image of Fig. 1(a)) that are not distributed with it.  These generators build
stand-ins with the same structure: piecewise-smooth objects on a background, additive
Gaussian noise and a handful of user marker points inside one object (Sec. 2.2, the marker
set S).  Nothing here computes any part of the segmentation method; both the CUDA path and
the oracle receive exactly these arrays.

Coordinates: an image is an (n, m) array indexed [i, j] = [row, column]; a marker is a pair
(x, y) = (column, row) in pixel units, pixel centres at integer positions.
"""
from __future__ import annotations

import numpy as np

__all__ = ["disc_square", "ellipses", "ellipses_device", "Workload", "workload"]


def disc_square(n: int = 128, noise: float = 0.05, seed: int = 0, dtype=np.float64):
    """Two objects on a flat background: the small FP64 test case.

    Background 0.2; disc of radius 30 centred at (row 64, col 42) with value 0.8; square of
    side 40 centred at (row 64, col 100) with value 0.5; N(0, noise^2) noise.  Positions scale
    with n/128 so other sizes keep the same picture.  Markers: disc centre and +-10 px along
    the row and the column (5 points).
    """
    s = n / 128.0
    rng = np.random.Generator(np.random.PCG64(seed))
    i, j = np.mgrid[0:n, 0:n].astype(np.float64)
    img = np.full((n, n), 0.2)
    disc = (i - 64 * s) ** 2 + (j - 42 * s) ** 2 <= (30 * s) ** 2
    img[disc] = 0.8
    half = 20 * s
    sq = (np.abs(i - 64 * s) < half) & (np.abs(j - 100 * s) < half)
    img[sq] = 0.5
    if noise > 0:
        img = img + rng.normal(0.0, noise, size=img.shape)
    cx, cy = round(42 * s), round(64 * s)
    d = round(10 * s)
    markers = np.array([[cx, cy], [cx + d, cy], [cx - d, cy], [cx, cy + d], [cx, cy - d]],
                       dtype=np.float64)
    return img.astype(dtype), markers, disc


def ellipses(n: int, m: int | None = None, n_ellipses: int = 12, axes=(20.0, 200.0),
             n_markers: int = 8, noise: float = 0.05, seed: int = 1, dtype=np.float32):
    """Random ellipses with intensity ramps on a ramped background.

    Background 0.1 + 0.2 * (x cos(psi) + y sin(psi)) / max(n, m).  Each ellipse: centre uniform
    in the image, full axes uniform in ``axes`` (px), angle U(0, pi), value U(0, 1) plus an
    in-ellipse ramp of slope U(-0.1, 0.1) per semi-axis; painted in order (later ones on top).
    Markers: ``n_markers`` points uniform inside 0.8x the last-painted ellipse (it is on top, so
    every marker lies on visible pixels of the chosen object).  Noise N(0, noise^2).
    Returns (image, markers, mask_of_chosen_ellipse).
    """
    m = n if m is None else m
    rng = np.random.Generator(np.random.PCG64(seed))
    psi = rng.uniform(0, np.pi)
    img = np.empty((n, m), dtype=np.float64)
    xs = np.arange(m, dtype=np.float64)
    rows = np.arange(n, dtype=np.float64)
    img[:] = 0.1 + 0.2 * (xs[None, :] * np.cos(psi) + rows[:, None] * np.sin(psi)) / max(n, m)
    params = []
    for _ in range(n_ellipses):
        cy, cx = rng.uniform(0, n), rng.uniform(0, m)
        a, b = rng.uniform(*axes, size=2) / 2.0
        ang = rng.uniform(0, np.pi)
        val = rng.uniform(0, 1)
        s1, s2 = rng.uniform(-0.1, 0.1, size=2)
        params.append((cy, cx, a, b, ang, val, s1, s2))
    chosen = None
    for (cy, cx, a, b, ang, val, s1, s2) in params:
        # paint inside the bounding box only (keeps large images cheap)
        r = max(a, b) + 1
        i0, i1 = max(int(cy - r), 0), min(int(cy + r) + 2, n)
        j0, j1 = max(int(cx - r), 0), min(int(cx + r) + 2, m)
        if i0 >= i1 or j0 >= j1:
            continue
        ii, jj = np.mgrid[i0:i1, j0:j1].astype(np.float64)
        u = (jj - cx) * np.cos(ang) + (ii - cy) * np.sin(ang)
        v = -(jj - cx) * np.sin(ang) + (ii - cy) * np.cos(ang)
        inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        sub = img[i0:i1, j0:j1]
        sub[inside] = (val + s1 * u / a + s2 * v / b)[inside]
    chosen = params[-1]
    if noise > 0:
        img += rng.normal(0.0, noise, size=img.shape)
    cy, cx, a, b, ang, *_ = chosen
    pts = []
    while len(pts) < n_markers:
        ru, rv = rng.uniform(-1, 1, size=2)
        if ru * ru + rv * rv > 1:
            continue
        u, v = 0.8 * a * ru, 0.8 * b * rv
        x = cx + u * np.cos(ang) - v * np.sin(ang)
        y = cy + u * np.sin(ang) + v * np.cos(ang)
        if 0 <= x <= m - 1 and 0 <= y <= n - 1:
            pts.append((round(x), round(y)))
    ii, jj = np.mgrid[0:n, 0:m].astype(np.float64)
    u = (jj - cx) * np.cos(ang) + (ii - cy) * np.sin(ang)
    v = -(jj - cx) * np.sin(ang) + (ii - cy) * np.cos(ang)
    chosen_mask = (u / a) ** 2 + (v / b) ** 2 <= 1.0
    return img.astype(dtype), np.array(pts, dtype=np.float64), chosen_mask


def ellipses_device(n: int, m: int | None = None, n_ellipses: int = 200, axes=(100.0, 3000.0),
                    n_markers: int = 20, noise: float = 0.05, seed: int = 2, device="cuda"):
    """The ellipse recipe of `ellipses` drawn with torch on `device`, for images too large for
    host-side generation (25000 x 25000 and up).  Same distributions; the random stream is
    torch's (not numpy's), so the pixels differ from `ellipses` with the same seed.
    Returns (float32 tensor on device, markers as a numpy (k, 2) array)."""
    import torch

    m = n if m is None else m
    g = torch.Generator(device="cpu").manual_seed(seed)
    u = lambda lo, hi: float(lo + (hi - lo) * torch.rand(1, generator=g, dtype=torch.float64))
    psi = u(0, np.pi)
    xs = torch.arange(m, device=device, dtype=torch.float32)
    img = torch.empty((n, m), device=device, dtype=torch.float32)
    step = 4096
    for r0 in range(0, n, step):
        rows = torch.arange(r0, min(n, r0 + step), device=device, dtype=torch.float32)
        img[r0:r0 + len(rows)] = 0.1 + 0.2 * (xs[None, :] * np.cos(psi) + rows[:, None] * np.sin(psi)) / max(n, m)
    params = []
    for _ in range(n_ellipses):
        cy, cx = u(0, n), u(0, m)
        a, b = u(*axes) / 2.0, u(*axes) / 2.0
        ang, val, s1, s2 = u(0, np.pi), u(0, 1), u(-0.1, 0.1), u(-0.1, 0.1)
        params.append((cy, cx, a, b, ang, val, s1, s2))
    for (cy, cx, a, b, ang, val, s1, s2) in params:
        r = max(a, b) + 1
        i0, i1 = max(int(cy - r), 0), min(int(cy + r) + 2, n)
        j0, j1 = max(int(cx - r), 0), min(int(cx + r) + 2, m)
        if i0 >= i1 or j0 >= j1:
            continue
        ii = torch.arange(i0, i1, device=device, dtype=torch.float32)[:, None]
        jj = torch.arange(j0, j1, device=device, dtype=torch.float32)[None, :]
        uu = (jj - cx) * np.cos(ang) + (ii - cy) * np.sin(ang)
        vv = -(jj - cx) * np.sin(ang) + (ii - cy) * np.cos(ang)
        inside = (uu / a) ** 2 + (vv / b) ** 2 <= 1.0
        sub = img[i0:i1, j0:j1]
        sub[inside] = (val + s1 * uu / a + s2 * vv / b)[inside]
    if noise > 0:
        gd = torch.Generator(device=device).manual_seed(seed)
        for r0 in range(0, n, step):
            blk = img[r0:r0 + step]
            blk += noise * torch.randn(blk.shape, generator=gd, device=device, dtype=torch.float32)
    cy, cx, a, b, ang, *_ = params[-1]
    pts = []
    while len(pts) < n_markers:
        ru, rv = u(-1, 1), u(-1, 1)
        if ru * ru + rv * rv > 1:
            continue
        x = cx + 0.8 * a * ru * np.cos(ang) - 0.8 * b * rv * np.sin(ang)
        y = cy + 0.8 * a * ru * np.sin(ang) + 0.8 * b * rv * np.cos(ang)
        if 0 <= x <= m - 1 and 0 <= y <= n - 1:
            pts.append((round(x), round(y)))
    return img, np.array(pts, dtype=np.float64)


class Workload:
    """A named synthetic workload: image, markers and solver settings."""

    def __init__(self, name, image, markers, levels, tol, precision, note):
        self.name, self.image, self.markers = name, image, markers
        self.levels, self.tol, self.precision, self.note = levels, tol, precision, note

    @property
    def shape(self):
        return self.image.shape


def workload(name: str) -> Workload:
    """The synthetic workloads used by tests and the bench.

    ``disc128``: 128x128 FP64, disc + square, 5 markers, 5 levels, V(2,2), tol 1e-8.
    ``ellipse1024``: 1024x1024 FP32, 12 ellipses, 8 markers, 9 levels, tol 1e-6.
    ``ellipseN`` for other N: the same generator scaled (more ellipses for larger N).
    """
    if name == "disc128":
        img, mk, _ = disc_square(128, 0.05, 0)
        return Workload(name, img, mk, 5, 1e-8, "f64", "disc r=30 + square 40, sigma 0.05")
    if name.startswith("ellipse"):
        n = int(name[len("ellipse"):])
        if n == 1024:
            img, mk, _ = ellipses(1024, 1024, 12, (20, 200), 8, 0.05, 1)
        else:
            k = max(12, int(12 * n / 1024))
            img, mk, _ = ellipses(n, n, k, (20 * n / 1024, 200 * n / 1024), 8, 0.05, 1)
        levels = 1
        s = n
        while s // 2 >= 4 and levels < 12:
            s //= 2
            levels += 1
        return Workload(name, img, mk, levels, 1e-6, "f32", f"{n}^2 ellipses, sigma 0.05")
    raise KeyError(name)
