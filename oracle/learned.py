"""Learned per-cell relaxation weights for the point updates of Hybrid Smoother 2: a plain FP64
numpy restatement of the network, of its training loss and of the loss gradient.

TEST INFRASTRUCTURE ONLY: the checker of the CUDA library's inference and training kernels.
It shares no code with the library.  Only the tests, the package's smoke check and the bench's
CPU-baseline leg may use it.

Method.  The paper designs its smoother cell by cell from the local coefficients (Sec. 4: the
LFA rate of each pixel's stencil decides the scheme).  This extension learns a relaxation
weight omega in (0, 2) for every non-member cell from the same local stencil.  The point update
becomes phi <- phi + omega (g - phi), with g the GSLEX-I value of eq. gslexrc.

  input (5 channels per cell), from the four row-scaled face coefficients c_X of the cell
  (X = S, N, E, W; zero on a boundary face):
      x_k = c_X / sum_X c_X                        (k = 0..3 for S, N, E, W)
      x_4 = log(max c / min c over the faces that exist) / 8
  network: three 3x3 convolutions (cross-correlation, zero padding):
      5 -> 16 (ReLU) -> 16 (ReLU) -> 1,  omega = 2 sigmoid(z)
  parameters, flattened: W1 (16,5,3,3), b1 (16), W2 (16,16,3,3), b2 (16), W3 (1,16,3,3), b3 (1).

Training loss on a crop (coefficients c_X, diagonal S = sum c + 1/tau, right-hand side f and
state u recorded from a plain solve): one red and one black damped point update on the cells at
least one cell inside the crop, then
      loss = 1/2 mean over the cells at least two cells inside of r^2,  r = f - (sum_X c_X u_X - S u)
the residual of the frozen equations (the quantity the smoother must reduce).

A second loss ("hf") keeps only the high-frequency part of that residual, the part a multigrid
smoother is responsible for (the coarse grid corrects the smooth part, Sec. 3.1):
      h = 4 r - (r_S + r_N + r_E + r_W)      (the 5-point Laplacian of r; r as above, zero
                                              outside the cells at least one cell inside)
      loss = 1/2 mean over the cells at least two cells inside of h^2.
The Laplacian's Fourier symbol 4 - 2 cos t1 - 2 cos t2 vanishes on constants and is largest (8)
on the checkerboard mode, so the loss weighs each residual mode by the square of that symbol.
"""
from __future__ import annotations

import numpy as np

C_IN, C_HID = 5, 16
SHAPES = [(C_HID, C_IN, 3, 3), (C_HID,), (C_HID, C_HID, 3, 3), (C_HID,), (1, C_HID, 3, 3), (1,)]
NPARAM = int(sum(np.prod(s) for s in SHAPES))     # 3201


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == NPARAM
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(cS, cN, cE, cW):
    """The 5 input channels of every cell (see the module docstring)."""
    c = np.stack([cS, cN, cE, cW]).astype(np.float64)
    tot = c.sum(axis=0)
    x = np.zeros((C_IN,) + cS.shape)
    x[:4] = c / np.where(tot > 0, tot, 1.0)
    has = c > 0
    mx = np.where(has, c, -np.inf).max(axis=0)
    mn = np.where(has, c, np.inf).min(axis=0)
    ok = np.isfinite(mx) & np.isfinite(mn) & (mn > 0)
    x[4] = np.where(ok, np.log(np.where(ok, mx / np.where(ok, mn, 1.0), 1.0)) / 8.0, 0.0)
    return x


def conv3(x, W, b):
    """3x3 cross-correlation with zero padding: y[o] = b[o] + sum_i,di,dj W[o,i,di,dj] x[i, r+di-1, c+dj-1]."""
    cin, n, m = x.shape
    xp = np.zeros((cin, n + 2, m + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((W.shape[0], n, m))
    for o in range(W.shape[0]):
        acc = np.full((n, m), b[o], dtype=np.float64)
        for i in range(cin):
            for di in range(3):
                for dj in range(3):
                    acc += W[o, i, di, dj] * xp[i, di:di + n, dj:dj + m]
        y[o] = acc
    return y


def forward(theta, x, bf16=False):
    """omega (n, m) and the cached activations.  bf16: weights, inputs and hidden activations
    rounded to BF16 (the GPU inference's storage), accumulation in FP64 here."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    if bf16:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
        x = bf16_round(x)
    z1 = conv3(x, W1, b1)
    a1 = np.maximum(z1, 0.0)
    if bf16:
        a1 = bf16_round(a1)
    z2 = conv3(a1, W2, b2)
    a2 = np.maximum(z2, 0.0)
    if bf16:
        a2 = bf16_round(a2)
    z3 = conv3(a2, W3, b3)[0]
    sig = 1.0 / (1.0 + np.exp(-z3))
    return 2.0 * sig, dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, sig=sig, W=(W1, W2, W3))


def conv3_backward(x, W, dy):
    """Gradients of conv3 with respect to W, b and x, given dL/dy."""
    cin, n, m = x.shape
    xp = np.zeros((cin, n + 2, m + 2))
    xp[:, 1:-1, 1:-1] = x
    dW = np.zeros_like(W)
    db = dy.sum(axis=(1, 2))
    dxp = np.zeros_like(xp)
    for o in range(W.shape[0]):
        for i in range(cin):
            for di in range(3):
                for dj in range(3):
                    dW[o, i, di, dj] = np.sum(dy[o] * xp[i, di:di + n, dj:dj + m])
                    dxp[i, di:di + n, dj:dj + m] += W[o, i, di, dj] * dy[o]
    return dW, db, dxp[:, 1:-1, 1:-1]


def damped_rb(c, S, f, u, omega, parity0=0):
    """One red then one black damped point update on the cells at least one cell inside.
    c: (4, n, m) coefficients toward S, N, E, W; red = (i + j + parity0) even."""
    u = u.astype(np.float64).copy()
    n, m = u.shape
    ii, jj = np.mgrid[0:n, 0:m]
    inner = (ii >= 1) & (ii < n - 1) & (jj >= 1) & (jj < m - 1)
    for colour in (0, 1):
        sel = inner & (((ii + jj + parity0) % 2) == colour)
        g = np.zeros_like(u)
        g[1:-1, 1:-1] = (c[0][1:-1, 1:-1] * u[2:, 1:-1] + c[1][1:-1, 1:-1] * u[:-2, 1:-1]
                         + c[2][1:-1, 1:-1] * u[1:-1, 2:] + c[3][1:-1, 1:-1] * u[1:-1, :-2]
                         - f[1:-1, 1:-1]) / S[1:-1, 1:-1]
        u[sel] = u[sel] + omega[sel] * (g[sel] - u[sel])
    return u


def residual(c, S, f, u):
    """r = f - (sum_X c_X u_X - S u) on the cells at least one cell inside (zero elsewhere)."""
    r = np.zeros_like(u, dtype=np.float64)
    r[1:-1, 1:-1] = f[1:-1, 1:-1] - (c[0][1:-1, 1:-1] * u[2:, 1:-1] + c[1][1:-1, 1:-1] * u[:-2, 1:-1]
                                     + c[2][1:-1, 1:-1] * u[1:-1, 2:] + c[3][1:-1, 1:-1] * u[1:-1, :-2]
                                     - S[1:-1, 1:-1] * u[1:-1, 1:-1])
    return r


def loss_cells(n, m):
    ii, jj = np.mgrid[0:n, 0:m]
    return (ii >= 2) & (ii < n - 2) & (jj >= 2) & (jj < m - 2)


def high_pass(r):
    """h = 4 r - (sum of the four neighbours of r), on the cells at least one inside (the
    neighbours of the loss cells are all defined there)."""
    h = np.zeros_like(r)
    h[1:-1, 1:-1] = 4.0 * r[1:-1, 1:-1] - (r[2:, 1:-1] + r[:-2, 1:-1] + r[1:-1, 2:] + r[1:-1, :-2])
    return h


def crop_loss(theta, c, S, f, u, parity0=0, loss="full"):
    """The training loss of one crop (module docstring); loss "full" or "hf"."""
    omega, _ = forward(theta, features(*c))
    u2 = damped_rb(c, S, f, u, omega, parity0)
    r = residual(c, S, f, u2)
    if loss == "hf":
        r = high_pass(r)
    L = loss_cells(*u.shape)
    return 0.5 * np.mean(r[L] ** 2)


def crop_loss_grad(theta, c, S, f, u, parity0=0, loss="full"):
    """Loss and its gradient with respect to theta (reverse-mode, written out by hand)."""
    n, m = u.shape
    x = features(*c)
    omega, cache = forward(theta, x)
    # forward through the two colour phases, keeping the states
    ii, jj = np.mgrid[0:n, 0:m]
    inner = (ii >= 1) & (ii < n - 1) & (jj >= 1) & (jj < m - 1)
    states, gvals, sels = [u.astype(np.float64).copy()], [], []
    cur = states[0]
    for colour in (0, 1):
        sel = inner & (((ii + jj + parity0) % 2) == colour)
        g = np.zeros_like(cur)
        g[1:-1, 1:-1] = (c[0][1:-1, 1:-1] * cur[2:, 1:-1] + c[1][1:-1, 1:-1] * cur[:-2, 1:-1]
                         + c[2][1:-1, 1:-1] * cur[1:-1, 2:] + c[3][1:-1, 1:-1] * cur[1:-1, :-2]
                         - f[1:-1, 1:-1]) / S[1:-1, 1:-1]
        nxt = cur.copy()
        nxt[sel] = cur[sel] + omega[sel] * (g[sel] - cur[sel])
        gvals.append(g)
        sels.append(sel)
        states.append(nxt)
        cur = nxt
    u2 = states[2]
    r = residual(c, S, f, u2)
    L = loss_cells(n, m)
    cnt = L.sum()
    if loss == "hf":
        h = high_pass(r)
        value = 0.5 * np.sum(h[L] ** 2) / cnt
        # dL/dr through h = 4 r - sum of neighbours (the stencil is symmetric: its transpose)
        dh = np.where(L, h / cnt, 0.0)
        dr = high_pass(dh)
        ii, jj = np.mgrid[0:n, 0:m]
        dr = np.where((ii >= 1) & (ii < n - 1) & (jj >= 1) & (jj < m - 1), dr, 0.0)
    else:
        value = 0.5 * np.sum(r[L] ** 2) / cnt
        dr = np.where(L, r / cnt, 0.0)
    # dL/du2 through r = f - (sum c_X u_X - S u)
    du = np.zeros_like(u2)
    du[1:-1, 1:-1] += S[1:-1, 1:-1] * dr[1:-1, 1:-1]
    du[2:, 1:-1] -= c[0][1:-1, 1:-1] * dr[1:-1, 1:-1]
    du[:-2, 1:-1] -= c[1][1:-1, 1:-1] * dr[1:-1, 1:-1]
    du[1:-1, 2:] -= c[2][1:-1, 1:-1] * dr[1:-1, 1:-1]
    du[1:-1, :-2] -= c[3][1:-1, 1:-1] * dr[1:-1, 1:-1]
    domega = np.zeros_like(u2)
    for ph in (1, 0):
        sel, g, prev = sels[ph], gvals[ph], states[ph]
        # u_new[sel] = prev + omega (g(prev) - prev); elsewhere u_new = prev
        dnew = np.where(sel, du, 0.0)
        domega += dnew * (g - prev)
        dprev = np.where(sel, du * (1.0 - omega), du)
        t = np.where(sel, dnew * omega / S, 0.0)           # dL/dg at the updated cells
        dprev[2:, 1:-1] += c[0][1:-1, 1:-1] * t[1:-1, 1:-1]
        dprev[:-2, 1:-1] += c[1][1:-1, 1:-1] * t[1:-1, 1:-1]
        dprev[1:-1, 2:] += c[2][1:-1, 1:-1] * t[1:-1, 1:-1]
        dprev[1:-1, :-2] += c[3][1:-1, 1:-1] * t[1:-1, 1:-1]
        du = dprev
    # through omega = 2 sigmoid(z3) and the three convolutions
    sig = cache["sig"]
    dz3 = (domega * 2.0 * sig * (1.0 - sig))[None]
    W1, W2, W3 = cache["W"]
    dW3, db3, da2 = conv3_backward(cache["a2"], W3, dz3)
    dz2 = da2 * (cache["z2"] > 0)
    dW2, db2, da1 = conv3_backward(cache["a1"], W2, dz2)
    dz1 = da1 * (cache["z1"] > 0)
    dW1, db1, _ = conv3_backward(cache["x"], W1, dz1)
    grad = np.concatenate([a.ravel() for a in (dW1, db1, dW2, db2, dW3, db3)])
    return value, grad


def adam_step(theta, grad, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015); state = (m, v, t)."""
    m, v, t = state
    t += 1
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), (m, v, t)
