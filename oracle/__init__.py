"""FP64 CPU oracle for the selective-segmentation multigrid method (test infrastructure only).

The oracle is a plain C restatement of the paper's discretisation, grid transfers, smoothers,
FAS V-cycle and outer driver (``oracle.c``), plus the Local Fourier Analysis tooling
(``lfa.py``).  It is the independent checker of the CUDA library: it shares no code with it,
and only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may use it.

``build()`` compiles ``oracle.c`` with gcc into ``oracle/_build/liboracle.so`` (the checker, one
core).  ``build(openmp=True)`` compiles the same file with ``-fopenmp`` into ``liboracle_omp.so``:
its loops marked independent run on all host cores with bitwise the same results.  It is used only
to time the oracle on all cores (``Solver(..., openmp=True)``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lib = None
_lib_omp = None
_lock = threading.Lock()


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle shared library (plain C, -O2, no fast-math; -fopenmp for the all-core
    timing build)."""
    out = _OUT_OMP if openmp else _OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *flags, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class Params(C.Structure):
    """Mirror of ``or_params`` (oracle.c)."""

    _fields_ = [
        ("model", C.c_int), ("mu", C.c_double), ("lambda1", C.c_double), ("lambda2", C.c_double),
        ("theta", C.c_double), ("nu", C.c_double), ("eps", C.c_double), ("beta", C.c_double),
        ("beta_edge", C.c_double), ("sigma_blur", C.c_double), ("sigma_d", C.c_double),
        ("Sigma", C.c_double), ("inv_tau", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
        ("levels", C.c_int), ("smoother", C.c_int), ("coarse_maxit", C.c_int),
        ("coarse_tol", C.c_double), ("coarse_solver", C.c_int), ("aos_dt", C.c_double),
    ]


def params(n=None, m=None, **kw) -> Params:
    """Default parameters: the Spencer-Chen model with mu = 1, lambda1 = lambda2 = 10,
    theta = 1, eps = 1, beta = 1e-6, sigma_blur = 1, beta_edge = 1, Sigma = 2, tau = 1,
    V(2,2), Hybrid Smoother 2 (parallel ordering).  sigma_d defaults to 0.05 max(n, m)."""
    sd = 0.05 * max(n or 128, m or n or 128)
    d = dict(model=0, mu=1.0, lambda1=10.0, lambda2=10.0, theta=1.0, nu=1.0, eps=1.0, beta=1e-6,
             beta_edge=1.0, sigma_blur=1.0, sigma_d=sd, Sigma=2.0, inv_tau=1.0, nu1=2,
             nu2=2, levels=5, smoother=0, coarse_maxit=100, coarse_tol=1e-13, coarse_solver=0,
             aos_dt=10.0)
    if "tau" in kw:
        t = kw.pop("tau")
        kw["inv_tau"] = 0.0 if t is None or t == float("inf") else 1.0 / t
    d.update(kw)
    return Params(**d)


def lib(openmp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if openmp else _lib) is None:
            L = C.CDLL(build(openmp=openmp))
            D = C.POINTER(C.c_double)
            I = C.POINTER(C.c_int)
            P = C.POINTER(Params)
            sig = {
                "or_gauss_blur": ([D, C.c_int, C.c_int, C.c_double, D], None),
                "or_edge_detector": ([D, C.c_int, C.c_int, C.c_double, D], None),
                "or_distance": ([C.c_int, C.c_int, D, D, C.c_int, C.c_double, D], None),
                "or_initial_phi": ([C.c_int, C.c_int, D, D, C.c_int, C.c_double, D, D], C.c_int),
                "or_region_means": ([D, D, C.c_int, C.c_int, C.c_double, D, D], None),
                "or_restrict": ([D, C.c_int, C.c_int, D], None),
                "or_interpolate_add": ([D, C.c_int, C.c_int, D, C.c_int, C.c_int], None),
                "or_apply_L": ([D, D, D, C.c_int, C.c_int, C.c_double, P, C.c_double, C.c_double, D], None),
                "or_fitting": ([D, D, D, C.c_int, C.c_int, C.c_double, C.c_double, P, D], None),
                "or_classify": ([C.c_double] * 4 + [C.c_int] * 4 + [C.c_double], C.c_int),
                "or_coarse_solve": ([D, D, D, D, C.c_int, C.c_int, C.c_double, P, C.c_double, C.c_double], C.c_int),
                "or_create": ([D, C.c_int, C.c_int, D, D, C.c_int, P], C.c_void_p),
                "or_destroy": ([C.c_void_p], None),
                "or_begin_step": ([C.c_void_p], C.c_double),
                "or_vcycle": ([C.c_void_p], C.c_double),
                "or_end_step": ([C.c_void_p], C.c_double),
                "or_get_phi": ([C.c_void_p, D], None),
                "or_set_phi": ([C.c_void_p, D], None),
                "or_get_level": ([C.c_void_p, C.c_int, C.c_int, D], None),
                "or_get_scalars": ([C.c_void_p, D], None),
                "or_set_c": ([C.c_void_p, C.c_double, C.c_double], None),
                "or_set_inv_tau": ([C.c_void_p, C.c_double], None),
                "or_frozen_coeffs": ([D, D, D, D, C.c_int, C.c_int, C.c_double, P, C.c_double, C.c_double, D], None),
                "or_smooth_given": ([D, C.c_int, C.c_int, C.c_double, C.c_int, D], None),
                "or_members": ([D, C.c_int, C.c_int, C.c_double, C.c_int, I], None),
                "or_aos_iteration": ([D, D, D, D, C.c_int, C.c_int, C.c_double, P, C.c_double, C.c_double,
                                      C.c_double], None),
                "or_solver_aos": ([C.c_void_p, C.c_double, C.c_int, C.c_double, D], C.c_int),
                "or_set_omega": ([C.c_void_p, C.c_int, D], None),
                "or_smooth_given_omega": ([D, D, C.c_int, C.c_int, C.c_double, C.c_int, D], None),
                "or_energy": ([D, D, D, D, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, P], C.c_double),
                "or_solver_energy": ([C.c_void_p], C.c_double),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            if openmp:
                _lib_omp = L
            else:
                _lib = L
    return _lib_omp if openmp else _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


# ---- thin wrappers over the C routines -----------------------------------------------------

def gauss_blur(z, sigma=1.0):
    z, pz = _d(z)
    out = np.empty_like(z)
    lib().or_gauss_blur(pz, z.shape[0], z.shape[1], sigma, _d(out)[1])
    return out


def edge_detector(zb, beta_edge=1.0):
    zb, p = _d(zb)
    out = np.empty_like(zb)
    lib().or_edge_detector(p, zb.shape[0], zb.shape[1], beta_edge, _d(out)[1])
    return out


def distance(n, m, markers, sigma_d):
    mk = np.asarray(markers, dtype=np.float64).reshape(-1, 2)
    mx, px = _d(mk[:, 0].copy())
    my, py = _d(mk[:, 1].copy())
    out = np.empty((n, m))
    lib().or_distance(n, m, px, py, len(mk), sigma_d, _d(out)[1])
    return out


def initial_phi(n, m, markers, r0=None):
    mk = np.asarray(markers, dtype=np.float64).reshape(-1, 2)
    mx, px = _d(mk[:, 0].copy())
    my, py = _d(mk[:, 1].copy())
    out = np.empty((n, m))
    area = np.zeros(1)
    r0 = 0.05 * max(n, m) if r0 is None else r0
    h = lib().or_initial_phi(n, m, px, py, len(mk), r0, _d(out)[1], _d(area)[1])
    return out, float(area[0]), h


def aos_iteration(phi, w, Fn, rhs, h=1.0, p=None, n0m0=None, A1=0.0, dt=1.0):
    """One AOS iteration of the pseudo-time-step problem L(phi) = rhs (or_aos_iteration)."""
    phi, _ = _d(phi)
    out, po = _d(phi.copy())
    n, m = phi.shape
    p = p or params(n, m)
    w, pw = _d(w)
    Fn, pf = _d(Fn)
    rhs, pr = _d(rhs) if rhs is not None else (None, None)
    lib().or_aos_iteration(po, pw, pf, pr, n, m, h, C.byref(p),
                           float(n * m if n0m0 is None else n0m0), A1, dt)
    return out


def energy(phi, z, w, d, c1, c2, A1, p: Params):
    """Level-set energy of eq. scfunc / rcfunc on one grid in pixel units (or_energy)."""
    phi, pp = _d(phi)
    z, pz = _d(z)
    w, pw = _d(w)
    d, pd = _d(d)
    n, m = phi.shape
    return float(lib().or_energy(pp, pz, pw, pd, n, m, c1, c2, A1, C.byref(p)))


def region_means(phi, z, eps=1.0):
    phi, pp = _d(phi)
    z, pz = _d(z)
    c = np.zeros(2)
    lib().or_region_means(pp, pz, phi.shape[0], phi.shape[1], eps,
                          c[0:1].ctypes.data_as(C.POINTER(C.c_double)),
                          c[1:2].ctypes.data_as(C.POINTER(C.c_double)))
    return float(c[0]), float(c[1])


def restrict(f):
    f, p = _d(f)
    out = np.empty((f.shape[0] // 2, f.shape[1] // 2))
    lib().or_restrict(p, f.shape[0], f.shape[1], _d(out)[1])
    return out


def interpolate_add(e, f):
    e, pe = _d(e)
    out = np.array(f, dtype=np.float64, copy=True)
    lib().or_interpolate_add(pe, e.shape[0], e.shape[1], _d(out)[1], out.shape[0], out.shape[1])
    return out


def apply_L(phi, w, Fn, h=1.0, p=None, n0m0=None, A1=0.0):
    phi, pp = _d(phi)
    w, pw = _d(w)
    Fn, pf = _d(Fn)
    p = p or params(*phi.shape)
    out = np.empty_like(phi)
    n0m0 = float(phi.size) if n0m0 is None else n0m0
    lib().or_apply_L(pp, pw, pf, phi.shape[0], phi.shape[1], h, C.byref(p), n0m0, A1, _d(out)[1])
    return out


def fitting(z, d, phin, c1, c2, p):
    z, pz = _d(z)
    d, pd = _d(d)
    phin, pn = _d(phin)
    out = np.empty_like(z)
    lib().or_fitting(pz, pd, pn, z.shape[0], z.shape[1], c1, c2, C.byref(p), _d(out)[1])
    return out


def frozen_coeffs(phi, w, Fn, rhs=None, h=1.0, p=None, n0m0=None, A1=0.0):
    """Returns dict with A, B, C, D, S, f, delta (each n x m)."""
    phi, pp = _d(phi)
    w, pw = _d(w)
    Fn, pf = _d(Fn)
    prhs = None
    if rhs is not None:
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        prhs = rhs.ctypes.data_as(C.POINTER(C.c_double))
    p = p or params(*phi.shape)
    n, m = phi.shape
    out = np.empty((7, n, m))
    n0m0 = float(phi.size) if n0m0 is None else n0m0
    lib().or_frozen_coeffs(pp, pw, pf, prhs, n, m, h, C.byref(p), n0m0, A1, _d(out)[1])
    return dict(zip("A B C D S f delta".split(), out))


def smooth_given(coef, phi, Sigma=2.0, kind=0):
    """One outer iteration of a smoother with explicit frozen coefficients.
    coef: dict or array (6, n, m) with A, B, C, D, S, f."""
    if isinstance(coef, dict):
        coef = np.stack([coef[k] for k in "A B C D S f".split()])
    coef, pc = _d(coef)
    out, po = _d(np.array(phi, dtype=np.float64, copy=True))
    lib().or_smooth_given(pc, phi.shape[0], phi.shape[1], Sigma, kind, po)
    return out


def smooth_given_omega(coef, omega, phi, Sigma=2.0, kind=0):
    """smooth_given with per-cell relaxation weights of the point updates."""
    if isinstance(coef, dict):
        coef = np.stack([coef[k] for k in "A B C D S f".split()])
    coef, pc = _d(coef)
    om, po_ = _d(omega)
    out, po = _d(np.array(phi, dtype=np.float64, copy=True))
    lib().or_smooth_given_omega(pc, po_, phi.shape[0], phi.shape[1], Sigma, kind, po)
    return out


def members(coef, Sigma=2.0, piece=32):
    """Member flags (4, n, m) of the four sweeps; piece <= 0 means whole lines."""
    if isinstance(coef, dict):
        coef = np.stack([coef[k] for k in "A B C D".split()] + [coef["A"]] * 2)
    coef, pc = _d(coef)
    n, m = coef.shape[1:]
    out = np.zeros((4, n, m), dtype=np.int32)
    lib().or_members(pc, n, m, Sigma, piece, out.ctypes.data_as(C.POINTER(C.c_int)))
    return out.astype(bool)


def classify(A, B, Cc, D, has=(1, 1, 1, 1), Sigma=2.0):
    return lib().or_classify(A, B, Cc, D, *has, Sigma)


def coarse_solve(phi, w, Fn, rhs, h=1.0, p=None, n0m0=None, A1=0.0):
    phi, _ = _d(phi)
    out, po = _d(phi.copy())
    w, pw = _d(w)
    Fn, pf = _d(Fn)
    rhs, pr = _d(rhs)
    p = p or params(*phi.shape)
    n0m0 = float(phi.size) if n0m0 is None else n0m0
    it = lib().or_coarse_solve(po, pw, pf, pr, phi.shape[0], phi.shape[1], h, C.byref(p), n0m0, A1)
    return out, it


class Solver:
    """The oracle's FAS solver over one image (create / begin_step / vcycle / end_step)."""

    def __init__(self, image, markers, p: Params, openmp: bool = False):
        img, pi = _d(image)
        mk = np.asarray(markers, dtype=np.float64).reshape(-1, 2)
        self._mx, px = _d(mk[:, 0].copy())
        self._my, py = _d(mk[:, 1].copy())
        self.n, self.m = img.shape
        self.p = p
        self._L = lib(openmp)
        self._h = self._L.or_create(pi, self.n, self.m, px, py, len(mk), C.byref(p))

    def close(self):
        if self._h:
            self._L.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def begin_step(self) -> float:
        return self._L.or_begin_step(self._h)

    def vcycle(self) -> float:
        return self._L.or_vcycle(self._h)

    def end_step(self) -> float:
        return self._L.or_end_step(self._h)

    @property
    def phi(self):
        out = np.empty((self.n, self.m))
        self._L.or_get_phi(self._h, _d(out)[1])
        return out

    @phi.setter
    def phi(self, v):
        v, p = _d(v)
        assert v.shape == (self.n, self.m)
        self._L.or_set_phi(self._h, p)

    def level(self, l, which):
        names = ["phi", "w", "z", "d", "Fn", "rhs", "tmp"]
        idx = names.index(which)
        n, m = self.n, self.m
        for _ in range(l):
            n, m = n // 2, m // 2
        out = np.empty((n, m))
        self._L.or_get_level(self._h, l, idx, _d(out)[1])
        return out

    def scalars(self):
        out = np.zeros(5)
        self._L.or_get_scalars(self._h, _d(out)[1])
        return dict(c1=out[0], c2=out[1], A1=out[2], res0=out[3], picard=int(out[4]))

    def set_c(self, c1, c2):
        self._L.or_set_c(self._h, c1, c2)

    def aos(self, dt, max_iter, eta):
        """AOS iterations on the finest grid until the relative change < eta (or_solver_aos).
        Returns (iterations, rho)."""
        r = np.zeros(1)
        it = self._L.or_solver_aos(self._h, dt, max_iter, eta, _d(r)[1])
        return it, float(r[0])

    def set_omega(self, l, omega):
        """Relaxation weights of the point updates on grid l (None: plain smoother)."""
        if omega is None:
            self._L.or_set_omega(self._h, l, None)
        else:
            w, pw = _d(omega)
            self._L.or_set_omega(self._h, l, pw)

    def energy(self) -> float:
        """Energy of the current finest-grid phi with the current c1, c2 (or_solver_energy)."""
        return float(self._L.or_solver_energy(self._h))

    def solve_step(self, tol, max_cycles=50):
        """One pseudo-time step: V-cycles until rho <= tol.  Returns list of rho."""
        self.begin_step()
        hist = []
        for _ in range(max_cycles):
            r = self.vcycle()
            hist.append(r)
            if r <= tol:
                break
        return hist

    def set_tau(self, tau):
        """tau of the following pseudo-time steps (None or inf: the stationary equation)."""
        self._L.or_set_inv_tau(self._h, 0.0 if tau is None or tau == float("inf") else 1.0 / tau)

    def solve_step_controlled(self, tau, tol, max_cycles=40, stall_ratio=0.6, max_halvings=10):
        """One pseudo-time step under the step-size control of the outer driver.

        The implicit step with pseudo-time tau is a nonlinear problem of its own; its lagged-
        coefficient V-cycles (Algorithm 1 with the Sec. 4 smoother) contract well for small
        enough tau and can stall for larger tau once the level set has flat parts, where the
        coefficients w / |grad phi|_beta become very large.  The paper solves the stationary
        equation and stops on the relative change only (Sec. 5), so it has no rule for this;
        the reading taken here:
          - an attempt runs V-cycles j = 1, 2, ... until rho_j <= tol (the step is accepted);
          - it is rejected when j >= 4 and rho_j > stall_ratio * rho_{j-2} (less than a factor
            1/stall_ratio gained in two V-cycles), when rho_j is not finite or above 1e3, or when
            max_cycles V-cycles did not reach tol;
          - a rejected attempt restores phi = phi^n and the step is tried again with tau / 2, at
            most max_halvings times.
        Returns (tau, attempts): the tau of the accepted step (the next step starts from it),
        and per attempt (tau, list of rho).  Raises RuntimeError when no attempt was accepted."""
        phin = self.phi
        attempts = []
        for _ in range(max_halvings + 1):
            self.set_tau(tau)
            self.begin_step()
            hist = []
            ok = False
            for j in range(1, max_cycles + 1):
                r = self.vcycle()
                hist.append(r)
                if r <= tol:
                    ok = True
                    break
                if not np.isfinite(r) or r > 1e3:
                    break
                if j >= 4 and r > stall_ratio * hist[-3]:
                    break
            attempts.append((tau, hist))
            if ok:
                return tau, attempts
            self.phi = phin
            tau = tau / 2.0
        raise RuntimeError(f"no pseudo-time step reached rho <= {tol}: {attempts}")
