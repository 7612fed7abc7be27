"""Python binding of the C ABI in include/segmg.h (argument marshalling only).

Every step of the solver runs in the CUDA library ``_build/libsegmg.so``; this module only
converts torch tensors / numpy arrays to pointers and error codes to exceptions.  It raises
``RuntimeError`` if the library has not been built (``paper_1807_02137_gb300.build()``) or if no
CUDA device is present: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import buildlib as _build

MG_F32, MG_F64, MG_MIXED = 0, 1, 2
MG_MODEL_SC, MG_MODEL_RC = 0, 1
MG_SMOOTH_FUSED, MG_SMOOTH_PHASED, MG_SMOOTH_FUSED_VEC, MG_SMOOTH_GSLINE, MG_SMOOTH_HS1 = 0, 1, 2, 3, 4
MG_COARSE_PICARD, MG_COARSE_AOS = 0, 1
ERRORS = {0: "MG_OK", -1: "MG_ERR_ARG", -2: "MG_ERR_NAN", -3: "MG_ERR_CUDA", -4: "MG_ERR_DIVERGED",
          -5: "MG_ERR_TIMEOUT", -6: "MG_ERR_NOT_SPD", -7: "MG_ERR_NOMEM", -8: "MG_ERR_STATE"}
EXPORTS = ["mg_default_params", "mg_setup", "mg_reset", "mg_begin_step", "mg_vcycle", "mg_end_step",
           "mg_solve_step", "mg_solve", "mg_mask", "mg_get_phi", "mg_set_phi", "mg_set_regions",
           "mg_get_level", "mg_get_stats", "mg_set_wait_limit", "mg_inject_divergence", "mg_debug_status", "mg_debug_selftest", "mg_segment_host", "mg_segment_host_release", "mg_get_stream", "mg_destroy",
           "mg_strerror", "mg_last_error", "mg_time_kernels", "mg_time_residuals", "mg_time_sweeps_graph", "mg_residual_norm_noalloc", "mg_autotune", "mg_set_tile_shapes", "mg_set_bottom_kernel", "mg_set_bottom_level", "mg_set_cluster_level", "mg_energy", "mg_aos", "mg_set_learned", "mg_set_omega", "mg_learned_nparam",
           "mg_trainer_create", "mg_trainer_record", "mg_trainer_load", "mg_trainer_count", "mg_trainer_set_loss", "mg_trainer_grad",
           "mg_trainer_train", "mg_trainer_get", "mg_trainer_destroy",
           "mg_batch_setup", "mg_batch_solve_step", "mg_batch_autotune", "mg_batch_handle",
           "mg_batch_destroy"]


class Params(C.Structure):
    """Mirror of mg_params."""

    _fields_ = [
        ("model", C.c_int), ("mu", C.c_double), ("lambda1", C.c_double), ("lambda2", C.c_double),
        ("theta", C.c_double), ("nu", C.c_double), ("eps", C.c_double), ("beta", C.c_double),
        ("beta_edge", C.c_double), ("sigma_blur", C.c_double), ("sigma_d", C.c_double),
        ("Sigma", C.c_double), ("tau", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
        ("levels", C.c_int), ("precision", C.c_int), ("smoother", C.c_int),
        ("coarse_maxit", C.c_int), ("coarse_tol", C.c_double), ("use_graph", C.c_int),
        ("coarse_solver", C.c_int), ("aos_dt", C.c_double), ("stall_ratio", C.c_double),
        ("max_halvings", C.c_int),
    ]


class Stats(C.Structure):
    """Mirror of mg_stats."""

    _fields_ = [
        ("n", C.c_int), ("m", C.c_int), ("levels", C.c_int), ("precision", C.c_int),
        ("steps", C.c_int), ("cycles_step", C.c_int), ("cycles_total", C.c_int),
        ("picard_last", C.c_int), ("rho", C.c_double), ("res0", C.c_double), ("eta", C.c_double),
        ("c1", C.c_double), ("c2", C.c_double), ("A1", C.c_double), ("device_bytes", C.c_size_t),
        ("launches", C.c_longlong), ("learned_accepted", C.c_longlong), ("learned_rejected", C.c_longlong),
        ("bottom_level", C.c_int), ("cluster_level", C.c_int), ("tau", C.c_double),
        ("attempts_rejected", C.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SegmgError(RuntimeError):
    def __init__(self, code, where, detail):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({detail})")


class DebugInfo(C.Structure):
    """mg_debug_info: the device error words of the bounds-checked (MG_DEBUG) build."""
    _fields_ = [("enabled", C.c_int), ("first_site", C.c_int), ("first_index", C.c_longlong),
                ("sites", C.c_ulonglong), ("count", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path():
    """The library this process loads: the bounds-checked build when SEGMG_DEBUG=1."""
    return _build.LIB_DEBUG if os.environ.get("SEGMG_DEBUG") == "1" else _build.LIB


def lib():
    """Loads the built library (no build here: a missing library is an error)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run paper_1807_02137_gb300.build())")
        L = C.CDLL(path)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        P = C.POINTER(Params)
        D = C.POINTER(C.c_double)
        sig = {
            "mg_default_params": ([P, i, i], i),
            "mg_setup": ([C.POINTER(vp), vp, i, i, D, i, P, vp, vp], i),
            "mg_reset": ([vp, vp, D, i], i),
            "mg_begin_step": ([vp, D], i),
            "mg_vcycle": ([vp, D], i),
            "mg_end_step": ([vp, D], i),
            "mg_solve_step": ([vp, d, i, C.POINTER(i), D], i),
            "mg_solve": ([vp, d, i, d, i, C.POINTER(i)], i),
            "mg_mask": ([vp, vp], i),
            "mg_get_phi": ([vp, vp], i),
            "mg_set_phi": ([vp, vp], i),
            "mg_set_regions": ([vp, d, d], i),
            "mg_get_level": ([vp, i, i, vp], i),
            "mg_get_stats": ([vp, C.POINTER(Stats)], i),
            "mg_set_wait_limit": ([vp, C.c_longlong], i),
            "mg_inject_divergence": ([vp, i], i),
            "mg_debug_status": ([C.POINTER(DebugInfo), i], i),
            "mg_debug_selftest": ([], i),
            "mg_segment_host": ([vp, i, i, D, i, P, d, i, d, i, vp, vp, C.POINTER(Stats)], i),
            "mg_segment_host_release": ([], None),
            "mg_get_stream": ([vp], vp),
            "mg_time_kernels": ([vp, i, i, D], i),
            "mg_time_residuals": ([vp, i, i, D], i),
            "mg_time_sweeps_graph": ([vp, i, i, D], i),
            "mg_residual_norm_noalloc": ([vp, vp, vp, i, i, P, D, vp], i),
            "mg_autotune": ([vp, i, C.POINTER(i)], i),
            "mg_set_tile_shapes": ([vp, C.POINTER(i)], i),
            "mg_set_bottom_kernel": ([vp, i, C.POINTER(i)], i),
            "mg_set_bottom_level": ([vp, i], i),
            "mg_set_cluster_level": ([vp, i], i),
            "mg_energy": ([vp, C.POINTER(C.c_double)], i),
            "mg_aos": ([vp, C.c_double, i, C.c_double, C.POINTER(i), C.POINTER(C.c_double)], i),
            "mg_set_learned": ([vp, C.POINTER(C.c_float), i, i], i),
            "mg_set_omega": ([vp, i, vp], i),
            "mg_learned_nparam": ([], i),
            "mg_trainer_create": ([C.POINTER(vp), i, i, C.c_ulonglong, C.POINTER(C.c_float)], i),
            "mg_trainer_record": ([vp, vp, i], i),
            "mg_trainer_load": ([vp, C.POINTER(C.c_float), i], i),
            "mg_trainer_count": ([vp], i),
            "mg_trainer_set_loss": ([vp, i], i),
            "mg_trainer_grad": ([vp, C.POINTER(i), i, C.POINTER(C.c_float), C.POINTER(C.c_double)], i),
            "mg_trainer_train": ([vp, i, i, C.c_double, C.POINTER(C.c_double)], i),
            "mg_trainer_get": ([vp, C.POINTER(C.c_float)], i),
            "mg_trainer_destroy": ([vp], None),
            "mg_batch_setup": ([C.POINTER(vp), i, C.POINTER(vp), C.POINTER(i), C.POINTER(i),
                                C.POINTER(D), C.POINTER(i), P, vp], i),
            "mg_batch_solve_step": ([vp, d, i, C.POINTER(i), D], i),
            "mg_batch_autotune": ([vp, i], i),
            "mg_batch_handle": ([vp, i], vp),
            "mg_batch_destroy": ([vp], None),
            "mg_destroy": ([vp], None),
            "mg_strerror": ([i], C.c_char_p),
            "mg_last_error": ([], C.c_char_p),
        }
        for name, (a, r) in sig.items():
            f = getattr(L, name)
            f.argtypes, f.restype = a, r
        _lib = L
    return _lib


def _check(rc, where):
    if rc != 0:
        raise SegmgError(rc, where, lib().mg_last_error().decode())


def debug_status(clear=False) -> dict:
    """mg_debug_status: out-of-range indices the bounds-checked build recorded (enabled = 0 in
    the default build); clear=True zeroes the device words after reading them."""
    d = DebugInfo()
    _check(lib().mg_debug_status(C.byref(d), 1 if clear else 0), "mg_debug_status")
    return d.as_dict()


def debug_selftest():
    """mg_debug_selftest: records one out-of-range index (no memory access) in the bounds-checked
    build, to test the reporting path; nothing in the default build."""
    _check(lib().mg_debug_selftest(), "mg_debug_selftest")


def default_params(n, m, **kw) -> Params:
    """mg_default_params plus overrides (for example precision=MG_F64, levels=5)."""
    p = Params()
    _check(lib().mg_default_params(C.byref(p), n, m), "mg_default_params")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _markers(mk):
    a = np.ascontiguousarray(np.asarray(mk, dtype=np.float64).reshape(-1, 2))
    return a, a.ctypes.data_as(C.POINTER(C.c_double)), len(a)


class Solver:
    """One image's solver (mg_setup ... mg_destroy).  `image` is a CUDA torch tensor of shape
    (n, m), float32 for MG_F32 or float64 for MG_F64."""

    def __init__(self, image, markers, params: Params, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the solver has no CPU path")
        dt = torch.float64 if params.precision == MG_F64 else torch.float32
        if not (image.is_cuda and image.dtype == dt and image.dim() == 2):
            raise TypeError(f"image must be a 2-D CUDA tensor of {dt}")
        self.image = image.contiguous()
        self.n, self.m = self.image.shape
        self.params = params
        self.dtype = dt
        self._mk, pm, k = _markers(markers)
        torch.cuda.current_stream().synchronize()
        h = C.c_void_p()
        st = None if stream is None else C.c_void_p(stream)
        _check(lib().mg_setup(C.byref(h), C.c_void_p(self.image.data_ptr()), self.n, self.m, pm, k,
                              C.byref(params), None, st), "mg_setup")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream_ptr(self) -> int:
        return lib().mg_get_stream(self._h) or 0

    def reset(self, image, markers):
        import torch
        img = image.contiguous()
        _, pm, k = _markers(markers)
        torch.cuda.current_stream().synchronize()
        _check(lib().mg_reset(self._h, C.c_void_p(img.data_ptr()), pm, k), "mg_reset")

    def begin_step(self) -> float:
        r = C.c_double()
        _check(lib().mg_begin_step(self._h, C.byref(r)), "mg_begin_step")
        return r.value

    def vcycle(self) -> float:
        r = C.c_double()
        _check(lib().mg_vcycle(self._h, C.byref(r)), "mg_vcycle")
        return r.value

    def end_step(self) -> float:
        e = C.c_double()
        _check(lib().mg_end_step(self._h, C.byref(e)), "mg_end_step")
        return e.value

    def solve_step(self, tol, max_cycles=50, raise_on_cap=False):
        """One pseudo-time step; returns (cycles, rho)."""
        c, r = C.c_int(), C.c_double()
        rc = lib().mg_solve_step(self._h, tol, max_cycles, C.byref(c), C.byref(r))
        if rc != 0 and (rc != -5 or raise_on_cap):
            _check(rc, "mg_solve_step")
        return c.value, r.value

    def solve(self, tol, max_cycles, eta_stop, max_steps) -> int:
        s = C.c_int()
        _check(lib().mg_solve(self._h, tol, max_cycles, eta_stop, max_steps, C.byref(s)), "mg_solve")
        return s.value

    def mask(self, out=None):
        import torch
        out = torch.empty((self.n, self.m), dtype=torch.uint8, device=self.image.device) if out is None else out
        _check(lib().mg_mask(self._handle, C.c_void_p(out.data_ptr())), "mg_mask")
        return out

    def phi(self):
        import torch
        out = torch.empty((self.n, self.m), dtype=self.dtype, device=self.image.device)
        _check(lib().mg_get_phi(self._handle, C.c_void_p(out.data_ptr())), "mg_get_phi")
        return out

    def set_phi(self, phi):
        import torch
        t = phi.to(device=self.image.device, dtype=self.dtype).contiguous()
        torch.cuda.current_stream().synchronize()
        _check(lib().mg_set_phi(self._h, C.c_void_p(t.data_ptr())), "mg_set_phi")

    def set_regions(self, c1, c2):
        _check(lib().mg_set_regions(self._h, float(c1), float(c2)), "mg_set_regions")

    def level(self, l, field):
        """field: 0 phi, 1 w, 2 z, 3 d, 4 F, 5 rhs, 6 G, 7 omega."""
        import torch
        names = {"phi": 0, "w": 1, "z": 2, "d": 3, "F": 4, "rhs": 5, "G": 6, "omega": 7}
        f = names.get(field, field)
        n, m = self.n >> l, self.m >> l
        out = torch.empty((n, m), dtype=self.dtype, device=self.image.device)
        _check(lib().mg_get_level(self._h, l, f, C.c_void_p(out.data_ptr())), "mg_get_level")
        return out

    @classmethod
    def view(cls, handle, n, m, params, device):
        """A non-owning Solver over a handle that belongs to a Batch."""
        import torch
        obj = cls.__new__(cls)
        obj._h = None
        obj._view = C.c_void_p(handle)
        obj.n, obj.m, obj.params = n, m, params
        obj.dtype = torch.float64 if params.precision == MG_F64 else torch.float32
        obj.image = torch.empty(0, device=device)
        return obj

    @property
    def _handle(self):
        return self._h if self._h else self._view

    def autotune(self, reps=2):
        """mg_autotune inside the current step; returns the tile shape chosen per grid."""
        out = (C.c_int * 16)()
        _check(lib().mg_autotune(self._h, reps, out), "mg_autotune")
        return list(out)[: self.params.levels - 1]

    def set_tile_shapes(self, shapes):
        arr = (C.c_int * 16)(*shapes)
        _check(lib().mg_set_tile_shapes(self._h, arr), "mg_set_tile_shapes")

    def aos(self, dt, max_iter, eta):
        """AOS time marching on the finest grid (mg_aos); returns (iterations, rho)."""
        it, r = C.c_int(), C.c_double()
        _check(lib().mg_aos(self._h, dt, max_iter, eta, C.byref(it), C.byref(r)), "mg_aos")
        return it.value, r.value

    def set_learned(self, theta=None, mode=1, refresh=4):
        """Learned relaxation weights (mg_set_learned): theta (3201 floats) or None."""
        import numpy as np
        ptr = None
        if theta is not None:
            th = np.ascontiguousarray(theta, dtype=np.float32)
            assert th.size == lib().mg_learned_nparam()
            ptr = th.ctypes.data_as(C.POINTER(C.c_float))
        _check(lib().mg_set_learned(self._h, ptr, mode, refresh), "mg_set_learned")

    def set_omega(self, level, omega):
        """Fixed relaxation weights of one grid (mg_set_omega); None switches them off."""
        import numpy as np
        if omega is None:
            _check(lib().mg_set_omega(self._h, level, None), "mg_set_omega")
            return
        dt = np.float64 if str(self.dtype) == "torch.float64" else np.float32
        w = np.ascontiguousarray(omega, dtype=dt)
        _check(lib().mg_set_omega(self._h, level, C.c_void_p(w.ctypes.data)), "mg_set_omega")

    def energy(self) -> float:
        """Level-set energy of the current phi with the current c1, c2 (mg_energy)."""
        e = C.c_double()
        _check(lib().mg_energy(self._h, C.byref(e)), "mg_energy")
        return e.value

    def set_bottom_kernel(self, enable=True):
        """Switches the one-block bottom-of-cycle kernel (mg_set_bottom_kernel); returns the first
        grid it covers, or -1 when it does not apply."""
        lb = C.c_int(-1)
        _check(lib().mg_set_bottom_kernel(self._h, 1 if enable else 0, C.byref(lb)), "mg_set_bottom_kernel")
        return lb.value

    def set_bottom_level(self, level):
        """First grid of the bottom kernel (mg_set_bottom_level); -1 for none."""
        _check(lib().mg_set_bottom_level(self._h, int(level)), "mg_set_bottom_level")

    def set_cluster_level(self, level):
        """First grid of the cluster bottom kernel (mg_set_cluster_level); -1 for none."""
        _check(lib().mg_set_cluster_level(self._h, int(level)), "mg_set_cluster_level")

    def time_kernels(self, level=0, reps=3):
        """Mean ms per launch of snapshot, sweeps A..D and residual on `level` (mg_time_kernels)."""
        out = (C.c_double * 6)()
        _check(lib().mg_time_kernels(self._h, level, reps, out), "mg_time_kernels")
        return list(out)

    def time_residuals(self, level=0, reps=3):
        """Mean ms of the residual-norm kernels and of the residual with full weighting on `level`
        (mg_time_residuals; the second is -1 on the coarsest grid)."""
        out = (C.c_double * 2)()
        _check(lib().mg_time_residuals(self._h, level, reps, out), "mg_time_residuals")
        return list(out)

    def time_sweeps_graph(self, level=0, reps=8):
        """Mean ms per Hybrid Smoother 2 sweep on `level`, the sweeps of `reps` outer iterations
        replayed from one CUDA graph (mg_time_sweeps_graph)."""
        out = (C.c_double * 1)()
        _check(lib().mg_time_sweeps_graph(self._h, level, reps, out), "mg_time_sweeps_graph")
        return out[0]

    def set_wait_limit(self, rounds):
        """Bound of the fused sweep's device-side waits (mg_set_wait_limit); 0 gives up at once."""
        _check(lib().mg_set_wait_limit(self._h, int(rounds)), "mg_set_wait_limit")

    def inject_divergence(self, cycle):
        """mg_inject_divergence: the cycle-th V-cycle from now reports a diverged residual once."""
        _check(lib().mg_inject_divergence(self._h, int(cycle)), "mg_inject_divergence")

    def stats(self) -> dict:
        s = Stats()
        _check(lib().mg_get_stats(self._handle, C.byref(s)), "mg_get_stats")
        return s.as_dict()


class Batch:
    """Many images solved together (mg_batch_*): one CUDA graph launch per V-cycle."""

    def __init__(self, images, markers, params, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the solver has no CPU path")
        self.images = [im.contiguous() for im in images]
        cnt = len(self.images)
        self._mks = [np.ascontiguousarray(np.asarray(mk, dtype=np.float64).reshape(-1, 2)) for mk in markers]
        self.params = list(params)
        imgs = (C.c_void_p * cnt)(*[im.data_ptr() for im in self.images])
        ns = (C.c_int * cnt)(*[im.shape[0] for im in self.images])
        ms = (C.c_int * cnt)(*[im.shape[1] for im in self.images])
        mks = (C.POINTER(C.c_double) * cnt)(*[mk.ctypes.data_as(C.POINTER(C.c_double)) for mk in self._mks])
        ks = (C.c_int * cnt)(*[len(mk) for mk in self._mks])
        ps = (Params * cnt)(*self.params)
        torch.cuda.current_stream().synchronize()
        b = C.c_void_p()
        _check(lib().mg_batch_setup(C.byref(b), cnt, imgs, ns, ms, mks, ks, ps,
                                    None if stream is None else C.c_void_p(stream)), "mg_batch_setup")
        self._b = b
        self.count = cnt

    def close(self):
        if getattr(self, "_b", None):
            lib().mg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, reps=2):
        _check(lib().mg_batch_autotune(self._b, reps), "mg_batch_autotune")

    def reset(self, images=None, markers=None):
        """mg_reset on every image's handle (the same images and markers by default)."""
        import torch
        images = self.images if images is None else [im.contiguous() for im in images]
        mks = self._mks if markers is None else [
            np.ascontiguousarray(np.asarray(mk, dtype=np.float64).reshape(-1, 2)) for mk in markers]
        torch.cuda.current_stream().synchronize()
        for i in range(self.count):
            h = lib().mg_batch_handle(self._b, i)
            _check(lib().mg_reset(h, C.c_void_p(images[i].data_ptr()),
                                  mks[i].ctypes.data_as(C.POINTER(C.c_double)), len(mks[i])), "mg_reset")
        self.images, self._mks = images, mks

    def solve_step(self, tol, max_cycles=60, raise_on_cap=False):
        cyc = (C.c_int * self.count)()
        rho = (C.c_double * self.count)()
        rc = lib().mg_batch_solve_step(self._b, tol, max_cycles, cyc, rho)
        if rc != 0 and (rc != -5 or raise_on_cap):
            _check(rc, "mg_batch_solve_step")
        return list(cyc), list(rho)

    def solver(self, i) -> "Solver":
        h = lib().mg_batch_handle(self._b, i)
        n, m = self.images[i].shape
        return Solver.view(h, n, m, self.params[i], self.images[i].device)


def residual_norm_noalloc(phi, w, F, params: Params) -> float:
    """mg_residual_norm_noalloc on dense CUDA tensors of the params' precision (no allocation
    inside the library).  The three tensors must be 2-D of one shape, of the dtype the precision
    implies (float64 for MG_F64, else float32), contiguous and on a CUDA device: anything else is
    refused here, before the library reads any of them."""
    import torch
    want = torch.float64 if params.precision == MG_F64 else torch.float32
    ts = {"phi": phi, "w": w, "F": F}
    for name, t in ts.items():
        if not isinstance(t, torch.Tensor) or t.dim() != 2 or tuple(t.shape) != tuple(phi.shape):
            raise TypeError(f"{name} must be a 2-D tensor of phi's shape {tuple(phi.shape)}")
    for name, t in ts.items():
        if t.dtype != want:
            raise TypeError(f"{name} is {t.dtype}; the params' precision needs {want}")
    for name, t in ts.items():
        if not t.is_contiguous():
            raise TypeError(f"{name} must be contiguous (dense row-major)")
    for name, t in ts.items():
        if not t.is_cuda:
            raise TypeError(f"{name} must be on a CUDA device")
    n, m = phi.shape
    out = C.c_double()
    rc = lib().mg_residual_norm_noalloc(C.c_void_p(phi.data_ptr()), C.c_void_p(w.data_ptr()),
                                        C.c_void_p(F.data_ptr()), n, m, C.byref(params),
                                        C.byref(out), None)
    if rc != 0:
        raise SegmgError(rc, "mg_residual_norm_noalloc", "see include/segmg.h")
    return out.value


def segment_host(image, markers, params: Params, tol=1e-6, max_cycles=50, eta_stop=0.0,
                 max_steps=1, want_phi=False, mask_out=None):
    """Whole pipeline from host buffers (mg_segment_host): returns (mask, phi or None, stats).
    mask_out: an n x m uint8 C-contiguous array to write the mask into (for example one in
    page-locked memory, reused across calls); a new array when None."""
    img = np.ascontiguousarray(image, dtype=np.float32)
    n, m = img.shape
    _, pm, k = _markers(markers)
    if mask_out is not None:
        if mask_out.shape != (n, m) or mask_out.dtype != np.uint8 or not mask_out.flags["C_CONTIGUOUS"]:
            raise TypeError("mask_out must be a C-contiguous n x m uint8 array")
        mask = mask_out
    else:
        mask = np.empty((n, m), dtype=np.uint8)
    phi = np.empty((n, m), dtype=np.float32) if want_phi else None
    st = Stats()
    _check(lib().mg_segment_host(img.ctypes.data_as(C.c_void_p), n, m, pm, k, C.byref(params), tol,
                                 max_cycles, eta_stop, max_steps, mask.ctypes.data_as(C.c_void_p),
                                 phi.ctypes.data_as(C.c_void_p) if want_phi else None, C.byref(st)),
           "mg_segment_host")
    return mask, phi, st.as_dict()


def segment_host_release():
    """mg_segment_host_release: frees the context mg_segment_host keeps between calls."""
    lib().mg_segment_host_release()


class Trainer:
    """Training of the learned relaxation weights (mg_trainer_*)."""

    def __init__(self, capacity, batch_max=64, seed=0, theta0=None):
        import numpy as np
        h = C.c_void_p()
        ptr = None
        if theta0 is not None:
            self._t0 = np.ascontiguousarray(theta0, dtype=np.float32)
            ptr = self._t0.ctypes.data_as(C.POINTER(C.c_float))
        _check(lib().mg_trainer_create(C.byref(h), capacity, batch_max, seed, ptr), "mg_trainer_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().mg_trainer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def record(self, solver, count):
        _check(lib().mg_trainer_record(self._h, solver._handle, count), "mg_trainer_record")

    def load(self, records):
        import numpy as np
        r = np.ascontiguousarray(records, dtype=np.float32)
        _check(lib().mg_trainer_load(self._h, r.ctypes.data_as(C.POINTER(C.c_float)), r.shape[0]), "mg_trainer_load")

    @property
    def count(self):
        return lib().mg_trainer_count(self._h)

    def set_loss(self, kind):
        """mg_trainer_set_loss: 0 the residual, 1 its high-frequency part ("hf")."""
        _check(lib().mg_trainer_set_loss(self._h, {"full": 0, "hf": 1}.get(kind, kind)), "mg_trainer_set_loss")

    def grad(self, idx):
        import numpy as np
        ix = np.ascontiguousarray(idx, dtype=np.int32)
        g = np.zeros(lib().mg_learned_nparam(), dtype=np.float32)
        loss = C.c_double()
        _check(lib().mg_trainer_grad(self._h, ix.ctypes.data_as(C.POINTER(C.c_int)), ix.size,
                                     g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)), "mg_trainer_grad")
        return loss.value, g

    def train(self, iters, batch, lr):
        loss = C.c_double()
        _check(lib().mg_trainer_train(self._h, iters, batch, lr, C.byref(loss)), "mg_trainer_train")
        return loss.value

    def theta(self):
        import numpy as np
        out = np.zeros(lib().mg_learned_nparam(), dtype=np.float32)
        _check(lib().mg_trainer_get(self._h, out.ctypes.data_as(C.POINTER(C.c_float))), "mg_trainer_get")
        return out
