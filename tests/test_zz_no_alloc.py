"""mg_residual_norm_noalloc: the residual norm for callers that cannot allocate device memory.

The entry point keeps its scratch in a static device array instead of allocating it.  It must
give the same norm as the solver's own start-of-step norm (mg_begin_step, which uses scratch the
handle allocated) for the same level set, on two calls in a row (the second call reuses the array
the first one left behind).  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1807_02137_gb300 import synth
from tests.gpu_common import gpu_solver, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,shape", [("f32", (1024, 1024)), ("f64", (128, 128)),
                                             ("f32", (300, 173))])
def test_noalloc_norm_matches_the_solver_norm_twice(precision, shape):
    segmg = need_gpu()
    prec = segmg.MG_F64 if precision == "f64" else segmg.MG_F32
    n, m = shape
    img, mk, _ = synth.ellipses(n, m, 10, (10, min(n, m) / 3), 6, 0.05, 21)
    s, p = gpu_solver(segmg, img, mk, precision=prec)
    ref = s.begin_step()                       # ||L(phi^n)||, scratch allocated by the handle
    phi, w, F = s.phi(), s.level(0, "w"), s.level(0, "F")
    got1 = segmg.residual_norm_noalloc(phi, w, F, p)
    got2 = segmg.residual_norm_noalloc(phi, w, F, p)
    assert ref > 0
    assert abs(got1 - ref) <= 1e-12 * ref
    assert abs(got2 - ref) <= 1e-12 * ref
    # different inputs in between (the curvature term is invariant to scaling phi, so change F):
    # the array holds only the last call's values
    other = segmg.residual_norm_noalloc(phi, w, F * 0.5, p)
    assert abs(other - ref) > 1e-6 * ref
    assert abs(segmg.residual_norm_noalloc(phi, w, F, p) - ref) <= 1e-12 * ref
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import ctypes
    segmg = need_gpu()
    p = segmg.default_params(8200, 8200)
    t = torch.zeros(1, device="cuda")
    out = ctypes.c_double(-1.0)
    # 257 x 257 tiles of 32 x 32 cells exceed the 65536 the static array holds; the size check
    # comes before any device access, so the one-element buffers are never read
    rc = segmg.lib().mg_residual_norm_noalloc(t.data_ptr(), t.data_ptr(), t.data_ptr(), 8200, 8200,
                                              ctypes.byref(p), ctypes.byref(out), None)
    assert rc == -1 and out.value == -1.0
