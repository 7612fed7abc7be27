"""The C-ABI library builds for sm_103a and exports every function include/segmg.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "segmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(mg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1807_02137_gb300 import buildlib
    return buildlib.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["mg_setup", "mg_vcycle", "mg_solve", "mg_mask", "mg_destroy", "mg_get_stats",
                 "mg_strerror", "mg_segment_host", "mg_begin_step", "mg_end_step"]:
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mg_\w+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing


def test_library_loads_and_binding_matches_struct_layouts(libpath):
    import ctypes
    from paper_1807_02137_gb300 import segmg
    L = segmg.lib()
    for name in declared_functions():
        assert hasattr(L, name)
    # sizes of the C structs, compiled with the host compiler from the header
    code = ('#include <stdio.h>\n#include "segmg.h"\n'
            'int main(){printf("%zu %zu %zu %zu", sizeof(mg_params), sizeof(mg_stats), sizeof(mg_allocator),'
            ' sizeof(mg_debug_info));}')
    exe = os.path.join(os.path.dirname(libpath), "abi_sizes")
    subprocess.run(["gcc", "-x", "c", "-", "-I", os.path.join(ROOT, "include"), "-o", exe], input=code,
                   text=True, check=True)
    sizes = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert int(sizes[0]) == ctypes.sizeof(segmg.Params)
    assert int(sizes[1]) == ctypes.sizeof(segmg.Stats)
    assert int(sizes[3]) == ctypes.sizeof(segmg.DebugInfo)


def test_host_only_calls_without_a_gpu(libpath):
    from paper_1807_02137_gb300 import segmg
    p = segmg.default_params(1024, 1024)
    assert p.levels == 9 and p.tau == 1.0 and p.Sigma == 2.0 and abs(p.sigma_d - 51.2) < 1e-12
    assert segmg.lib().mg_strerror(-6) == b"coarsest system not positive definite"
    # a NULL handle is rejected before any CUDA call
    assert segmg.lib().mg_vcycle(None, None) == -1


def test_noalloc_binding_refuses_mismatched_tensors_before_any_call(libpath):
    # float32 tensors with FP64 params would make the kernel read twice the buffers' bytes: the
    # binding refuses them (and non-CUDA, strided or mis-shaped tensors) before the library runs
    import torch
    from paper_1807_02137_gb300 import segmg
    p = segmg.default_params(8, 8, precision=segmg.MG_F64)
    f32 = torch.zeros(8, 8, dtype=torch.float32)
    with pytest.raises(TypeError, match="precision"):
        segmg.residual_norm_noalloc(f32, f32, f32, p)
    f64 = torch.zeros(8, 8, dtype=torch.float64)
    with pytest.raises(TypeError, match="shape"):
        segmg.residual_norm_noalloc(f64, f64, torch.zeros(8, 9, dtype=torch.float64), p)
    with pytest.raises(TypeError, match="contiguous"):
        segmg.residual_norm_noalloc(f64, f64, torch.zeros(8, 16, dtype=torch.float64)[:, ::2], p)
    with pytest.raises(TypeError, match="CUDA"):
        segmg.residual_norm_noalloc(f64, f64, f64, p)


def test_default_build_reports_no_bounds_checks(libpath):
    # the default library has no checks: mg_debug_status says so without touching the device,
    # and the self-test of the reporting path does nothing
    from paper_1807_02137_gb300 import segmg
    if os.environ.get("SEGMG_DEBUG") == "1":
        pytest.skip("the bounds-checked library is selected")
    d = segmg.debug_status()
    assert d == {"enabled": 0, "first_site": -1, "first_index": 0, "sites": 0, "count": 0}
    segmg.debug_selftest()
    assert segmg.lib().mg_debug_status(None, 0) == -1


def test_bounds_checked_build_compiles_and_exports_every_symbol():
    # -DMG_DEBUG variant: its own objects, the same C ABI
    from paper_1807_02137_gb300 import buildlib
    path = buildlib.build(debug=True)
    assert path.endswith("libsegmg_debug.so")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mg_\w+)", out))
    assert not set(declared_functions()) - exported


def test_segment_host_binding_refuses_a_bad_mask_buffer_before_any_call(libpath):
    # the mask buffer is written by the library: wrong shape, type or layout is refused first
    import numpy as np
    from paper_1807_02137_gb300 import segmg
    p = segmg.default_params(16, 16)
    img = np.zeros((16, 16), np.float32)
    mk = np.array([[8.0, 8.0]])
    for bad in (np.zeros((16, 15), np.uint8), np.zeros((16, 16), np.int32), np.zeros((16, 32), np.uint8)[:, ::2]):
        with pytest.raises(TypeError, match="mask_out"):
            segmg.segment_host(img, mk, p, mask_out=bad)
    segmg.segment_host_release()   # nothing kept: a no-op without a device
