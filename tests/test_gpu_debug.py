"""The bounds-checked build (-DMG_DEBUG): on small, tiny, ragged and degenerate cases that reach
every kernel family, no checked access goes out of range, the results equal the default build's
bit for bit, and the reporting path records what it is given."""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_cases(out, debug):
    env = dict(os.environ, SEGMG_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_cases.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(out))


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    need_gpu()
    from paper_1807_02137_gb300 import buildlib
    buildlib.build(debug=True)
    d = tmp_path_factory.mktemp("debug")
    return run_cases(d / "release.npz", False), run_cases(d / "debug.npz", True)


def test_no_checked_access_is_out_of_range(results):
    rel, dbg = results
    assert str(dbg["library"]).endswith("libsegmg_debug.so")
    enabled, first_site, first_index, sites, count = (int(v) for v in dbg["debug/status"])
    assert enabled == 1
    assert count == 0 and sites == 0 and first_site == -1, (first_site, first_index, hex(sites), count)
    # the default build has no checks and says so
    assert int(rel["debug/status"][0]) == 0


def test_results_equal_the_default_build_bitwise(results):
    rel, dbg = results
    keys = sorted(k for k in rel if not k.startswith("debug/") and k != "library")
    assert keys == sorted(k for k in dbg if not k.startswith("debug/") and k != "library")
    assert len(keys) > 40
    for k in keys:
        assert rel[k].shape == dbg[k].shape, k
        assert np.array_equal(rel[k], dbg[k], equal_nan=True), k


def test_reporting_path_records_site_index_and_count(results):
    _, dbg = results
    enabled, first_site, first_index, sites, count = (int(v) for v in dbg["debug/selftest"])
    assert (enabled, first_site, first_index, count) == (1, 10, 1005, 1)
    assert sites == 1 << 10
    assert list(dbg["debug/cleared"]) == [0, 0]
