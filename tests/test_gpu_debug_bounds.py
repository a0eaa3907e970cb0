"""GPU: the debug build's index checks (-DLF2_DEBUG_BOUNDS) on every instrumented kernel.

The library built with the checks runs the one-step, streaming, temporal-blocking (1 to 6
components), ensemble, energy and fused step + energy kernels on small cases with ragged tiles
and z-chunks.  It must count no index outside an allocation, and its results must be bitwise
those of the release library (the checks change no value)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run_battery(lib_path, out_path):
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_battery.py"), lib_path, out_path],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_counts_no_violation_and_changes_no_result(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1508_05610_gb300 import build, lf2
    release = build.build()
    debug = build.build(debug_bounds=True)
    assert debug == lf2.DEBUG_LIB_PATH
    got_dbg = run_battery(debug, str(tmp_path / "dbg.npz"))
    got_rel = run_battery(release, str(tmp_path / "rel.npz"))
    assert got_dbg["violations"] == 0
    assert got_rel["violations"] is None
    a, b = np.load(tmp_path / "dbg.npz"), np.load(tmp_path / "rel.npz")
    assert sorted(a.files) == sorted(b.files) and len(a.files) == got_dbg["arrays"] > 20
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
