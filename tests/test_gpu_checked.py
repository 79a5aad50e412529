"""Bounds-checked library variant (FDTD_CHECK=1): every global store and TMA x origin of the fused
kernels is checked before it happens; a failing check would be skipped and reported as a device status
(FdtdError at the next synchronising call).  The configurations of tests/checked_runs.py run with it in
a subprocess: none may report, and every field must equal the normal library's bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_reports_nothing_and_matches(tmp_path):
    from tests import checked_runs
    normal = checked_runs.run_all()
    out = tmp_path / "checked.npz"
    env = dict(os.environ, FDTD_CHECK="1")
    r = subprocess.run([sys.executable, "-m", "tests.checked_runs", str(out)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    checked = np.load(out)
    assert set(checked.files) == set(normal)
    for k in checked.files:
        assert np.array_equal(checked[k], normal[k]), k
