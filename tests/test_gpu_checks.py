"""The BSPLINE_CHECKS=1 build: every particle kernel with index checks (stencil origin inside the staged
tile, output and record indices inside their arrays, sorted slots inside their brick's segment) that
count a failure in a status word and skip the access instead of trapping.  On the small parity cases
no check may fail, and the checked build must give the default build's bits."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(lib, path):
    env = dict(os.environ, BSPLINE_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checks_cases.py"), path], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(path))


def test_checks_build_passes_and_matches_default_build(tmp_path):
    from paper_1201_4060_gb300 import _build
    default = _build.build()
    checked = _build.build(checks=True)
    a = _run(checked, str(tmp_path / "checks.npz"))
    b = _run(default, str(tmp_path / "default.npz"))
    status = {k: int(v) for k, v in a.items() if k.startswith("status_")}
    assert status and all(v == 0 for v in status.values()), status
    for k, v in b.items():
        if k.startswith("status_") or k.endswith("_det"):
            continue
        assert np.array_equal(v, a[k], equal_nan=True), k
    # the deterministic spread is bit-identical between the two builds as well
    for k in b:
        if k.endswith("_det"):
            assert np.array_equal(a[k], b[k]), k
