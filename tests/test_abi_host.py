"""The C-ABI library builds, loads and exports every symbol include/bspline.h declares.

No compute calls: only argument checks that return before any CUDA call.
"""
import os
import re

import pytest

from paper_1201_4060_gb300 import _build
from paper_1201_4060_gb300 import bspline as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def _declared():
    txt = open(os.path.join(ROOT, "include", "bspline.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bspline_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert "bspline_interp" in names and "bspline_coeffs" in names and len(names) >= 14
    lib = B.lib()
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_version():
    assert B.status_string(B.OK) == "ok"
    assert "not implemented" in B.status_string(B.ERR_NOT_IMPLEMENTED)
    assert B.status_string(12345) == "unknown status"
    assert B.version().startswith("bspline-gb300")


def test_plan_argument_checks_before_cuda():
    assert B.lib().bspline_plan(None, 32, 4, B.F32) == B.ERR_INVALID_ARG
    for N in (0, 4, 7, 12, 24, 36, 80, 1536, 2048):      # 3 * 2^k grids start at 48
        rc, h = B.bspline_plan(N, 4, B.F32)
        assert rc == B.ERR_UNSUPPORTED_N and h == 0
    for order in (0, 1, 9, -3):
        rc, h = B.bspline_plan(32, order, B.F32)
        assert rc == B.ERR_UNSUPPORTED_ORDER and h == 0
    rc, h = B.bspline_plan(32, 4, 7)
    assert rc == B.ERR_INVALID_ARG and h == 0


def test_null_plan_is_rejected_everywhere():
    assert B.bspline_destroy(0) == B.OK
    assert B.bspline_coeffs(0, 16, 32) == B.ERR_INVALID_ARG
    assert B.bspline_interp(0, 16, 16, 10, 16, 16, 0) == B.ERR_INVALID_ARG
    assert B.bspline_eval(0, 16, 32, 16, 10, 16, 16, 0) == B.ERR_INVALID_ARG
    assert B.bspline_plan_set_stream(0, 0) == B.ERR_INVALID_ARG
    assert B.bspline_plan_set_length(0, 1.0) == B.ERR_INVALID_ARG
    assert B.bspline_plan_set_prefilter(0, 0) == B.ERR_INVALID_ARG
    assert B.bspline_workspace_bytes(0, 10)[0] == B.ERR_INVALID_ARG
    assert B.bspline_coeffs_bytes(0)[0] == B.ERR_INVALID_ARG
    assert B.bspline_uhat_bytes(0)[0] == B.ERR_INVALID_ARG
    assert B.bspline_status(0)[0] == B.ERR_INVALID_ARG
    assert B.bspline_run_host(0, 16, 16, 1, 16, 16) == B.ERR_INVALID_ARG
    assert B.bspline_run_host_async(0, 16, 16, 1, 16, 16) == B.ERR_INVALID_ARG
    assert B.bspline_wait(0) == B.ERR_INVALID_ARG
    assert B.lib().bspline_plan_set_gather_split(None, 8) == B.ERR_INVALID_ARG
    assert B.lib().bspline_plan_autotune(None, None, None, 10, None, None, None, None) == B.ERR_INVALID_ARG
    assert B.bspline_spread_adjoint(0, 0, 0, 0, 0, 0, 0, 0, 0) == B.ERR_INVALID_ARG
    assert B.bspline_plan_set_timing(0, 1) == B.ERR_INVALID_ARG
    assert B.bspline_stage_times(0)[0] == B.ERR_INVALID_ARG
    assert B.bspline_plan_set_test_hooks(0, 1) == B.ERR_INVALID_ARG
    lib = B.lib()
    assert lib.bspline_batch_create(None, 1, None) == B.ERR_INVALID_ARG
    h = B.ctypes.c_void_p()
    assert lib.bspline_batch_create(B.ctypes.byref(h), 0, None) == B.ERR_INVALID_ARG and not h.value
    plans = (B.ctypes.c_void_p * 2)(0, 0)
    assert lib.bspline_batch_create(B.ctypes.byref(h), 2, plans) == B.ERR_INVALID_ARG and not h.value
    assert lib.bspline_batch_launch(None, None) == B.ERR_INVALID_ARG
    assert lib.bspline_batch_autotune(None, None, None, None) == B.ERR_INVALID_ARG
    assert lib.bspline_batch_capture(None, 1, None, None, None, None, None, None) == B.ERR_INVALID_ARG
    assert lib.bspline_batch_destroy(None) == B.OK


def test_binding_checks_buffers_before_passing_their_pointers():
    """The Python binding refuses buffers the library would overrun: wrong shape, dtype, strides or side."""
    torch = pytest.importorskip("torch")
    ok = torch.empty((5, 3), dtype=torch.float32)
    B._require(ok, "u", (5, 3), torch.float32, "cpu")
    bad = [
        (torch.empty((4, 3), dtype=torch.float32), (5, 3), torch.float32, "cpu"),       # too few rows
        (torch.empty((5, 3), dtype=torch.float64), (5, 3), torch.float32, "cpu"),       # wrong dtype
        (torch.empty((3, 5), dtype=torch.float32).t(), (5, 3), torch.float32, "cpu"),   # strided view
        (ok, (5, 3), torch.float32, "cuda"),                                            # host tensor for device
    ]
    for t, shape, dtype, side in bad:
        with pytest.raises(ValueError):
            B._require(t, "u", shape, dtype, side)


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "bspline.h"

int main(void) {
    bspline_plan_t plan = 0;
    size_t bytes = 0;
    int64_t n = 0;
    /* argument checks that return before any CUDA call */
    if (bspline_plan(NULL, 64, 4, BSPLINE_F32) != BSPLINE_ERR_INVALID_ARG) return 1;
    if (bspline_plan(&plan, 100, 4, BSPLINE_F32) != BSPLINE_ERR_UNSUPPORTED_N || plan) return 2;
    if (bspline_plan(&plan, 64, 9, BSPLINE_F32) != BSPLINE_ERR_UNSUPPORTED_ORDER) return 3;
    if (bspline_coeffs_bytes(NULL, &bytes) != BSPLINE_ERR_INVALID_ARG) return 4;
    if (bspline_status(NULL, &n) != BSPLINE_ERR_INVALID_ARG) return 5;
    if (bspline_interp(NULL, NULL, NULL, 0, NULL, NULL, 0) != BSPLINE_ERR_INVALID_ARG) return 6;
    if (strlen(bspline_status_string(BSPLINE_ERR_TIMEOUT)) == 0) return 7;
    printf("%s\n", bspline_version());
    return 0;
}
"""


def test_header_compiles_as_c99_and_links_from_c(tmp_path):
    """include/bspline.h is plain C: a C99 client builds with warnings as errors, links against the
    library and gets the documented status codes from calls that need no GPU."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    lib_dir = os.path.dirname(_build.LIB)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", lib_dir, "-lbspline", "-Wl,-rpath," + lib_dir, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == B.version()


@pytest.mark.parametrize("N", [8, 16, 48, 64, 96, 512])
@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7, 8])
def test_library_prefilter_table_matches_the_oracle(N, order):
    """The c(k) the library computes on the host (node values by the Cox-de Boor recurrence, cosines
    of k d reduced mod N, angle reduced to an octant) against the oracle's literal DFT sum
    (interpolating prefilter) and its sinc / Poisson-sum form (L2 prefilter).

    Bound: the oracle's angles 2 pi k x / N reach 2 pi N, so each cosine carries up to 2 pi N eps of
    phase rounding; F = 1/c is a sum with weights summing to one, and |dc| = c^2 |dF|, so
    |dc| / max c <= max c * 2 pi N eps (plus a few eps for the sums themselves)."""
    import math

    import numpy as np
    from oracle import bspline_oracle as O
    eps = np.finfo(np.float64).eps
    for kind, ref in ((B.PREFILTER_INTERP, O.prefilter(N, order)), (B.PREFILTER_L2, O.prefilter_l2(N, order))):
        rc, c = B.bspline_prefilter_values(N, order, kind)
        assert rc == B.OK
        c = np.asarray(c)
        assert c.shape == (N,)
        cmax = np.abs(ref).max()
        tol = cmax * 2 * math.pi * N * eps + 16 * eps
        assert np.abs(c - ref).max() <= tol * cmax


def test_prefilter_values_argument_checks():
    assert B.bspline_prefilter_values(100, 4, B.PREFILTER_INTERP)[0] == B.ERR_UNSUPPORTED_N
    assert B.bspline_prefilter_values(64, 9, B.PREFILTER_INTERP)[0] == B.ERR_UNSUPPORTED_ORDER
    assert B.bspline_prefilter_values(64, 4, 7)[0] == B.ERR_INVALID_ARG
    assert B.lib().bspline_prefilter_values(64, 4, 0, None) == B.ERR_INVALID_ARG
