"""bspline_interp_noalloc: the allocation-free entry point, for callers that cannot allocate device
memory (inside another framework's graph capture, in code that must never stall the GPU, or under a
fixed device-memory budget).  Its outputs must match bspline_interp's on a plan with the same grid,
order, type and domain, on consecutive calls that reuse the library's one fixed scratch array.
This file is collected last so that a run stopping at the first failure has run every other test."""
import math

import numpy as np
import pytest

from paper_1201_4060_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": (1e-12, 1e-12), "f32": (2e-5, 5e-5), "bf16": (2e-2, 5e-2)}


@pytest.fixture(scope="module")
def B():
    from paper_1201_4060_gb300 import _build
    _build.build()
    from paper_1201_4060_gb300 import bspline
    return bspline


def normwise(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def plan_path(B, N, order, dtype, L, x, seed):
    plan = B.Plan(N, order, dtype, L=L)
    half = synth.kolmogorov_field(N, seed=seed).dense()
    coef = plan.coeffs(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
    u, g = plan.interp(coef, x)
    torch.cuda.synchronize()
    return plan, coef, u, g


def noalloc(B, coef, N, order, dtype, L, x, out_dtype):
    P = x.shape[0]
    u = torch.full((P, 3), float("nan"), dtype=out_dtype, device="cuda")
    g = torch.full((P, 3, 3), float("nan"), dtype=out_dtype, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = B.bspline_interp_noalloc(coef.data_ptr(), N, order, B.DTYPES[dtype], L, x.data_ptr(), P,
                                  u.data_ptr(), g.data_ptr(), 0, stream)
    assert rc == B.OK, B.status_string(rc)
    torch.cuda.synchronize()
    return u, g


def test_noalloc_matches_plan_path_on_consecutive_calls(B):
    L = 2.0 * math.pi
    cases = [
        # larger call first, then a smaller one with another grid: stale scratch would show
        (64, 6, "f64", L, synth.clustered_particles(B.NOALLOC_MAX_PARTICLES, seed=7), 31),
        (32, 4, "f32", L, synth.uniform_particles(5003, seed=8), 32),
        (16, 5, "bf16", 3.0, np.random.default_rng(9).uniform(-3.0, 6.0, (777, 3)), 33),
        # the largest scratch the documented limits allow: N at its maximum, FP64 (8^3 bricks, 32-byte
        # records), order 8, the maximum particle count
        (B.NOALLOC_MAX_N, 8, "f64", L, synth.uniform_particles(B.NOALLOC_MAX_PARTICLES, seed=10), 34),
    ]
    for N, order, dtype, Lc, xs, seed in cases:
        x = torch.from_numpy(xs).cuda()
        plan, coef, u_ref, g_ref = plan_path(B, N, order, dtype, Lc, x, seed)
        u, g = noalloc(B, coef, N, order, dtype, Lc, x, plan.out_dtype)
        tu, tg = TOL[dtype]
        assert normwise(u, u_ref) <= tu and normwise(g, g_ref) <= tg, (N, order, dtype)
        # the same call again on the same scratch
        u2, g2 = noalloc(B, coef, N, order, dtype, Lc, x, plan.out_dtype)
        assert normwise(u2, u_ref) <= tu and normwise(g2, g_ref) <= tg, (N, order, dtype)
        plan.close()


def test_noalloc_call_changes_no_device_allocation(B):
    """After a first call (which loads the library's kernels and its fixed array), a call leaves the
    device's free memory and torch's allocated bytes exactly as they were."""
    N, order = 32, 4
    x = torch.from_numpy(synth.uniform_particles(20000, seed=12)).cuda()
    plan, coef, u_ref, g_ref = plan_path(B, N, order, "f32", 2.0 * math.pi, x, 35)
    u = torch.empty_like(u_ref)
    g = torch.empty_like(g_ref)
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        rc = B.bspline_interp_noalloc(coef.data_ptr(), N, order, B.F32, 2.0 * math.pi, x.data_ptr(), x.shape[0],
                                      u.data_ptr(), g.data_ptr(), 0, stream)
        assert rc == B.OK
        torch.cuda.synchronize()

    call()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0
    assert normwise(u, u_ref) <= TOL["f32"][0] and normwise(g, g_ref) <= TOL["f32"][1]
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(B):
    buf = torch.zeros(1 << 12, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    too_many = B.NOALLOC_MAX_PARTICLES + 1
    assert B.bspline_interp_noalloc(p, 32, 4, B.F32, 1.0, p, too_many, p, p, 0, 0) == B.ERR_TOO_LARGE
    assert B.bspline_interp_noalloc(p, 2 * B.NOALLOC_MAX_N, 4, B.F32, 1.0, p, 10, p, p, 0, 0) == B.ERR_TOO_LARGE
    assert B.bspline_interp_noalloc(p, 32, 4, B.F32, 1.0, p, 0, p, p, 0, 0) == B.OK
    assert "scratch" in B.status_string(B.ERR_TOO_LARGE)
