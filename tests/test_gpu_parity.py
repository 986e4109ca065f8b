"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (normwise per output quantity: max_p |gpu - oracle| / max_p |oracle|):
* F64 plans: 1e-12 (the target the method's FP64 path is held to);
* F32 plans: TOL32 below, derived from the FP32 arithmetic of the transform
  (~log2(N^3) rounding steps on values of the size of the coefficients) and
  of the n^3-term stencil sums with FP32 weights;
* BF16 plans: TOL16, dominated by the 2^-9 relative rounding of each stored
  coefficient (reported, not a precision claim).
The FP32 form is also held to the statistical bar of the method: its error
against the FP64 oracle stays below the interpolation's own truncation error.
"""
import math

import numpy as np
import pytest

from oracle import bspline_oracle as O
from paper_1201_4060_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = 2.0 * math.pi
TOL64 = 1e-12
TOL32 = {"u": 2e-5, "grad": 5e-5}
TOL16 = {"u": 2e-2, "grad": 5e-2}


@pytest.fixture(scope="module")
def B():
    from paper_1201_4060_gb300 import _build
    _build.build()
    from paper_1201_4060_gb300 import bspline
    assert torch.cuda.is_available()
    return bspline


def normwise(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def gpu_path(B, half, x, N, order, dtype, prefilter="interp", grad=True):
    plan = B.Plan(N, order, dtype, prefilter=prefilter)
    uh = torch.from_numpy(np.ascontiguousarray(half)).to(plan.uhat_dtype).cuda()
    coef = plan.coeffs(uh)
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    res = plan.interp(coef, xt, grad=grad)
    nonfinite = plan.status()
    torch.cuda.synchronize()
    c = coef.float().cpu().numpy() if dtype == "bf16" else coef.cpu().numpy()
    if grad:
        u, g = res
        return c, u.cpu().numpy(), g.cpu().numpy(), nonfinite
    return c, res.cpu().numpy(), None, nonfinite


def rounded_input(half, dtype):
    return half if dtype == "f64" else half.astype(np.complex64).astype(np.complex128)


# ----------------------------------------------------------------------- coefficients

@pytest.mark.parametrize("N", [8, 16, 32, 64])
@pytest.mark.parametrize("order", [2, 3, 4, 6, 8])
def test_coeffs_f64(B, N, order):
    half = synth.random_half_spectrum(N, seed=N + order, hermitian=True)
    x = synth.uniform_particles(64, seed=1)
    c, _, _, _ = gpu_path(B, half, x, N, order, "f64")
    ref = O.coefficients(half, order)
    assert normwise(c, ref) < TOL64


@pytest.mark.parametrize("N", [8, 32, 128])
def test_coeffs_f64_non_hermitian_input_follows_c2r_semantics(B, N):
    half = synth.random_half_spectrum(N, seed=3, hermitian=False)
    c, _, _, _ = gpu_path(B, half, synth.uniform_particles(8, 2), N, 4, "f64")
    assert normwise(c, O.coefficients(half, 4)) < TOL64


@pytest.mark.parametrize("order", [3, 4, 6])
def test_coeffs_l2_prefilter_f64(B, order):
    N = 32
    half = synth.kolmogorov_field(N, seed=7).dense()
    c, _, _, _ = gpu_path(B, half, synth.uniform_particles(8, 2), N, order, "f64", prefilter="l2")
    assert normwise(c, O.coefficients(half, order, kind="l2")) < TOL64


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("N", [32, 256])
def test_coeffs_reduced_precision(B, dtype, N):
    half = synth.kolmogorov_field(N, seed=11).dense()
    c, _, _, _ = gpu_path(B, half.astype(np.complex64), synth.uniform_particles(8, 2), N, 6, dtype)
    err = normwise(c, O.coefficients(rounded_input(half, dtype), 6))
    assert err < (2e-6 if dtype == "f32" else 4e-3), err


# ----------------------------------------------------------------------- interpolation

def test_parity_32cubed_cubic_f64(B):
    """Plain method, FP64: 32^3 Kolmogorov field, order 4, 10^4 uniform particles."""
    wl = synth.WORKLOADS["parity32"]
    N, order = wl["N"], wl["order"]
    half = synth.kolmogorov_field(N, seed=wl["field_seed"]).dense()
    x = synth.uniform_particles(wl["P"], seed=wl["particle_seed"])
    _, u, g, nf = gpu_path(B, half, x, N, order, "f64")
    ru, rg = O.interpolate(half, x, order)
    assert nf == 0
    for c in range(3):
        assert normwise(u[:, c], ru[:, c]) < TOL64
        for d in range(3):
            assert normwise(g[:, c, d], rg[:, c, d]) < TOL64


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("N", [8, 16, 64])
def test_interp_f64_orders_and_sizes(B, order, N):
    half = synth.kolmogorov_field(N, seed=order).dense()
    rng = np.random.default_rng(order * 100 + N)
    x = rng.uniform(-L, 2 * L, (3001, 3))                   # outside [0, L) too, ragged count
    _, u, g, nf = gpu_path(B, half, x, N, order, "f64")
    ru, rg = O.interpolate(half, x, order)
    assert nf == 0
    assert normwise(u, ru) < TOL64
    assert normwise(g, rg) < TOL64


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_interp_reduced_precision(B, dtype, order):
    N = 64
    half = synth.kolmogorov_field(N, seed=21).dense().astype(np.complex64)
    x = synth.clustered_particles(20000, seed=5)
    _, u, g, nf = gpu_path(B, half, x, N, order, dtype)
    ru, rg = O.interpolate(rounded_input(half.astype(np.complex128), dtype), x, order)
    tol = TOL32 if dtype == "f32" else TOL16
    assert nf == 0
    assert normwise(u, ru) < tol["u"], normwise(u, ru)
    assert normwise(g, rg) < tol["grad"], normwise(g, rg)


def test_no_grad_flag_matches(B):
    N, order = 32, 6
    half = synth.kolmogorov_field(N, seed=3).dense()
    x = synth.uniform_particles(5000, seed=9)
    _, u1, _, _ = gpu_path(B, half, x, N, order, "f64", grad=False)
    ru, _ = O.interpolate(half, x, order)
    assert normwise(u1, ru) < TOL64


# ----------------------------------------------------------------------- edge cases

def test_edge_cases_f64(B):
    N, order = 16, 4
    half = synth.kolmogorov_field(N, seed=4).dense()
    h = L / N
    pts = [
        [0.0, 0.0, 0.0],                     # on a node, t = 0
        [h, 2 * h, 3 * h],                   # on nodes
        [L, L, L],                           # the far corner wraps to 0
        [-1e-13, 1e-13, L - 1e-13],          # just across the periodic seam
        [-7.5 * L, 3.25 * L, 1e3],           # far outside, still many fractional bits
        [0.5 * h, 0.5 * h, 0.5 * h],
    ]
    # many particles in a single cell and in a single brick, plus a ragged count
    rng = np.random.default_rng(0)
    pts += (np.array([3.3, 4.4, 5.5]) * h + rng.uniform(0, h, (777, 3))).tolist()
    x = np.array(pts)
    _, u, g, nf = gpu_path(B, half, x, N, order, "f64")
    ru, rg = O.interpolate(half, x, order)
    assert nf == 0
    assert normwise(u, ru) < TOL64
    assert normwise(g, rg) < TOL64


@pytest.mark.parametrize("order", [4, 5])
def test_edge_cases_f32(B, order):
    """FP32 plans locate particles from an integer product of the significands of x and N/L
    (no FP64 multiply); positions on nodes, on the seam, far outside, tiny and negative."""
    N = 16
    half = synth.kolmogorov_field(N, seed=4).dense().astype(np.complex64).astype(np.complex128)
    h = L / N
    pts = [
        [0.0, 0.0, 0.0],
        [h, 2 * h, 3 * h],
        [L, L, L],
        [-1e-13, 1e-13, L - 1e-13],
        [-7.5 * L, 3.25 * L, 1e3],
        [0.5 * h, 0.5 * h, 0.5 * h],
        [1e-30, 5e-324, 2.0 ** -70],
        [np.nextafter(h, 0.0), np.nextafter(h, 1.0), 7 * h],
        [1e6, -1e6, 123.456],
    ]
    rng = np.random.default_rng(1)
    pts += rng.uniform(-3 * L, 4 * L, (500, 3)).tolist()
    x = np.array(pts)
    _, u, g, nf = gpu_path(B, half, x, N, order, "f32")
    ru, rg = O.interpolate(half, x, order)
    assert nf == 0
    assert normwise(u, ru) < TOL32["u"]
    assert normwise(g, rg) < TOL32["grad"]


def test_nonfinite_positions_f32(B):
    N, order = 16, 6
    half = synth.kolmogorov_field(N, seed=4).dense().astype(np.complex64).astype(np.complex128)
    x = synth.uniform_particles(100, seed=3)
    x[5, 0] = np.nan
    x[17, 2] = np.inf
    x[42, 1] = -np.inf
    x[60, 1] = 1e300
    x[61, 0] = -1e300
    x[62, 2] = 2.0 ** 60                      # no fraction bits left at FP64 precision
    _, u, g, nf = gpu_path(B, half, x, N, order, "f32")
    bad = [5, 17, 42, 60, 61, 62]
    assert nf == len(bad)
    assert np.all(np.isnan(u[bad])) and np.all(np.isnan(g[bad]))
    good = np.setdiff1d(np.arange(100), bad)
    ru, rg = O.interpolate(half, x[good], order)
    assert normwise(u[good], ru) < TOL32["u"]
    assert normwise(g[good], rg) < TOL32["grad"]


def test_nonfinite_positions_give_nan_and_status(B):
    N, order = 16, 4
    half = synth.kolmogorov_field(N, seed=4).dense()
    x = synth.uniform_particles(100, seed=3)
    x[5, 0] = np.nan
    x[17, 2] = np.inf
    x[42, 1] = -np.inf
    x[60, 1] = 1e300                        # finite but beyond any fractional resolution
    _, u, g, nf = gpu_path(B, half, x, N, order, "f64")
    bad = [5, 17, 42, 60]
    assert nf == len(bad)
    assert np.all(np.isnan(u[bad])) and np.all(np.isnan(g[bad]))
    good = np.setdiff1d(np.arange(100), bad)
    ru, rg = O.interpolate(half, x[good], order)
    assert normwise(u[good], ru) < TOL64
    assert normwise(g[good], rg) < TOL64


def test_zero_and_one_particle(B):
    N, order = 16, 6
    half = synth.kolmogorov_field(N, seed=5).dense()
    plan = B.Plan(N, order, "f64")
    coef = plan.coeffs(torch.from_numpy(half).cuda())
    x0 = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    u0, g0 = plan.interp(coef, x0)
    assert u0.shape == (0, 3) and g0.shape == (0, 3, 3)
    x1 = np.array([[1.0, 2.0, 3.0]])
    u1, g1 = plan.interp(coef, torch.from_numpy(x1).cuda())
    ru, rg = O.interpolate(half, x1, order)
    assert normwise(u1.cpu().numpy(), ru) < TOL64
    assert normwise(g1.cpu().numpy(), rg) < TOL64


def test_abi_rejects_bad_arguments_on_gpu(B):
    plan = B.Plan(16, 4, "f32")
    h = plan.handle
    assert B.bspline_interp(h, 0, 0, 10, 0, 0, 0) == B.ERR_INVALID_ARG
    buf = torch.empty(1 << 16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert B.bspline_interp(h, p, p + 4, 10, p, p, 0) == B.ERR_INVALID_ARG       # misaligned x
    assert B.bspline_interp(h, p, p, -1, p, p, 0) == B.ERR_INVALID_ARG
    assert B.bspline_interp(h, p, p, 10, p, 0, 0) == B.ERR_INVALID_ARG           # grad NULL without flag
    assert B.bspline_interp(h, p, p, 10, p, p, 0x80) == B.ERR_INVALID_ARG        # unknown flag
    assert B.bspline_coeffs(h, p, p) == B.ERR_INVALID_ARG                        # aliasing
    assert B.bspline_spread_adjoint(h, p, p, 10, p, p, 0, p, 0) == B.ERR_INVALID_ARG   # g_u_hat without g_coeffs
    assert B.bspline_plan_set_length(h, -1.0) == B.ERR_INVALID_ARG


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_transform_wait_timeout_is_reported_and_context_survives(B, dtype):
    """A bounded wait of the transform runs out (its producer signals are dropped by a test hook):
    bspline_status reports TIMEOUT, and the next transform on the same plan is correct."""
    N, order = 64, 4
    half = synth.kolmogorov_field(N, seed=13).dense()
    plan = B.Plan(N, order, dtype)
    uh = torch.from_numpy(half).to(plan.uhat_dtype).cuda()
    plan.set_test_hooks(B.TEST_DROP_TRANSFORM_SIGNALS)
    plan.coeffs(uh)
    rc, _ = B.bspline_status(plan.handle)
    assert rc == B.ERR_TIMEOUT
    plan.set_test_hooks(0)
    coef = plan.coeffs(uh)
    rc, _ = B.bspline_status(plan.handle)
    assert rc == B.OK
    ref = O.coefficients(rounded_input(half, dtype), order)
    assert normwise(coef.double().cpu().numpy(), ref) < (TOL64 if dtype == "f64" else 2e-6)


def test_tile_wait_timeout_gives_nan_and_status_and_context_survives(B):
    """A TMA tile wait runs out (a test hook arms the tile's barrier but issues no copy): the particles of
    that tile get NaN outputs (NaN position gradients in the adjoint), bspline_status reports TIMEOUT,
    particles of tiles staged by cp.async on the periodic seams are still right, and the next call
    without the hook is correct everywhere with an OK status."""
    N, order = 64, 4
    half = synth.kolmogorov_field(N, seed=17).dense()
    h = L / N
    # a few particles of the interior brick (16..31, 12..23, 16..31): stencil origin floor(s) - 1 there, so TMA
    inner = np.array([[20.3, 14.6, 21.2], [25.9, 18.1, 30.4], [17.5, 22.7, 17.05]]) * h
    # and a few of a seam brick (x from 48): staged by cp.async
    seam = np.array([[55.2, 5.4, 3.3], [61.7, 60.2, 62.9]]) * h
    xs = np.concatenate([inner, seam])
    plan = B.Plan(N, order, "f32")
    coef = plan.coeffs(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
    plan.set_gather_split(0)
    x = torch.from_numpy(xs).cuda()
    ru, rg = O.interpolate(rounded_input(half, "f32"), xs, order)
    plan.set_test_hooks(B.TEST_SKIP_TMA_ISSUE)
    u, g = plan.interp(coef, x)
    rc, _ = B.bspline_status(plan.handle)
    assert rc == B.ERR_TIMEOUT
    u, g = u.cpu().numpy(), g.cpu().numpy()
    ni = len(inner)
    assert np.isnan(u[:ni]).all() and np.isnan(g[:ni]).all()
    assert normwise(u[ni:], ru[ni:]) < TOL32["u"] and normwise(g[ni:], rg[ni:]) < TOL32["grad"]
    # the adjoint's position gradient stages its tiles the same way
    gu = torch.ones((len(xs), 3), dtype=torch.float32, device="cuda")
    _, g_x, _ = plan.spread_adjoint(x, g_u=gu, coef=coef, u_hat_grad=False)
    rc, _ = B.bspline_status(plan.handle)
    assert rc == B.ERR_TIMEOUT
    gx_bad = g_x.cpu().numpy()
    assert np.isnan(gx_bad[:ni]).all() and np.isfinite(gx_bad[ni:]).all()
    plan.set_test_hooks(0)
    u, g = plan.interp(coef, x)
    assert plan.status() == 0
    assert normwise(u.cpu().numpy(), ru) < TOL32["u"] and normwise(g.cpu().numpy(), rg) < TOL32["grad"]
    _, g_x, _ = plan.spread_adjoint(x, g_u=gu, coef=coef, u_hat_grad=False)
    assert plan.status() == 0
    assert np.isfinite(g_x.cpu().numpy()).all()
    assert np.allclose(g_x.cpu().numpy()[ni:], gx_bad[ni:], rtol=0, atol=0)


def test_run_host_matches_device_path(B):
    N, order = 32, 4
    half = synth.kolmogorov_field(N, seed=8).dense().astype(np.complex64)
    x = synth.uniform_particles(4096, seed=8)
    _, u, g, _ = gpu_path(B, half, x, N, order, "f32")
    plan = B.Plan(N, order, "f32")
    uh = torch.from_numpy(half).pin_memory()
    xh = torch.from_numpy(x).pin_memory()
    uo = torch.empty((4096, 3), dtype=torch.float32).pin_memory()
    go = torch.empty((4096, 3, 3), dtype=torch.float32).pin_memory()
    plan.run_host(uh, xh, uo, go)
    assert np.array_equal(uo.numpy(), u) and np.array_equal(go.numpy(), g)
    # again on the same plan (buffers and the second stream are reused), u only, with a non-finite position
    x2 = x.copy()
    x2[7, 1] = np.nan
    uo2 = torch.full((4096, 3), 5.0, dtype=torch.float32).pin_memory()
    plan.run_host(uh, torch.from_numpy(x2).pin_memory(), uo2, None)
    assert plan.status() == 1
    ok = np.ones(4096, bool)
    ok[7] = False
    assert np.isnan(uo2.numpy()[7]).all()
    assert np.array_equal(uo2.numpy()[ok], u[ok])


def test_run_host_async_on_alternating_plans(B):
    """Steps queued with bspline_run_host_async on two plans (two streams) and collected with
    bspline_wait give the synchronous results; a plan that has run nothing waits at once."""
    N, order, P = 32, 6, 5000
    fields = [synth.kolmogorov_field(N, seed=30 + k).dense().astype(np.complex64) for k in range(4)]
    xs = [synth.clustered_particles(P, seed=40 + k) for k in range(4)]
    ref = []
    for k in range(4):
        _, u, g, _ = gpu_path(B, fields[k], xs[k], N, order, "f32")
        ref.append((u, g))
    plans = [B.Plan(N, order, "f32") for _ in range(2)]
    plans[1].wait()
    streams = [torch.cuda.Stream() for _ in range(2)]
    uh = [torch.from_numpy(f).pin_memory() for f in fields]
    xh = [torch.from_numpy(x).pin_memory() for x in xs]
    outs = [(torch.full((P, 3), np.nan, dtype=torch.float32).pin_memory(),
             torch.full((P, 3, 3), np.nan, dtype=torch.float32).pin_memory()) for _ in range(4)]
    for k in range(4):
        i = k % 2
        plans[i].wait()
        plans[i].run_host(uh[k], xh[k], *outs[k], stream=streams[i], wait=False)
    for p in plans:
        p.wait()
    for k in range(4):
        assert np.array_equal(outs[k][0].numpy(), ref[k][0]) and np.array_equal(outs[k][1].numpy(), ref[k][1])


@pytest.mark.parametrize("dtype,N,order", [("f32", 48, 6), ("f64", 32, 5), ("bf16", 64, 4)])
def test_eval_matches_coeffs_then_interp(B, dtype, N, order):
    """bspline_eval (sort on the second stream, overlapping the transform) gives the
    two-call results bit for bit, call after call on one plan, also u only and with
    a non-finite position; the FP64 case is held to the oracle too."""
    half = synth.kolmogorov_field(N, seed=21).dense()
    x = synth.clustered_particles(20000, seed=21)
    c_ref, u_ref, g_ref, _ = gpu_path(B, half, x, N, order, dtype)
    plan = B.Plan(N, order, dtype)
    uh = torch.from_numpy(half).to(plan.uhat_dtype).cuda()
    xt = torch.from_numpy(x).cuda()
    for _ in range(3):
        coef, u, g = plan.eval(uh, xt)
        assert plan.status() == 0
        c = coef.float().cpu().numpy() if dtype == "bf16" else coef.cpu().numpy()
        assert np.array_equal(c, c_ref)
        assert np.array_equal(u.cpu().numpy(), u_ref) and np.array_equal(g.cpu().numpy(), g_ref)
    if dtype == "f64":
        ru, rg = O.interpolate(half, x, order)
        assert normwise(u_ref, ru) < TOL64 and normwise(g_ref, rg) < TOL64
    x2 = x.copy()
    x2[11, 2] = np.inf
    coef2, u2 = plan.eval(uh, torch.from_numpy(x2).cuda(), coef=coef, grad=False)
    assert plan.status() == 1
    ok = np.ones(len(x), bool)
    ok[11] = False
    u2 = u2.cpu().numpy()
    assert np.isnan(u2[11]).all() and np.array_equal(u2[ok], u_ref[ok])
    # no particles: only the transform runs
    coef3, u3, g3 = plan.eval(uh, torch.empty((0, 3), dtype=torch.float64, device="cuda"))
    assert u3.shape == (0, 3) and g3.shape == (0, 3, 3)
    c3 = coef3.float().cpu().numpy() if dtype == "bf16" else coef3.cpu().numpy()
    assert np.array_equal(c3, c_ref)


@pytest.mark.parametrize("N,order,P", [(32, 6, 400000), (256, 4, 600000)])
def test_eval_grid_stride_sort_matches_coeffs_then_interp(B, N, order, P):
    """Beside the transform the sort runs as a bounded grid (two CTAs per SM) whose threads loop over the
    particles; with more particles than that grid's threads it must give the two-call results bit for
    bit: 12 bricks (warp-aggregated counters) and 5632 bricks (one atomic per particle)."""
    half = synth.kolmogorov_field(N, seed=31).dense()
    plan = B.Plan(N, order, "f32")
    uh = torch.from_numpy(half).to(plan.uhat_dtype).cuda()
    x = synth.clustered_particles(P, seed=32)
    x[7, 0] = np.nan
    xt = torch.from_numpy(x).cuda()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert P > 2 * sms * 256 * 1.5
    coef = plan.coeffs(uh)
    u_ref, g_ref = plan.interp(coef, xt)
    for _ in range(2):
        coef2, u, g = plan.eval(uh, xt)
        assert plan.status() == 1
        assert torch.equal(coef2, coef)
        assert torch.equal(torch.nan_to_num(u, 7.0), torch.nan_to_num(u_ref, 7.0))
        assert torch.equal(torch.nan_to_num(g, 7.0), torch.nan_to_num(g_ref, 7.0))
    assert torch.isnan(u[7]).all()


def test_eval_rejects_bad_arguments(B):
    plan = B.Plan(16, 4, "f32")
    h = plan.handle
    buf = torch.empty(1 << 18, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    q = p + (1 << 20)
    assert B.bspline_eval(h, p, p, q, 10, q, q, 0) == B.ERR_INVALID_ARG          # coeffs alias u_hat
    assert B.bspline_eval(h, p + 8, q, q, 10, q, q, 0) == B.ERR_INVALID_ARG      # misaligned u_hat
    assert B.bspline_eval(h, p, q, q + 4, 10, q, q, 0) == B.ERR_INVALID_ARG      # misaligned x
    assert B.bspline_eval(h, p, q, 0, 10, q, q, 0) == B.ERR_INVALID_ARG          # x NULL with P > 0
    assert B.bspline_eval(h, p, q, q, 10, q, 0, 0) == B.ERR_INVALID_ARG          # grad NULL without flag
    assert B.bspline_eval(h, p, q, q, -1, q, q, 0) == B.ERR_INVALID_ARG
    assert B.bspline_eval(h, p, q, q, 10, q, q, 0x80) == B.ERR_INVALID_ARG       # unknown flag


@pytest.mark.parametrize("dtype,N,order", [("f32", 16, 4), ("f32", 32, 6), ("f32", 48, 3), ("f32", 32, 8),
                                           ("bf16", 32, 5), ("bf16", 16, 2)])
def test_direct_and_staged_gathers_agree_bit_for_bit(B, dtype, N, order):
    """The gather split only moves bricks between the staged gather (tile in shared memory) and the
    direct one (stencils from global memory): same bits for every split, positions on the periodic
    seams included; and the result holds against the oracle."""
    half = synth.kolmogorov_field(N, seed=50 + order).dense()
    rng = np.random.default_rng(order)
    h = L / N
    x = np.concatenate([
        synth.uniform_particles(300, seed=order),                              # sparse bricks
        np.array([2.5, 1.5, 3.5]) * h * 4 + rng.uniform(0, 2 * h, (700, 3)),  # one dense clump
        np.column_stack([rng.uniform(0, L, 64), rng.uniform(0, L, 64),          # near the z, y and x seams
                         L - rng.uniform(0, 3 * h, 64)]),
        np.column_stack([L - rng.uniform(0, 3 * h, 64), L - rng.uniform(0, 3 * h, 64),
                         rng.uniform(0, L, 64)]),
    ])
    plan = B.Plan(N, order, dtype)
    uh = torch.from_numpy(half).to(plan.uhat_dtype).cuda()
    coef = plan.coeffs(uh)
    xt = torch.from_numpy(x).cuda()
    outs = []
    for split in (0, 8, 100, 2 ** 32 - 1, B.GATHER_SPLIT_AUTO):
        plan.set_gather_split(split)
        u, g = plan.interp(coef, xt)
        outs.append((u.cpu().numpy(), g.cpu().numpy()))
    for u, g in outs[1:]:
        assert np.array_equal(u, outs[0][0]) and np.array_equal(g, outs[0][1])
    plan.set_gather_split(2 ** 32 - 1)
    u, g = plan.interp(coef, xt, grad=True)
    u1 = plan.interp(coef, xt, grad=False)
    assert np.array_equal(u1.cpu().numpy(), outs[0][0])
    tol = TOL32 if dtype == "f32" else TOL16
    ru, rg = O.interpolate(rounded_input(half, "f32"), x, order)
    assert normwise(outs[0][0], ru) < tol["u"] and normwise(outs[0][1], rg) < tol["grad"]


@pytest.mark.parametrize("N,order,dtype", [(64, 6, "f32"), (96, 4, "f32"), (64, 8, "f32"), (128, 3, "f32"),
                                           (64, 6, "bf16"), (96, 5, "bf16"), (64, 8, "bf16")])
def test_tma_and_cp_async_staging_agree_bit_for_bit(B, N, order, dtype):
    """Bricks away from the periodic seams are staged by TMA tensor copies (FP32 tiles; the first copy
    of a BF16 pair tile), the others (and all of them with BSPLINE_TEST_NO_TMA) by cp.async: the same
    tile, so the same bits."""
    half = synth.kolmogorov_field(N, seed=70 + order).dense()
    x = torch.from_numpy(synth.clustered_particles(30000, seed=71)).cuda()
    plan = B.Plan(N, order, dtype)
    coef = plan.coeffs(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
    plan.set_gather_split(0)                              # every brick staged
    u_t, g_t = plan.interp(coef, x)
    plan.set_test_hooks(B.TEST_NO_TMA)
    u_c, g_c = plan.interp(coef, x)
    plan.set_test_hooks(0)
    assert plan.status() == 0
    assert torch.equal(u_t, u_c) and torch.equal(g_t, g_c)
    ru, rg = O.interpolate(rounded_input(half, "f32"), x.cpu().numpy(), order)
    tol = TOL32 if dtype == "f32" else TOL16
    assert normwise(u_t.cpu().numpy(), ru) < tol["u"] and normwise(g_t.cpu().numpy(), rg) < tol["grad"]


def brick_keys(x, N, order, dtype):
    """Brick key of each particle from the oracle's locate (first stencil node, Eq. alg-int-6), bricks of
    16 x 12 x 16 cells (16 x 8 x 16 above order 6; 8^3 for FP64) in x-major order; -1 for non-finite."""
    bx, by = (8, 8) if dtype == "f64" else (16, 12 if order <= 6 else 8)
    nbx, nby = -(-N // bx), -(-N // by)
    ok = np.isfinite(x).all(axis=1)
    nodes, _ = O.locate(np.where(ok[:, None], x, 0.0), N, order)
    a = nodes[:, :, 0]
    key = ((a[:, 0] // bx) * nby + a[:, 1] // by) * nbx + a[:, 2] // bx
    return np.where(ok, key, -1)


@pytest.mark.parametrize("dtype,N,order", [("f32", 64, 6), ("f32", 96, 4), ("bf16", 64, 8), ("f64", 32, 4),
                                           ("f32", 16, 3)])
def test_sorted_flag_bit_equal_to_unsorted_and_oracle(B, dtype, N, order):
    """bspline_sort_order gives a permutation in brick order (keys from the oracle's locate); positions
    permuted by it and passed with BSPLINE_INTERP_SORTED give the same bits as the sorting call, and match
    the oracle; with the promise broken (unsorted input) the flagged call still gives the same bits."""
    half = synth.kolmogorov_field(N, seed=80 + order).dense()
    xs = synth.clustered_particles(20000, seed=81)
    plan = B.Plan(N, order, dtype)
    coef = plan.coeffs(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
    x = torch.from_numpy(xs).cuda()
    perm = plan.sort_order(x).long()
    pm = perm.cpu().numpy()
    assert np.array_equal(np.sort(pm), np.arange(len(xs)))
    keys = brick_keys(xs, N, order, dtype)[pm]
    assert (np.diff(keys) >= 0).all()
    xp = x[perm].contiguous()
    u_s, g_s = plan.interp(coef, xp, sorted=True)
    assert plan.status() == 0
    u_r, g_r = plan.interp(coef, xp)
    assert torch.equal(u_s, u_r) and torch.equal(g_s, g_r)
    # promise broken: the flagged call sorts after all
    u_b, g_b = plan.interp(coef, x, sorted=True)
    u_n, g_n = plan.interp(coef, x)
    assert torch.equal(u_b, u_n) and torch.equal(g_b, g_n)
    assert torch.equal(u_b[perm], u_s) and torch.equal(g_b[perm], g_s)
    ru, rg = O.interpolate(rounded_input(half, dtype), xp.cpu().numpy(), order)
    tol = {"f64": (TOL64, TOL64), "f32": (TOL32["u"], TOL32["grad"]), "bf16": (TOL16["u"], TOL16["grad"])}[dtype]
    assert normwise(u_s.cpu().numpy(), ru) < tol[0] and normwise(g_s.cpu().numpy(), rg) < tol[1]


def test_sorted_flag_with_nonfinite_tail_and_eval(B):
    """Sorted positions with non-finite ones last (where bspline_sort_order puts them): NaN outputs and the
    count in the status word; bspline_eval with the flag gives the interp call's bits."""
    N, order = 64, 4
    half = synth.kolmogorov_field(N, seed=90).dense()
    xs = synth.uniform_particles(5000, seed=91)
    xs[[7, 100, 4000]] = [[np.nan, 1.0, 1.0], [1.0, np.inf, 2.0], [0.5, 0.5, -np.inf]]
    plan = B.Plan(N, order, "f32")
    uh = torch.from_numpy(half).to(plan.uhat_dtype).cuda()
    coef = plan.coeffs(uh)
    x = torch.from_numpy(xs).cuda()
    perm = plan.sort_order(x).long()
    pm = perm.cpu().numpy()
    assert set(pm[-3:].tolist()) == {7, 100, 4000}
    xp = x[perm].contiguous()
    u_s, g_s = plan.interp(coef, xp, sorted=True)
    assert plan.status() == 3
    assert torch.isnan(u_s[-3:]).all() and torch.isnan(g_s[-3:]).all()
    assert torch.isfinite(u_s[:-3]).all() and torch.isfinite(g_s[:-3]).all()
    u_r, g_r = plan.interp(coef, xp)
    assert torch.equal(u_s[:-3], u_r[:-3]) and torch.equal(g_s[:-3], g_r[:-3])
    _, u_e, g_e = plan.eval(uh, xp, sorted=True)
    assert plan.status() == 3
    assert torch.equal(u_e[:-3], u_s[:-3]) and torch.equal(g_e[:-3], g_s[:-3])
    ru, rg = O.interpolate(rounded_input(half, "f32"), xp[:-3].cpu().numpy(), order)
    assert normwise(u_s[:-3].cpu().numpy(), ru) < TOL32["u"] and normwise(g_s[:-3].cpu().numpy(), rg) < TOL32["grad"]


def test_outputs_only_4_byte_aligned(B):
    """Outputs may start on any 4-byte boundary: the gather's 8-byte stores are used only on 8-byte
    aligned arrays, with the same results either way."""
    N, order, P = 64, 6, 20000
    half = synth.kolmogorov_field(N, seed=80).dense()
    plan = B.Plan(N, order, "f32")
    coef = plan.coeffs(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
    x = torch.from_numpy(synth.clustered_particles(P, seed=81)).cuda()
    plan.set_gather_split(0)
    u_ref, g_ref = plan.interp(coef, x)
    ub = torch.full((3 * P + 1,), float("nan"), device="cuda")
    gb = torch.full((9 * P + 1,), float("nan"), device="cuda")
    u_off, g_off = ub[1:].view(P, 3), gb[1:].view(P, 3, 3)
    assert u_off.data_ptr() % 8 == 4 and g_off.data_ptr() % 8 == 4
    plan.interp(coef, x, u_off, g_off)
    torch.cuda.synchronize()
    assert torch.equal(u_off, u_ref) and torch.equal(g_off, g_ref)


def test_gather_autotune_and_its_cache(B, tmp_path, monkeypatch):
    N, order, P = 32, 6, 4000
    half = synth.kolmogorov_field(N, seed=60).dense()
    x = torch.from_numpy(synth.uniform_particles(P, seed=61)).cuda()
    cache = tmp_path / "autotune.jsonl"
    monkeypatch.setenv("BSPLINE_AUTOTUNE_CACHE", str(cache))
    plan = B.Plan(N, order, "f32")
    coef = plan.coeffs(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
    split, ms = plan.autotune(coef, x)
    assert split in (0, 8, 32, 128, 512, 2 ** 32 - 1) and ms > 0
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and f'"direct_below": {split}' in lines[0] and "|N32|o6|f32|p2^12" in lines[0]
    u_tuned, g_tuned = plan.interp(coef, x)
    plan2 = B.Plan(N, order, "f32")
    split2, ms2 = plan2.autotune(coef, x)                # taken from the cache, no timing
    assert split2 == split and ms2 == 0
    assert len(cache.read_text().splitlines()) == 1
    u2, g2 = plan2.interp(coef, x)
    assert torch.equal(u_tuned, u2) and torch.equal(g_tuned, g2)
    assert B.lib().bspline_plan_autotune(plan.handle, 0, 0, P, 0, 0, None, None) == B.ERR_INVALID_ARG


def test_custom_domain_length(B):
    N, order, Lc = 16, 4, 3.0
    half = synth.kolmogorov_field(N, seed=12).dense()
    x = np.random.default_rng(1).uniform(0, Lc, (500, 3))
    plan = B.Plan(N, order, "f64", L=Lc)
    coef = plan.coeffs(torch.from_numpy(half).cuda())
    u, g = plan.interp(coef, torch.from_numpy(x).cuda())
    ru, rg = O.evaluate(O.coefficients(half, order), x, order, L=Lc)
    assert normwise(u.cpu().numpy(), ru) < TOL64
    assert normwise(g.cpu().numpy(), rg) < TOL64


# ----------------------------------------------------------------------- 3 * 2^k grids (radix-3 stage)

@pytest.mark.parametrize("N", [48, 96, 192])
@pytest.mark.parametrize("order", [2, 4, 6])
def test_radix3_grids_f64(B, N, order):
    half = synth.random_half_spectrum(N, seed=N + order, hermitian=False)
    x = np.random.default_rng(N).uniform(-L, 2 * L, (2001, 3))
    c, u, g, nf = gpu_path(B, half, x, N, order, "f64")
    assert normwise(c, O.coefficients(half, order)) < TOL64
    ru, rg = O.interpolate(half, x, order)
    assert nf == 0
    assert normwise(u, ru) < TOL64
    assert normwise(g, rg) < TOL64


@pytest.mark.parametrize("N", [48, 192])
def test_radix3_grids_f32(B, N):
    half = synth.kolmogorov_field(N, seed=7).dense().astype(np.complex64)
    x = synth.clustered_particles(20000, seed=8)
    _, u, g, nf = gpu_path(B, half, x, N, 4, "f32")
    ru, rg = O.interpolate(half.astype(np.complex128), x, 4)
    assert nf == 0
    assert normwise(u, ru) < TOL32["u"]
    assert normwise(g, rg) < TOL32["grad"]
