"""GPU checks at the workloads' full sizes.

* 256^3, orders 2/4/6/8, 10^6 cell-sorted uniform particles: the FP32 form's
  error against the FP64 oracle (E_prec) stays below the method's truncation
  error (E_trunc), both normalised by the RMS of the quantity; the FP64 form
  matches the oracle to 1e-12 on sampled particles.
* 512^3, order 6, 2^24 clustered particles (the benchmark's launch
  configuration): sampled outputs of the FP32, BF16 and FP64 forms match the
  oracle, computed particle by particle from the oracle's full-size FP64
  coefficients (FP64 to 1e-12).
"""
import math

import numpy as np
import pytest

from oracle import bspline_oracle as O
from paper_1201_4060_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = 2.0 * math.pi


@pytest.fixture(scope="module")
def B():
    from paper_1201_4060_gb300 import _build
    _build.build()
    from paper_1201_4060_gb300 import bspline
    return bspline


def normwise(a, b):
    return np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max()


def rms_rel(a, b, ref):
    return math.sqrt(np.mean((np.asarray(a, np.float64) - b) ** 2) / np.mean(ref ** 2))


@pytest.fixture(scope="module")
def field256():
    wl = synth.WORKLOADS["orders256"]
    F = synth.kolmogorov_field(wl["N"], seed=wl["field_seed"])
    x = synth.make_particles(wl["particles"], wl["P"], wl["particle_seed"], wl["N"])
    sample = np.sort(np.random.default_rng(0).choice(wl["P"], 4000, replace=False))
    exact = O.direct_sum_modes(wl["N"], F.idx, F.val, x[sample[:256]])
    return wl, F, x, sample, exact


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_fp32_error_below_truncation_256(B, field256, order):
    wl, F, x, sample, (eu_ref, eg_ref) = field256
    N, P = wl["N"], wl["P"]
    xs = x[sample]
    xt = torch.from_numpy(x).cuda()
    res = {}
    for dtype in ("f64", "f32"):
        plan = B.Plan(N, order, dtype)
        uh = torch.zeros((3, N, N, N // 2 + 1), dtype=plan.uhat_dtype, device="cuda")
        idx = torch.from_numpy(F.idx).cuda()
        uh[:, idx[:, 0], idx[:, 1], idx[:, 2]] = torch.from_numpy(F.val).cuda().to(plan.uhat_dtype)
        coef = plan.coeffs(uh)
        u, g = plan.interp(coef, xt)
        assert plan.status() == 0
        st = torch.from_numpy(sample).cuda()
        res[dtype] = (u[st].double().cpu().numpy(), g[st].double().cpu().numpy())
        del uh, coef, u, g
        plan.close()
    half = F.dense()
    ou, og = O.evaluate(O.coefficients(half, order), xs, order)
    # FP64 parity on the sample
    assert normwise(res["f64"][0], ou) < 1e-12
    assert normwise(res["f64"][1], og) < 1e-12
    # truncation error: oracle vs the exact field (closed form of Section 5, cross-checked
    # against the direct trigonometric sum on the first 256 sampled particles)
    mse_u, mse_g = O.l2_error_field(N, F.idx, F.val, order)
    trunc_u = math.sqrt(mse_u.sum() / 3.0 / np.mean(ou ** 2))
    trunc_g = math.sqrt(mse_g.sum() / 9.0 / np.mean(og ** 2))
    ds_u = rms_rel(ou[:256], eu_ref, eu_ref)
    ds_g = rms_rel(og[:256], eg_ref, eg_ref)
    assert 0.5 < ds_u / trunc_u < 2.0 and 0.5 < ds_g / trunc_g < 2.0, (ds_u, trunc_u, ds_g, trunc_g)
    prec_u = rms_rel(res["f32"][0], ou, ou)
    prec_g = rms_rel(res["f32"][1], og, og)
    print(f"order {order}: E_trunc u {trunc_u:.3e} grad {trunc_g:.3e}; E_prec(FP32) u {prec_u:.3e} grad {prec_g:.3e}")
    assert prec_u < trunc_u and prec_g < trunc_g


def test_full_size_512_quintic_sampled_parity(B):
    wl = synth.WORKLOADS["throughput512"]
    N, order, P = wl["N"], wl["order"], wl["P"]
    F = synth.kolmogorov_field(N, seed=wl["field_seed"])
    x = synth.clustered_particles(P, seed=wl["particle_seed"])
    rng = np.random.default_rng(42)
    sample = np.sort(rng.choice(P, 1500, replace=False))
    got = {}
    xt = torch.from_numpy(x).cuda()
    for dtype in ("f32", "bf16", "f64"):
        plan = B.Plan(N, order, dtype)
        uh = torch.zeros((3, N, N, N // 2 + 1), dtype=plan.uhat_dtype, device="cuda")
        idx = torch.from_numpy(F.idx).cuda()
        uh[:, idx[:, 0], idx[:, 1], idx[:, 2]] = torch.from_numpy(F.val).cuda().to(plan.uhat_dtype)
        coef = plan.coeffs(uh)
        u, g = plan.interp(coef, xt)
        assert plan.status() == 0
        assert bool(torch.isfinite(u).all()) and bool(torch.isfinite(g).all())
        st = torch.from_numpy(sample).cuda()
        got[dtype] = (u[st].double().cpu().numpy(), g[st].double().cpu().numpy())
        del uh, coef, u, g
        plan.close()
        torch.cuda.empty_cache()
    def oracle_at_sample(field):
        ou = np.empty((sample.size, 3))
        og = np.empty((sample.size, 3, 3))
        for c in range(3):     # one component at a time keeps the oracle's host memory bounded
            half = np.zeros((1, N, N, N // 2 + 1), np.complex128)
            half[0, field.idx[:, 0], field.idx[:, 1], field.idx[:, 2]] = field.val[c]
            coef_c = O.coefficients(half, order)[0]
            cb = np.broadcast_to(coef_c, (3, N, N, N))
            uc, gc = O.evaluate(cb, x[sample], order)
            ou[:, c] = uc[:, 0]
            og[:, c, :] = gc[:, 0, :]
            del coef_c, cb, half
        return ou, og

    # FP32 and BF16 plans take a complex64 spectrum: held to the oracle of that rounded input
    ou, og = oracle_at_sample(F.rounded(np.complex64))
    eu32, eg32 = normwise(got["f32"][0], ou), normwise(got["f32"][1], og)
    eu16, eg16 = normwise(got["bf16"][0], ou), normwise(got["bf16"][1], og)
    # the FP64 form (the plain GPU path the FP32 form is compared with) on the exact input
    ou64, og64 = oracle_at_sample(F)
    eu64, eg64 = normwise(got["f64"][0], ou64), normwise(got["f64"][1], og64)
    print(f"512^3 quintic: FP32 normwise u {eu32:.2e} grad {eg32:.2e}; BF16 u {eu16:.2e} grad {eg16:.2e}; "
          f"FP64 u {eu64:.2e} grad {eg64:.2e}")
    assert eu32 < 2e-5 and eg32 < 5e-5
    assert eu16 < 2e-2 and eg16 < 5e-2
    assert eu64 < 1e-12 and eg64 < 1e-12


@pytest.mark.parametrize("N", [768, 1024])
def test_largest_grids_against_direct_sum(B, N):
    """The largest compiled grids (768 = 3 * 256 with the radix-3 stage, and 1024), FP32, quintic: a
    low-wavenumber field, whose interpolation error is far below FP32 rounding, against the direct
    trigonometric sum at sampled positions."""
    F = synth.kolmogorov_field(N, seed=31, kmax=4)
    plan = B.Plan(N, 6, "f32")
    uh = torch.zeros((3, N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
    idx = torch.from_numpy(F.idx).cuda()
    uh[:, idx[:, 0], idx[:, 1], idx[:, 2]] = torch.from_numpy(F.val).to(torch.complex64).cuda()
    coef = plan.coeffs(uh)
    x = synth.uniform_particles(4096, seed=32)
    u, g = plan.interp(coef, torch.from_numpy(x).cuda())
    assert plan.status() == 0
    ru, rg = O.direct_sum_modes(N, F.idx, F.val.astype(np.complex64).astype(np.complex128), x)
    assert normwise(u.cpu().numpy(), ru) < 2e-5
    assert normwise(g.cpu().numpy(), rg) < 5e-5
    del uh, coef, u, g
    plan.close()
    torch.cuda.empty_cache()
