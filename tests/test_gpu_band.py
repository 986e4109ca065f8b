"""Band-limited input (bspline_plan_set_band): a plan told that every mode beyond |kx|, |ky|, kz <= K is
zero skips those modes in the transform and in the host-to-device copies.  Its coefficients and particle
outputs must be the full path's bits for a field that is zero there, whatever the input holds outside the
band, through bspline_coeffs, bspline_eval and bspline_run_host."""
import math

import numpy as np
import pytest

from oracle import bspline_oracle as O
from paper_1201_4060_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1201_4060_gb300 import _build
    _build.build()
    from paper_1201_4060_gb300 import bspline
    assert torch.cuda.is_available()
    return bspline


def outside_band(N, K):
    """Boolean mask [N][N][N/2+1] of the modes outside the box |kx|, |ky|, kz <= K."""
    idx = np.arange(N)
    signed = np.where(idx <= N // 2, idx, idx - N)
    kx = np.abs(signed)[:, None, None]
    ky = np.abs(signed)[None, :, None]
    kz = np.arange(N // 2 + 1)[None, None, :]
    return (kx > K) | (ky > K) | (kz > K)


def band_field(N, K, seed):
    """A field inside the band (Kolmogorov spectrum on |k| <= K), and the same field with large values
    written everywhere outside the band."""
    half = synth.kolmogorov_field(N, seed=seed, kmax=K).dense()
    assert not np.any(half[:, outside_band(N, K)])
    rng = np.random.default_rng(seed)
    dirty = half.copy()
    m = outside_band(N, K)
    dirty[:, m] = 1e3 * (rng.standard_normal((3, int(m.sum()))) + 1j * rng.standard_normal((3, int(m.sum()))))
    return half, dirty


CASES = [(16, 5, "f32"), (48, 16, "f32"), (64, 21, "bf16"), (96, 32, "f64"), (128, 42, "f32"), (256, 85, "f32"),
         (32, 1, "f32"), (64, 31, "f32"), (8, 3, "f64")]


@pytest.mark.parametrize("N,K,dtype", CASES)
def test_band_coefficients_equal_the_full_transform(B, N, K, dtype):
    half, dirty = band_field(N, K, seed=N + K)
    full = B.Plan(N, 5, dtype)
    band = B.Plan(N, 5, dtype)
    band.set_band(K)
    c_full = full.coeffs(torch.from_numpy(half).to(full.uhat_dtype).cuda())
    c_band = band.coeffs(torch.from_numpy(dirty).to(band.uhat_dtype).cuda())
    torch.cuda.synchronize()
    assert band.status() == 0
    assert torch.equal(c_full, c_band)
    if dtype == "f64":
        assert np.abs(c_band.cpu().numpy() - O.coefficients(half, 5)).max() < 1e-12 * np.abs(c_band.cpu().numpy()).max()


@pytest.mark.parametrize("N,K,dtype", [(64, 21, "f32"), (96, 32, "bf16"), (48, 16, "f64")])
def test_band_eval_and_host_path_equal_the_full_path(B, N, K, dtype):
    half, dirty = band_field(N, K, seed=7 * N)
    P = 20000
    x = synth.clustered_particles(P, seed=N)
    full = B.Plan(N, 6, dtype)
    band = B.Plan(N, 6, dtype)
    band.set_band(K)
    xt = torch.from_numpy(x).cuda()
    cf, uf, gf = full.eval(torch.from_numpy(half).to(full.uhat_dtype).cuda(), xt)
    cb, ub, gb = band.eval(torch.from_numpy(dirty).to(band.uhat_dtype).cuda(), xt)
    torch.cuda.synchronize()
    assert torch.equal(cf, cb) and torch.equal(uf, ub) and torch.equal(gf, gb)
    # host buffers: only the band box is copied; the dirty modes outside it are never read
    uh = torch.from_numpy(dirty).to(band.uhat_dtype).pin_memory()
    xh = torch.from_numpy(x).pin_memory()
    uo = torch.empty((P, 3), dtype=band.out_dtype).pin_memory()
    go = torch.empty((P, 3, 3), dtype=band.out_dtype).pin_memory()
    for _ in range(2):                                     # the device u_hat keeps stale modes the second time
        uo.fill_(float("nan"))
        band.run_host(uh, xh, uo, go)
        assert torch.equal(uo, uf.cpu()) and torch.equal(go, gf.cpu())
    assert band.status() == 0


@pytest.mark.parametrize("N,K,dtype", [(48, 16, "f64"), (64, 21, "f32"), (32, 1, "f32")])
def test_band_adjoint_is_the_full_adjoint_inside_and_zero_outside(B, N, K, dtype):
    """The banded forward path ignores the modes outside the band, so the gradient there is zero; inside,
    the transposed transform gives the full one's bits."""
    rng = np.random.default_rng(N + K)
    full = B.Plan(N, 4, dtype)
    band = B.Plan(N, 4, dtype)
    band.set_band(K)
    g = torch.from_numpy(rng.standard_normal((3, N, N, N))).to(full.out_dtype).cuda()
    x = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    gf, _, _ = full.spread_adjoint(x, g_coef=g.clone())
    gb, _, _ = band.spread_adjoint(x, g_coef=g.clone())
    torch.cuda.synchronize()
    out = torch.from_numpy(outside_band(N, K)).cuda()
    expect = torch.where(out[None], torch.zeros_like(gf), gf)
    assert torch.equal(gb, expect)


def test_band_off_and_argument_checks(B):
    plan = B.Plan(32, 4, "f32")
    for bad in (-1, 16, 40):
        with pytest.raises(B.BSplineError) as exc:
            plan.set_band(bad)
        assert exc.value.code == B.ERR_INVALID_ARG
    half, dirty = band_field(32, 10, seed=3)
    plan.set_band(10)
    plan.set_band(0)                                        # off again: the full transform, which reads every mode
    c = plan.coeffs(torch.from_numpy(dirty).to(plan.uhat_dtype).cuda())
    ref = B.Plan(32, 4, "f32").coeffs(torch.from_numpy(dirty).to(plan.uhat_dtype).cuda())
    torch.cuda.synchronize()
    assert torch.equal(c, ref)
