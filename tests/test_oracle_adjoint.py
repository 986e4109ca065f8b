"""Pins of the oracle's adjoint (differentiation) functions.

The adjoint is the transpose of the forward path, so every pin here ties it
to the already-pinned forward oracle or to closed forms: textbook second
derivatives of the cubic B-spline, finite differences, the inner-product
identity <g, F a> = <F^T g, a> with random vectors, brute-force sums on tiny
grids, and the exact linearity of the path in u_hat.  A dropped term, a wrong
sign or conjugation, a missing multiplicity or scale factor in the adjoint
fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import bspline_oracle as O
from paper_1201_4060_gb300 import synth

L = 2.0 * math.pi


def _random_half(N, rng):
    """Arbitrary complex half spectrum: non-Hermitian kz = 0 plane and Nyquist entries included."""
    nh = N // 2 + 1
    return rng.standard_normal((3, N, N, nh)) + 1j * rng.standard_normal((3, N, N, nh))


def _away_from_faces(x, N, n, margin=0.03):
    s = x * N / L - n / 2
    return np.where(np.abs(s - np.round(s)) < margin, x + 0.1 * L / N, x)


def test_second_derivative_weights_cubic_closed_form():
    # cubic B-spline pieces (1-t)^3/6, (3t^3-6t^2+4)/6, (-3t^3+3t^2+3t+1)/6, t^3/6
    t = np.linspace(0.0, 1.0, 23)
    W2 = O.weights2(t, 4)
    ref = np.stack([1 - t, 3 * t - 2, 1 - 3 * t, t], axis=1)
    np.testing.assert_allclose(W2, ref, atol=1e-14)


def test_second_derivative_weights_quadratic_closed_form():
    t = np.linspace(0.0, 1.0, 11)
    np.testing.assert_allclose(O.weights2(t, 3), np.tile([1.0, -2.0, 1.0], (11, 1)), atol=1e-14)
    np.testing.assert_allclose(O.weights2(t, 2), 0.0, atol=0)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_second_derivative_weights_fd_and_moments(n):
    t = np.linspace(0.05, 0.95, 19)
    h = 1e-5
    _, W1p = O.weights(t + h, n)
    _, W1m = O.weights(t - h, n)
    W2 = O.weights2(t, n)
    np.testing.assert_allclose(W2, (W1p - W1m) / (2 * h), atol=1e-8)
    j = np.arange(n, dtype=np.float64)
    # partition of unity and linear reproduction: sum_j W_j = 1, sum_j j W_j = t + const
    np.testing.assert_allclose(W2.sum(axis=1), 0.0, atol=1e-12)
    np.testing.assert_allclose(W2 @ j, 0.0, atol=1e-11)


@pytest.mark.parametrize("n", [4, 6])
def test_hessian_matches_fd_of_gradient_and_is_symmetric(n):
    N = 8
    coef = np.random.default_rng(1).standard_normal((3, N, N, N))
    x = _away_from_faces(np.random.default_rng(2).uniform(0, L, (40, 3)), N, n)
    H = O.hessian(coef, x, n)
    np.testing.assert_allclose(H, np.swapaxes(H, 2, 3), atol=1e-10 * np.abs(H).max())
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        _, gp = O.evaluate(coef, x + e, n)
        _, gm = O.evaluate(coef, x - e, n)
        np.testing.assert_allclose(H[:, :, :, d], (gp - gm) / (2 * h), atol=1e-6 * np.abs(H).max())


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_spread_is_adjoint_of_evaluate(n):
    N = 8
    rng = np.random.default_rng(10 + n)
    coef = rng.standard_normal((3, N, N, N))
    x = rng.uniform(0, L, (300, 3))
    g_u = rng.standard_normal((300, 3))
    g_grad = rng.standard_normal((300, 3, 3))
    u, g = O.evaluate(coef, x, n)
    lhs = (g_u * u).sum() + (g_grad * g).sum()
    rhs = (O.spread(x, g_u, g_grad, N, n) * coef).sum()
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(g_u * u).sum() + np.abs(g_grad * g).sum())
    # g_grad = None is the same as zero
    lhs0 = (g_u * u).sum()
    rhs0 = (O.spread(x, g_u, None, N, n) * coef).sum()
    assert abs(lhs0 - rhs0) <= 1e-12 * np.abs(g_u * u).sum()


def _kernel_derivative(y, n, h=1e-6):
    return (O.bspline_kernel(y + h, n) - O.bspline_kernel(y - h, n)) / (2 * h)


@pytest.mark.parametrize("n", [3, 4, 6])
def test_spread_brute_force_one_particle(n):
    # g_coef[q] = sum over periodic images q' of q of
    #   g_u B(s - q') + (N/L) sum_e g_grad_e B'(s_e - q'_e) prod_{d != e} B(s_d - q'_d)
    N = 6
    rng = np.random.default_rng(20 + n)
    x = rng.uniform(0, L, (1, 3))
    x = _away_from_faces(x, N, n, margin=0.01)
    g_u = rng.standard_normal((1, 3))
    g_grad = rng.standard_normal((1, 3, 3))
    s = x[0] * N / L
    ref = np.zeros((3, N, N, N))
    scale = N / L
    span = range(-2 * N, 3 * N)
    for qx in span:
        bx = O.bspline_kernel(np.array(s[0] - qx), n)
        dbx = _kernel_derivative(np.array(s[0] - qx), n)
        if bx == 0 and dbx == 0:
            continue
        for qy in span:
            by = O.bspline_kernel(np.array(s[1] - qy), n)
            dby = _kernel_derivative(np.array(s[1] - qy), n)
            if by == 0 and dby == 0:
                continue
            for qz in span:
                bz = O.bspline_kernel(np.array(s[2] - qz), n)
                dbz = _kernel_derivative(np.array(s[2] - qz), n)
                if bz == 0 and dbz == 0:
                    continue
                for c in range(3):
                    v = g_u[0, c] * bx * by * bz + scale * (g_grad[0, c, 0] * dbx * by * bz
                                                            + g_grad[0, c, 1] * bx * dby * bz
                                                            + g_grad[0, c, 2] * bx * by * dbz)
                    ref[c, qx % N, qy % N, qz % N] += v
    got = O.spread(x, g_u, g_grad, N, n)
    np.testing.assert_allclose(got, ref, atol=1e-7 * np.abs(ref).max())


def test_spread_skips_nonfinite_positions():
    N, n = 8, 4
    rng = np.random.default_rng(3)
    x = rng.uniform(0, L, (5, 3))
    g_u = rng.standard_normal((5, 3))
    bad = x.copy()
    bad[1, 0] = np.nan
    bad[3, 2] = np.inf
    keep = [0, 2, 4]
    np.testing.assert_array_equal(O.spread(bad, g_u, None, N, n), O.spread(x[keep], g_u[keep], None, N, n))
    gx = O.position_gradient(rng.standard_normal((3, N, N, N)), bad, g_u, None, n)
    assert np.isnan(gx[[1, 3]]).all() and np.isfinite(gx[keep]).all()


@pytest.mark.parametrize("kind", ["interp", "l2"])
@pytest.mark.parametrize("N,n", [(8, 4), (8, 6), (6, 3), (10, 8)])
def test_adjoint_transform_inner_product(N, n, kind):
    rng = np.random.default_rng(N * 10 + n)
    a = _random_half(N, rng)
    g = rng.standard_normal((3, N, N, N))
    lhs = (g * O.coefficients(a, n, kind)).sum()
    ga = O.adjoint_transform(g, n, kind)
    rhs = (np.conj(ga) * a).real.sum()
    assert abs(lhs - rhs) <= 1e-12 * np.abs(g).sum() * np.abs(ga).max()


def test_adjoint_transform_brute_force():
    N, n = 4, 4
    rng = np.random.default_rng(7)
    g = rng.standard_normal((3, N, N, N))
    c = O.prefilter(N, n)
    ref = np.zeros((3, N, N, N // 2 + 1), dtype=np.complex128)
    grid = np.arange(N)
    X, Y, Z = np.meshgrid(grid, grid, grid, indexing="ij")
    for kx in range(N):
        for ky in range(N):
            for kz in range(N // 2 + 1):
                m = 1.0 if kz in (0, N // 2) else 2.0
                ph = np.exp(-2j * np.pi * (kx * X + ky * Y + kz * Z) / N)
                for comp in range(3):
                    ref[comp, kx, ky, kz] = c[kx] * c[ky] * c[kz] * m * (g[comp] * ph).sum()
    np.testing.assert_allclose(O.adjoint_transform(g, n), ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n", [4, 6])
def test_position_gradient_matches_fd(n):
    N = 8
    half = synth.kolmogorov_field(N, seed=3).dense()
    coef = O.coefficients(half, n)
    rng = np.random.default_rng(11)
    x = _away_from_faces(rng.uniform(0, L, (30, 3)), N, n)
    g_u = rng.standard_normal((30, 3))
    g_grad = rng.standard_normal((30, 3, 3))
    gx = O.position_gradient(coef, x, g_u, g_grad, n)

    def loss(xx):
        u, g = O.evaluate(coef, xx, n)
        return (g_u * u).sum(axis=1) + (g_grad * g).sum(axis=(1, 2))

    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (loss(x + e) - loss(x - e)) / (2 * h)
        np.testing.assert_allclose(gx[:, d], fd, atol=1e-6 * np.abs(gx).max())


@pytest.mark.parametrize("kind", ["interp", "l2"])
def test_full_chain_is_exact_linear_response(kind):
    # the path is linear in u_hat: L(a + d) - L(a) = Re <g_u_hat, d> exactly
    N, n = 8, 4
    rng = np.random.default_rng(12)
    a = _random_half(N, rng)
    d = _random_half(N, rng)
    x = rng.uniform(0, L, (64, 3))
    g_u = rng.standard_normal((64, 3))
    g_grad = rng.standard_normal((64, 3, 3))

    def loss(h):
        u, g = O.interpolate(h, x, n, kind=kind)
        return (g_u * u).sum() + (g_grad * g).sum()

    g_hat, _, _ = O.interpolate_adjoint(a, x, g_u, g_grad, n, kind=kind)
    lhs = loss(a + d) - loss(a)
    rhs = (np.conj(g_hat) * d).real.sum()
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(rhs))


@pytest.mark.parametrize("kind", ["interp", "l2"])
def test_adjoint_transform_matches_torch_autograd(kind):
    # an independent transpose: PyTorch's reverse mode through irfftn, with the
    # prefilter multiply written in torch (gradient convention dL/dRe + i dL/dIm)
    torch = pytest.importorskip("torch")
    N, n = 8, 4
    rng = np.random.default_rng(13)
    a = _random_half(N, rng)
    g = rng.standard_normal((3, N, N, N))
    c = O.prefilter(N, n) if kind == "interp" else O.prefilter_l2(N, n)
    c3 = c[:, None, None] * c[None, :, None] * c[None, None, :N // 2 + 1]
    at = torch.tensor(a, requires_grad=True)
    coef = torch.fft.irfftn(at * torch.tensor(c3)[None], s=(N, N, N), dim=(1, 2, 3), norm="forward")
    np.testing.assert_allclose(coef.detach().numpy(), O.coefficients(a, n, kind), atol=1e-12)
    (coef * torch.tensor(g)).sum().backward()
    ref = at.grad.numpy()
    np.testing.assert_allclose(O.adjoint_transform(g, n, kind), ref, atol=1e-11 * np.abs(ref).max())
