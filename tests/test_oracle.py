"""Pins of the CPU FP64 oracle against what the paper and mathematics fix.

Each test pins a part of the oracle to something other than itself: values
the paper prints, textbook closed forms, brute force on tiny inputs,
identities (partition of unity, node reproduction, separability, linearity,
periodicity), convergence orders, continuity, and the closed-form L2 error of
Section 5.  A dropped term, wrong sign, wrong index or transposed operand in
the oracle fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import bspline_oracle as O
from paper_1201_4060_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
L = 2.0 * math.pi


def _read_paper_matrices():
    mats = {}
    cur = None
    with open(os.path.join(GOLDEN, "paper_bspline_matrices.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("order"):
                _, n, _, s = line.split()
                cur = (int(n), int(s))
                mats[cur[0]] = []
            else:
                mats[cur[0]].append([Fraction(int(v), cur[1]) for v in line.split()])
    return mats


# --------------------------------------------------------------------------- weights

def test_matrices_equal_printed_m1_to_m4():
    """Section 7 prints M_(1)..M_(4); Eq. B_spline_matrix must reproduce them exactly (0^0 = 1)."""
    printed = _read_paper_matrices()
    assert sorted(printed) == [1, 2, 3, 4]
    for n, M in printed.items():
        assert O.bspline_matrix_exact(n) == M, f"order {n}"


def _truncated_power_bspline(y, n):
    """Centred B-spline of order n from the textbook truncated-power form of the n-fold box convolution:
    B_n(y) = 1/(n-1)! sum_k (-1)^k C(n, k) (y + n/2 - k)_+^(n-1)."""
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros_like(y)
    for k in range(n + 1):
        z = y + n / 2.0 - k
        out += (-1) ** k * math.comb(n, k) * np.where(z > 0, z, 0.0) ** (n - 1)
    return out / math.factorial(n - 1)


@pytest.mark.parametrize("n", range(2, 9))
def test_kernel_from_matrix_matches_box_convolution_closed_form(n):
    y = np.random.default_rng(n).uniform(-n / 2 - 0.5, n / 2 + 0.5, 4000)
    np.testing.assert_allclose(O.bspline_kernel(y, n), _truncated_power_bspline(y, n), atol=1e-11)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_kernel_matches_numerical_box_convolution(n):
    """Brute force: convolve the unit box with itself n-1 times on a fine grid (Section 7 definition)."""
    h = 1e-3
    x = np.arange(-0.5, 0.5, h) + h / 2
    box = np.ones_like(x)
    f = box.copy()
    for _ in range(n - 1):
        f = np.convolve(f, box) * h
    xs = (np.arange(f.size) - (f.size - 1) / 2.0) * h
    sel = slice(None, None, 37)
    np.testing.assert_allclose(O.bspline_kernel(xs[sel], n), f[sel], atol=5e-3)


@pytest.mark.parametrize("n", range(1, 9))
def test_partition_of_unity(n):
    t = np.random.default_rng(10 + n).uniform(0, 1, 1000)
    W, W1 = O.weights(t, n)
    np.testing.assert_allclose(W.sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(W1.sum(axis=1), 0.0, atol=1e-12)
    assert np.all(W >= -1e-15)


@pytest.mark.parametrize("n", range(2, 9))
def test_derivative_weights_match_finite_differences(n):
    t = np.random.default_rng(20 + n).uniform(0.01, 0.99, 200)
    e = 1e-6
    Wp, _ = O.weights(t + e, n)
    Wm, _ = O.weights(t - e, n)
    _, W1 = O.weights(t, n)
    np.testing.assert_allclose(W1, (Wp - Wm) / (2 * e), atol=1e-8)


def _eulerian(m):
    """Eulerian numbers A(m, k), k = 0..m-1, by the textbook recurrence."""
    A = [1]
    for mm in range(2, m + 1):
        A = [(k + 1) * (A[k] if k < len(A) else 0) + (mm - k) * (A[k - 1] if k >= 1 else 0)
             for k in range(mm)]
    return A


@pytest.mark.parametrize("n", [2, 4, 6, 8])
def test_node_values_are_eulerian_numbers(n):
    """B_(n)(d) at integers d are A(n-1, k) / (n-1)! (even n)."""
    d, b = O.node_values(n)
    A = _eulerian(n - 1)
    expect = np.zeros_like(b)
    for k, a in enumerate(A):
        dd = k - (n - 2) / 2.0
        expect[np.isclose(d, dd)] = a / math.factorial(n - 1)
    np.testing.assert_allclose(b, expect, atol=1e-15)


def test_node_values_textbook_cubic_quintic():
    d, b = O.node_values(4)
    assert np.allclose(b[np.isin(d, [-1, 0, 1])], [1 / 6, 2 / 3, 1 / 6])
    d, b = O.node_values(6)
    assert np.allclose(b[np.isin(d, [-2, -1, 0, 1, 2])], [1 / 120, 13 / 60, 11 / 20, 13 / 60, 1 / 120])


def test_weights_equal_kernel_at_node_offsets():
    """Weight of node j = B(t + n/2 - j) (Eqs. alg-int-1 and alg-int-3)."""
    for n in range(2, 9):
        t = np.random.default_rng(30 + n).uniform(0, 1, 100)
        W, _ = O.weights(t, n)
        for j in range(1, n + 1):
            np.testing.assert_allclose(W[:, j - 1], _truncated_power_bspline(t + n / 2 - j, n), atol=1e-11)


# --------------------------------------------------------------------------- prefilter

def test_prefilter_at_nyquist_closed_forms():
    """F_D[B_D] at k = m/2 is 1, 1/3, 2/15, 17/315 for orders 2, 4, 6, 8 (alternating sum of node values)."""
    for n, v in [(2, 1.0), (4, 1 / 3), (6, 2 / 15), (8, 17 / 315)]:
        c = O.prefilter(16, n)
        assert abs(1.0 / c[8] - v) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_prefilter_poisson_summation(n):
    """F_D[B_D](k) = sum_i F[B](k/m + i) with F[B](kappa) = sinc(kappa)^n (B = n boxes convolved)."""
    m = 32
    k = np.arange(m)
    kappa = np.where(k < m / 2, k, k - m) / m
    i = np.arange(-20000, 20001)
    pois = (np.sinc(kappa[:, None] + i[None, :]) ** n).sum(axis=1)
    tol = 2e-4 if n == 2 else 1e-9
    np.testing.assert_allclose(1.0 / O.prefilter(m, n), pois, rtol=tol, atol=tol)


def test_l2_prefilter_denominator_poisson():
    for n in (3, 4, 6):
        kappa = np.linspace(-0.5, 0.5, 33)
        i = np.arange(-3000, 3001)
        direct = (np.sinc(kappa[:, None] + i) ** (2 * n)).sum(axis=1)
        np.testing.assert_allclose(O.transfer_discrete(kappa, 2 * n), direct, rtol=1e-12)


# --------------------------------------------------------------------------- transform

def _brute_inverse(half):
    """O(N^6) inverse of a half spectrum with real-to-complex weights (sum of m(kz) Re(X e^{i...}))."""
    N = half.shape[1]
    n = np.arange(N)
    out = np.zeros((3, N, N, N))
    for ix in range(N):
        for iy in range(N):
            for iz in range(N // 2 + 1):
                m = 1.0 if iz in (0, N // 2) else 2.0
                ph = np.exp(2j * np.pi * (ix * n[:, None, None] + iy * n[None, :, None] + iz * n[None, None, :]) / N)
                out += m * (half[:, ix, iy, iz][:, None, None, None] * ph[None]).real
    return out


@pytest.mark.parametrize("hermitian", [True, False])
def test_inverse_transform_brute_force(hermitian):
    half = synth.random_half_spectrum(6, seed=7, hermitian=hermitian)
    got = O.inverse_real_transform(half)
    np.testing.assert_allclose(got, _brute_inverse(half), atol=1e-11)


def test_direct_sum_equals_inverse_transform_at_nodes():
    half = synth.random_half_spectrum(8, seed=8, hermitian=False)
    f = O.grid_values(half)
    rng = np.random.default_rng(1)
    ijk = rng.integers(0, 8, size=(50, 3))
    u, _ = O.direct_sum(half, ijk * (L / 8))
    np.testing.assert_allclose(u, f[:, ijk[:, 0], ijk[:, 1], ijk[:, 2]].T, atol=1e-10)


@pytest.mark.parametrize("N,n", [(8, 2), (8, 3), (8, 4), (12, 4), (12, 5), (12, 6), (16, 8), (10, 7)])
def test_collocation_solve_matches_prefilter_and_fft(N, n):
    """Coefficients by the periodic banded collocation solve (u = u_B *_D B_D) equal prefilter + one FFT."""
    half = synth.random_half_spectrum(N, seed=N * 10 + n)
    via_fft = O.coefficients(half, n)
    via_solve = O.collocation_coefficients(O.grid_values(half), n)
    np.testing.assert_allclose(via_fft, via_solve, atol=1e-12 * np.abs(via_solve).max())


# --------------------------------------------------------------------------- evaluation

@pytest.mark.parametrize("n", range(2, 9))
def test_node_reproduction(n):
    """With the interpolating prefilter the interpolant passes through the grid values."""
    N = 16
    half = synth.kolmogorov_field(N, seed=100 + n).dense()
    f = O.grid_values(half)
    rng = np.random.default_rng(n)
    ijk = rng.integers(0, N, size=(200, 3))
    u, _ = O.interpolate(half, ijk * (L / N), n)
    np.testing.assert_allclose(u, f[:, ijk[:, 0], ijk[:, 1], ijk[:, 2]].T, atol=1e-12)


def _interp_1d(vals, s, n):
    """1D interpolant through periodic samples: collocation solve then weights (independent of the 3D path)."""
    m = vals.size
    coef = np.linalg.solve(O.collocation_matrix(m, n), vals)
    sh = s - n / 2.0
    base = np.floor(sh)
    t = sh - base
    W, W1 = O.weights(t, n)
    nodes = np.mod(base.astype(np.int64)[:, None] + np.arange(1, n + 1), m)
    return (W * coef[nodes]).sum(axis=1), (W1 * coef[nodes]).sum(axis=1)


@pytest.mark.parametrize("n", [2, 4, 5, 6])
def test_separability_product_mode(n):
    """Interpolant of f(x) g(y) = product of the 1D interpolants (Eq. condition)."""
    N, a, b = 16, 3, 5
    half = np.zeros((3, N, N, N // 2 + 1), complex)
    for sx, sy in [(a, b), (-a, -b), (a, -b), (-a, b)]:
        half[1, sx % N, sy % N, 0] = 0.25         # cos(a x) cos(b y) in component 1
    rng = np.random.default_rng(2)
    x = rng.uniform(0, L, (300, 3))
    u, g = O.interpolate(half, x, n)
    grid = np.arange(N) * (L / N)
    fx, dfx = _interp_1d(np.cos(a * grid), x[:, 0] * N / L, n)
    fy, dfy = _interp_1d(np.cos(b * grid), x[:, 1] * N / L, n)
    np.testing.assert_allclose(u[:, 1], fx * fy, atol=1e-12)
    np.testing.assert_allclose(g[:, 1, 0], dfx * (N / L) * fy, atol=1e-11)
    np.testing.assert_allclose(g[:, 1, 1], fx * dfy * (N / L), atol=1e-11)
    np.testing.assert_allclose(g[:, 1, 2], 0.0, atol=1e-12)
    np.testing.assert_allclose(u[:, [0, 2]], 0.0, atol=1e-15)


def test_linearity():
    N, n = 8, 4
    a = synth.random_half_spectrum(N, 1)
    b = synth.random_half_spectrum(N, 2)
    x = np.random.default_rng(3).uniform(0, L, (100, 3))
    ua, ga = O.interpolate(a, x, n)
    ub, gb = O.interpolate(b, x, n)
    uc, gc = O.interpolate(2.5 * a - 1.5j * 0 + (-0.75) * b, x, n)
    np.testing.assert_allclose(uc, 2.5 * ua - 0.75 * ub, atol=1e-11)
    np.testing.assert_allclose(gc, 2.5 * ga - 0.75 * gb, atol=1e-10)


@pytest.mark.parametrize("n", [2, 3, 4, 6, 8])
def test_gradient_matches_finite_differences(n):
    N = 16
    half = synth.kolmogorov_field(N, seed=5).dense()
    coef = O.coefficients(half, n)
    rng = np.random.default_rng(4)
    x = rng.uniform(0, L, (60, 3))
    # stay away from cell faces, where the order-2 derivative jumps
    s = x * N / L - n / 2
    x = np.where(np.abs(s - np.round(s)) < 0.05, x + 0.2 * L / N, x)
    _, g = O.evaluate(coef, x, n)
    h = 1e-5
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        up, _ = O.evaluate(coef, x + e, n)
        um, _ = O.evaluate(coef, x - e, n)
        np.testing.assert_allclose(g[:, :, j], (up - um) / (2 * h), atol=2e-6 * np.abs(g).max())


def test_periodicity_and_locate_edge_cases():
    N, n = 8, 4
    half = synth.kolmogorov_field(N, seed=9).dense()
    coef = O.coefficients(half, n)
    x = np.random.default_rng(5).uniform(0, L, (50, 3))
    u0, g0 = O.evaluate(coef, x, n)
    for shift in (L, -L, 3 * L):
        u1, g1 = O.evaluate(coef, x + shift, n)
        np.testing.assert_allclose(u1, u0, atol=1e-12)
        np.testing.assert_allclose(g1, g0, atol=1e-10)
    nodes, t = O.locate(np.array([[0.0, L / N, L - 1e-12]]), N, n)
    assert np.all((t >= 0) & (t < 1))
    assert nodes[0, 0].tolist() == [7, 0, 1, 2]          # floor(0 - 2) + j, wrapped
    assert t[0, 0] == 0.0 and t[0, 1] == 0.0


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_continuity_across_cell_faces(n):
    """u is C^(n-2): for n >= 3 the gradient is continuous across faces; for n = 2 only u is."""
    N = 16
    half = synth.kolmogorov_field(N, seed=11).dense()
    coef = O.coefficients(half, n)
    rng = np.random.default_rng(6)
    base = rng.uniform(0, L, (40, 3))
    face = (np.floor(base[:, 0] * N / L - n / 2) + 1 + n / 2) * (L / N)   # a plane where t jumps 1 -> 0
    eps = 1e-9
    xl = base.copy(); xl[:, 0] = face - eps
    xr = base.copy(); xr[:, 0] = face + eps
    ul, gl = O.evaluate(coef, xl, n)
    ur, gr = O.evaluate(coef, xr, n)
    np.testing.assert_allclose(ul, ur, atol=1e-6)
    jump = np.abs(gl[:, :, 0] - gr[:, :, 0]).max()
    if n >= 3:
        assert jump < 1e-5
    else:
        assert jump > 1e-3


# --------------------------------------------------------------------------- accuracy vs the exact field

@pytest.mark.parametrize("n", [2, 3, 4, 6, 8])
def test_convergence_order_single_mode(n):
    """Error of a single mode ~ h^n for the value and h^(n-1) for the derivative (Section 8, Table 2: n = N-1+1)."""
    k = 1
    errs_u, errs_g = [], []
    Ns = [16, 32, 64] if n >= 6 else [16, 32, 64, 128]
    for N in Ns:
        half = np.zeros((3, N, N, N // 2 + 1), complex)
        half[0, k, 0, 0] = 0.5
        half[0, N - k, 0, 0] = 0.5                       # u_0 = cos(k x)
        rng = np.random.default_rng(7)
        x = rng.uniform(0, L, (3000, 3))
        u, g = O.interpolate(half, x, n)
        errs_u.append(np.sqrt(np.mean((u[:, 0] - np.cos(k * x[:, 0])) ** 2)))
        errs_g.append(np.sqrt(np.mean((g[:, 0, 0] + k * np.sin(k * x[:, 0])) ** 2)))
    su = np.polyfit(np.log(Ns), np.log(errs_u), 1)[0]
    sg = np.polyfit(np.log(Ns), np.log(errs_g), 1)[0]
    assert abs(-su - n) < 0.3, (su, errs_u)
    assert abs(-sg - (n - 1)) < 0.3, (sg, errs_g)


@pytest.mark.parametrize("n", [2, 3, 4, 6, 8])
@pytest.mark.parametrize("k", [3, 7, 10])
def test_single_mode_error_matches_closed_form(n, k):
    """RMS error of a mode over a period equals Eq. l2-error (value) and Eq. l2-error-der (l = 1)."""
    N = 32
    half = np.zeros((3, N, N, N // 2 + 1), complex)
    half[2, k, 0, 0] = 0.5
    half[2, N - k, 0, 0] = 0.5                           # u_2 = cos(k x)
    coef = O.coefficients(half, n)
    M = 8192
    x = np.zeros((M, 3))
    x[:, 0] = (np.arange(M) + 0.3141) * (L / M)
    x[:, 1:] = 1.234
    u, g = O.evaluate(coef, x, n)
    rel_u = np.mean((u[:, 2] - np.cos(k * x[:, 0])) ** 2) / 0.5
    rel_g = np.mean((g[:, 2, 0] + k * np.sin(k * x[:, 0])) ** 2) / (0.5 * k * k)
    kappa = np.array([k / N])
    np.testing.assert_allclose(rel_u, O.l2_error_mode(kappa, n, 0)[0], rtol=2e-3)
    np.testing.assert_allclose(rel_g, O.l2_error_mode(kappa, n, 1)[0], rtol=2e-3)


@pytest.mark.parametrize("n", [3, 4, 6])
def test_l2_prefilter_minimises_single_mode_error(n):
    """Eq. B_spline_coeff is defined by d/dc ||phi - c phi~||^2 = 0: scaling the L2-optimal c of the mode
    by 1 +- 2 % must increase the interpolation error measured through the full oracle path, and the
    L2 choice must beat the interpolating one."""
    N, k = 16, 5
    M = 4096
    x = np.zeros((M, 3))
    x[:, 0] = (np.arange(M) + 0.37) * (L / M)
    exact = np.cos(k * x[:, 0])

    def err(kind, scale):
        half = np.zeros((3, N, N, N // 2 + 1), complex)
        half[0, k, 0, 0] = 0.5
        half[0, N - k, 0, 0] = 0.5
        coef = O.coefficients(half, n, kind=kind) * scale
        u, _ = O.evaluate(coef, x, n)
        return np.mean((u[:, 0] - exact) ** 2)

    e0 = err("l2", 1.0)
    assert e0 < err("l2", 0.98) and e0 < err("l2", 1.02)
    assert e0 < err("interp", 1.0)


def test_l2_closed_form_matches_truncated_alias_sum():
    kappa = np.array([0.1, 0.2, 1 / 3])
    for n in (3, 4, 6):
        for l in (0, 1):
            np.testing.assert_allclose(O.l2_error_mode(kappa, n, l), O.l2_error_mode(kappa, n, l, n_alias=4000),
                                       rtol=1e-6)


@pytest.mark.parametrize("n", [4, 6])
def test_direct_sum_agreement_within_predicted_error(n):
    """Oracle vs the direct trigonometric sum on a Kolmogorov field: the sample mean-square error
    matches the orthogonality-based prediction (Section 5 Theorem and Corollary, 3D by products)."""
    N = 32
    F = synth.kolmogorov_field(N, seed=1202)
    half = F.dense()
    x = synth.uniform_particles(4096, seed=4061)
    u, g = O.interpolate(half, x, n)
    ue, ge = O.direct_sum_modes(N, F.idx, F.val, x)
    mse_u, mse_g = O.l2_error_field(N, F.idx, F.val, n)
    got_u = np.mean((u - ue) ** 2, axis=0)
    got_g = np.mean((g - ge) ** 2, axis=0)
    np.testing.assert_allclose(got_u / mse_u, 1.0, atol=0.2)
    np.testing.assert_allclose(got_g / mse_g, 1.0, atol=0.2)


def test_direct_sum_gradient_fd():
    N = 8
    half = synth.random_half_spectrum(N, 3)
    x = np.random.default_rng(9).uniform(0, L, (20, 3))
    _, g = O.direct_sum(half, x)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3); e[j] = h
        up, _ = O.direct_sum(half, x + e)
        um, _ = O.direct_sum(half, x - e)
        np.testing.assert_allclose(g[:, :, j], (up - um) / (2 * h), atol=1e-6 * np.abs(g).max())


def test_table1_cost_formula():
    rows = {}
    with open(os.path.join(GOLDEN, "paper_table1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            label, _, v = line.strip().split(",")
            rows[label] = int(v)
    assert O.table1_fma_count(4) == rows["total"] == 672
    assert sum(v for k, v in rows.items() if k != "total") == 672
