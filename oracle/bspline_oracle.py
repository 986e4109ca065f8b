"""CPU FP64 oracle of B-spline interpolation for pseudo-spectral fields.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this module.  The CUDA library never
calls it, and it shares no code, table or constant generator with the CUDA
library.

The method (van Hinsberg, ten Thije Boonkkamp, Toschi, Clercx, "On the
efficiency and accuracy of interpolation methods for spectral codes"):

1. prefilter each Fourier mode by c(kx) c(ky) c(kz), c(k) = 1 / F_D[B_D](k)
   (Section 7, Eqs. B_spline_multiplication and B_spline_multiplication_3d);
2. one inverse FFT gives the B-spline coefficients u_B on the grid
   (Section 7, the coefficient transform u_B = u *_D B_D^-1);
3. evaluate the tensor-product B-spline of order n and its first derivatives
   at off-grid points with the monomial weight matrices M and M^(1) = M D
   (Sections 2-3, Eqs. interpolation1d2, interpolation, interpolation2;
   Section 7, Eq. B_spline_matrix), the stencil nodes given by Eq. alg-int-6.

Every step is written out plainly in float64.  Library primitives serve as
steps where the definition is a plain transform: numpy's inverse real FFT for
step 2 and numpy.linalg.solve for the independent collocation check.

Conventions (the readings the tests rely on):

* domain [0, L)^3 with N grid points per axis, h = L / N; grid units s = x / h;
* u(x) = sum_k u_hat_k exp(i (2 pi / L) k . x); u_hat is stored as the half
  spectrum [3][N][N][N//2+1] (kz >= 0) with real-to-complex semantics:
  the imaginary part of a self-conjugate mode is ignored, exactly as an
  inverse real FFT ignores it;
* M is indexed [stencil node j][power i] (row j gives the weight polynomial of
  node j, column i the coefficient of t^(i-1)), which is the layout of the
  printed matrices M_(1)..M_(4) and of Eq. alg-int-1; the sentence that
  defines B_(N),j with the indices the other way round is read as a
  transposition slip;
* 0^0 = 1 in Eq. B_spline_matrix;
* the discrete convolution of Section 7 sums y = 0..m-1;
* derivatives are returned in physical units: d/dx = (N / L) d/ds;
  grad[p][i][j] = d u_i / d x_j.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


# ---------------------------------------------------------------------------
# Section 7, Eq. B_spline_matrix: the weight matrix M_(n)
# ---------------------------------------------------------------------------

def _binom(n: int, k: int) -> int:
    if k < 0 or k > n:
        return 0
    return math.comb(n, k)


def bspline_matrix_exact(n: int) -> list[list[Fraction]]:
    """M_(n) of Eq. B_spline_matrix as exact rationals, indexed [node j-1][power i-1].

    M_{j,i} = 1/(n-1)! * C(n-1, n-i) * sum_{s=j}^{n} (-1)^(s-j) C(n, s-j) (n-s)^(n-i),
    with the paper's letters renamed so that the first index is the stencil
    node and the second the power (the paper prints the formula with (i, j)
    in that order: first index = row of the printed matrices).
    """
    if n < 1:
        raise ValueError("order must be >= 1")
    fact = math.factorial(n - 1)
    M = []
    for j in range(1, n + 1):          # row: stencil node
        row = []
        for i in range(1, n + 1):      # column: power t^(i-1)
            acc = 0
            for s in range(j, n + 1):
                base = n - s
                e = n - i
                p = 1 if e == 0 else base ** e      # 0^0 = 1
                acc += (-1) ** (s - j) * _binom(n, s - j) * p
            row.append(Fraction(_binom(n - 1, n - i) * acc, fact))
        M.append(row)
    return M


def bspline_matrix(n: int) -> np.ndarray:
    """float64 M_(n), [node][power]."""
    return np.array([[float(v) for v in row] for row in bspline_matrix_exact(n)], dtype=np.float64)


def derivative_matrix(n: int) -> np.ndarray:
    """D of Section 2 (Eq. interpolation1d2): a^(1)T = a^T D, D[i][i-1] = i (0-based powers)."""
    D = np.zeros((n, n), dtype=np.float64)
    for i in range(1, n):
        D[i, i - 1] = float(i)
    return D


def weights(t: np.ndarray, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Weights of the n stencil nodes and of their first derivative, monomial form.

    W[p, j] = sum_i M[j, i] t_p^i and W'[p, j] = sum_i (M D)[j, i] t_p^i,
    i.e. the columns of M x_bar and M^(1) x_bar (Eq. interpolation1d2).
    """
    t = np.asarray(t, dtype=np.float64)
    M = bspline_matrix(n)
    M1 = M @ derivative_matrix(n)
    xbar = t[..., None] ** np.arange(n, dtype=np.float64)      # [.., n]: 1, t, t^2, ...
    return xbar @ M.T, xbar @ M1.T


def bspline_kernel(y: np.ndarray, n: int) -> np.ndarray:
    """B_(n)(y) assembled from its pieces (Section 7): piece j covers
    y in [n/2 - j, n/2 - j + 1) and equals sum_i M[j, i] (y - n/2 + j)^(i-1)."""
    y = np.asarray(y, dtype=np.float64)
    M = bspline_matrix(n)
    j = np.ceil(n / 2.0 - y).astype(np.int64)           # 1-based piece index
    out = np.zeros_like(y)
    ok = (j >= 1) & (j <= n)
    jj = np.clip(j, 1, n) - 1
    loc = y - n / 2.0 + np.clip(j, 1, n)
    powers = loc[..., None] ** np.arange(n, dtype=np.float64)
    vals = (powers * M[jj]).sum(axis=-1)
    out[ok] = vals[ok]
    return out


# ---------------------------------------------------------------------------
# Section 7: the discrete kernel B_D and the prefilter c(k)
# ---------------------------------------------------------------------------

def discrete_kernel(m: int, n: int) -> np.ndarray:
    """B_D(x), x = 0..m-1: B(x) for x < m/2, B(x - m) for x >= m/2."""
    x = np.arange(m, dtype=np.float64)
    arg = np.where(x < m / 2.0, x, x - m)
    return bspline_kernel(arg, n)


def prefilter(m: int, n: int) -> np.ndarray:
    """c(k) = 1 / F_D[B_D](k), k = 0..m-1 (Eq. B_spline_multiplication).

    F_D[f](k) = sum_x f(x) exp(-2 pi i x k / m) is evaluated as that literal
    sum.  B is even, so the transform is real; its imaginary part is checked
    to vanish.
    """
    bd = discrete_kernel(m, n)
    x = np.arange(m, dtype=np.float64)
    k = np.arange(m, dtype=np.float64)
    F = (bd[None, :] * np.exp(-2j * np.pi * np.outer(k, x) / m)).sum(axis=1)
    if np.max(np.abs(F.imag)) > 1e-12 * np.max(np.abs(F.real)):
        raise AssertionError("F_D[B_D] is not real")
    return 1.0 / F.real


def sinc(x: np.ndarray) -> np.ndarray:
    return np.sinc(x)       # sin(pi x) / (pi x)


def node_values(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Integer offsets d inside the support of B_(n) and the values B_(n)(d)."""
    h = n // 2 + 1
    d = np.arange(-h, h + 1, dtype=np.float64)
    return d, bspline_kernel(d, n)


def transfer_discrete(kappa: np.ndarray, n: int) -> np.ndarray:
    """sum_d B_(n)(d) cos(2 pi kappa d): F_D[B_D] at k = kappa m for any m (finite sum)."""
    d, b = node_values(n)
    kappa = np.asarray(kappa, dtype=np.float64)
    return (b * np.cos(2.0 * np.pi * kappa[..., None] * d)).sum(axis=-1)


def prefilter_l2(m: int, n: int) -> np.ndarray:
    """L2-optimal c(k) of Eq. B_spline_coeff, kappa = k/m signed.

    Numerator F[B](kappa) = sinc(kappa)^n (B_(n) is n box functions convolved,
    Section 7).  The denominator sum_i sinc(kappa + i)^(2n) equals, by Poisson
    summation, the finite cosine sum of the node values of B_(2n).
    """
    k = np.arange(m, dtype=np.float64)
    kappa = np.where(k < m / 2.0, k, k - m) / m
    return sinc(kappa) ** n / transfer_discrete(kappa, 2 * n)


# ---------------------------------------------------------------------------
# Steps 1-2: prefilter and inverse transform -> coefficients
# ---------------------------------------------------------------------------

def prefilter_3d(u_hat: np.ndarray, n: int, kind: str = "interp") -> np.ndarray:
    """u_hat_B(k) = c(kx) c(ky) c(kz) u_hat(k) on the half spectrum (Eq. B_spline_multiplication_3d)."""
    u_hat = np.asarray(u_hat)
    N = u_hat.shape[1]
    c = prefilter(N, n) if kind == "interp" else prefilter_l2(N, n)
    nh = u_hat.shape[3]
    return u_hat.astype(np.complex128) * (c[:, None, None] * c[None, :, None] * c[None, None, :nh])[None]


def inverse_real_transform(u_hat_half: np.ndarray) -> np.ndarray:
    """Unnormalised inverse DFT of a half spectrum: f(x) = sum_k F(k) exp(2 pi i k.x / N)."""
    N = u_hat_half.shape[1]
    return np.fft.irfftn(u_hat_half, s=(N, N, N), axes=(1, 2, 3), norm="forward")


def coefficients(u_hat: np.ndarray, n: int, kind: str = "interp") -> np.ndarray:
    """B-spline coefficients u_B [3][N][N][N] from the half spectrum (Section 7)."""
    return inverse_real_transform(prefilter_3d(u_hat, n, kind))


def grid_values(u_hat: np.ndarray) -> np.ndarray:
    """The field itself at the grid nodes (no prefilter)."""
    return inverse_real_transform(np.asarray(u_hat, dtype=np.complex128))


# ---------------------------------------------------------------------------
# Step 3: locate, weights, stencil contraction
# ---------------------------------------------------------------------------

def locate(x: np.ndarray, N: int, n: int, L: float = 2.0 * math.pi):
    """Stencil origin and local variable (Eq. alg-int-6).

    s = x * (N / L) in float64; the nodes are floor(s - n/2 + j), j = 1..n,
    i.e. base + j with base = floor(s - n/2); the local variable is
    t = (s - n/2) - base in [0, 1).  Returned node indices are wrapped into
    [0, N) (periodic grid).
    """
    x = np.asarray(x, dtype=np.float64)
    s = x * (float(N) / float(L))
    sh = s - n / 2.0
    base = np.floor(sh)
    t = sh - base
    nodes = np.mod(base[..., None].astype(np.int64) + np.arange(1, n + 1, dtype=np.int64), N)
    return nodes, t


def evaluate(coef: np.ndarray, x: np.ndarray, n: int, L: float = 2.0 * math.pi,
             chunk: int = 4096) -> tuple[np.ndarray, np.ndarray]:
    """u [P][3] and grad [P][3][3] at positions x [P][3] (Eqs. interpolation, interpolation2).

    u_c = B_c x_1 (M xbar) x_2 (M ybar) x_3 (M zbar), and each first
    derivative replaces one factor by M^(1) (.) and scales by N / L.
    """
    coef = np.asarray(coef, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    N = coef.shape[1]
    P = x.shape[0]
    u = np.empty((P, 3))
    g = np.empty((P, 3, 3))
    scale = float(N) / float(L)
    for p0 in range(0, P, chunk):
        xs = x[p0:p0 + chunk]
        nodes, t = locate(xs, N, n, L)                # [p, 3, n], [p, 3]
        W, W1 = weights(t, n)                          # [p, 3, n]
        ix = nodes[:, 0, :, None, None]
        iy = nodes[:, 1, None, :, None]
        iz = nodes[:, 2, None, None, :]
        for c in range(3):
            B = coef[c][ix, iy, iz]                    # [p, n, n, n] stencil tensor
            u[p0:p0 + chunk, c] = np.einsum("pabc,pa,pb,pc->p", B, W[:, 0], W[:, 1], W[:, 2])
            g[p0:p0 + chunk, c, 0] = scale * np.einsum("pabc,pa,pb,pc->p", B, W1[:, 0], W[:, 1], W[:, 2])
            g[p0:p0 + chunk, c, 1] = scale * np.einsum("pabc,pa,pb,pc->p", B, W[:, 0], W1[:, 1], W[:, 2])
            g[p0:p0 + chunk, c, 2] = scale * np.einsum("pabc,pa,pb,pc->p", B, W[:, 0], W[:, 1], W1[:, 2])
    return u, g


def interpolate(u_hat: np.ndarray, x: np.ndarray, n: int, L: float = 2.0 * math.pi, kind: str = "interp"):
    """The whole path: prefilter, inverse transform, evaluation."""
    return evaluate(coefficients(u_hat, n, kind), x, n, L)


# ---------------------------------------------------------------------------
# Independent checks
# ---------------------------------------------------------------------------

def collocation_matrix(m: int, n: int) -> np.ndarray:
    """A[x, y] = B_D((x - y) mod m): u = u_B *_D B_D written as u = A u_B (Section 7)."""
    bd = discrete_kernel(m, n)
    i = np.arange(m)
    return bd[np.mod(i[:, None] - i[None, :], m)]


def collocation_coefficients(u_grid: np.ndarray, n: int) -> np.ndarray:
    """Coefficients by solving the periodic collocation system along each axis.

    The 3D operator is the Kronecker product of the 1D circulant matrices
    (Eq. B_spline_multiplication_3d), so u_B = (A^-1 x A^-1 x A^-1) u.
    """
    u_grid = np.asarray(u_grid, dtype=np.float64)
    m = u_grid.shape[1]
    A = collocation_matrix(m, n)
    out = u_grid.copy()
    for axis in (1, 2, 3):
        moved = np.moveaxis(out, axis, 0)
        sol = np.linalg.solve(A, moved.reshape(m, -1)).reshape(moved.shape)
        out = np.moveaxis(sol, 0, axis)
    return out


def _signed(idx: np.ndarray, N: int) -> np.ndarray:
    return np.where(idx < N // 2, idx, idx - N) if N > 0 else idx


def direct_sum(u_hat: np.ndarray, x: np.ndarray, L: float = 2.0 * math.pi) -> tuple[np.ndarray, np.ndarray]:
    """Direct trigonometric sum u(x) = sum_k u_hat_k exp(i 2pi/L k.x) and its gradient (Section 2).

    The half spectrum is summed with real-to-complex weights: modes with
    0 < kz < N/2 count twice (their conjugate partner is implied), the kz = 0
    and kz = N/2 planes once, and the real part is taken.  This is what an
    inverse real transform computes at the grid nodes.
    """
    u_hat = np.asarray(u_hat)
    N = u_hat.shape[1]
    nz = np.nonzero(np.any(u_hat != 0, axis=0))
    idx = np.stack(nz, axis=1)
    val = u_hat[:, nz[0], nz[1], nz[2]].astype(np.complex128)
    return direct_sum_modes(N, idx, val, x, L)


def direct_sum_modes(N: int, idx: np.ndarray, val: np.ndarray, x: np.ndarray,
                     L: float = 2.0 * math.pi) -> tuple[np.ndarray, np.ndarray]:
    """direct_sum over an explicit list of modes (index array [M, 3] into the half spectrum, values [3, M])."""
    return _direct_sum_modes(N, np.asarray(idx), np.asarray(val, dtype=np.complex128),
                             np.asarray(x, dtype=np.float64), L)


def _direct_sum_modes(N, idx, val, x, L, chunk_elems: int = 1 << 22):
    """Re sum_k m_k a_k exp(i K.x) and its gradient Re sum_k m_k a_k i K_j exp(i K.x), written with
    cos/sin of the phase; modes are taken in chunks of at most chunk_elems (particle, mode) pairs."""
    kx = _signed(idx[:, 0], N).astype(np.float64)
    ky = _signed(idx[:, 1], N).astype(np.float64)
    kz = idx[:, 2].astype(np.float64)
    mult = np.where((idx[:, 2] == 0) | (2 * idx[:, 2] == N), 1.0, 2.0)
    w = 2.0 * math.pi / L
    P = x.shape[0]
    u = np.zeros((P, 3))
    g = np.zeros((P, 3, 3))
    K = np.stack([kx, ky, kz], axis=1) * w                # [M, 3] physical wavenumbers
    chunk_modes = max(1, chunk_elems // max(P, 1))
    for m0 in range(0, idx.shape[0], chunk_modes):
        Kc = K[m0:m0 + chunk_modes]
        phase = x @ Kc.T                                     # [P, Mc]
        cs, sn = np.cos(phase), np.sin(phase)
        del phase
        for c in range(3):
            a = val[c, m0:m0 + chunk_modes] * mult[m0:m0 + chunk_modes]
            re = cs @ a.real - sn @ a.imag                   # Re(a e^{i phase}) summed over modes
            u[:, c] += re
            for j in range(3):
                # Re(i K_j a e^{i phase}) = -K_j Im(a e^{i phase})
                g[:, c, j] -= cs @ (Kc[:, j] * a.imag) + sn @ (Kc[:, j] * a.real)
    return u, g


def _zeta_excl0(kappa: np.ndarray, q: int, alternating: bool, n_terms: int = 4000) -> np.ndarray:
    """sum over i != 0 of s_i (kappa + i)^(-q), s_i = (-1)^i if alternating else 1.

    Summed directly for |i| <= n_terms; the non-alternating tail beyond is
    added by the midpoint rule, int_{n_terms+1/2}^inf of (x + kappa)^(-q) + (x - kappa)^(-q).
    """
    kappa = np.asarray(kappa, dtype=np.float64)
    i = np.arange(1, n_terms + 1, dtype=np.float64)
    s = (-1.0) ** i if alternating else np.ones_like(i)
    tot = (s * ((kappa[..., None] + i) ** (-q) + (kappa[..., None] - i) ** (-q))).sum(axis=-1)
    if not alternating:
        a = n_terms + 0.5
        tot = tot + ((a + kappa) ** (1 - q) + (a - kappa) ** (1 - q)) / (q - 1)
    return tot


def _alias_sums(kappa: np.ndarray, n: int, kind: str):
    """Per-axis transfer of one mode through prefilter and kernel (Section 5, Eq. discrete).

    The interpolant of the 1D mode kappa has components at kappa + i with
    amplitude F(kappa + i) = c(kappa) sinc(kappa + i)^n.  Returns
    F0 = F(kappa), D = F0 - 1, E0 = sum_{i != 0} F(kappa + i)^2 and
    E1 = sum_{i != 0} (kappa + i)^2 F(kappa + i)^2.  Using
    sinc(kappa + i) = (-1)^i sin(pi kappa) / (pi (kappa + i)), the alias sums
    are power sums over i, evaluated without cancellation; D uses the
    interpolating prefilter's identity 1/c = sum_i sinc(kappa + i)^n (Poisson
    summation of the node values).
    """
    kappa = np.asarray(kappa, dtype=np.float64)
    sn = np.sin(np.pi * kappa) / np.pi
    sk = sinc(kappa) ** n
    if kind == "interp":
        c = 1.0 / transfer_discrete(kappa, n)
        # 1/c - sinc^n = sum_{i != 0} sinc(kappa + i)^n
        rest = sn ** n * _zeta_excl0(kappa, n, alternating=(n % 2 == 1))
        D = -c * rest
    else:
        c = sk / transfer_discrete(kappa, 2 * n)
        D = c * sk - 1.0
    F0 = c * sk
    E0 = c ** 2 * sn ** (2 * n) * _zeta_excl0(kappa, 2 * n, alternating=False)
    E1 = c ** 2 * sn ** (2 * n) * _zeta_excl0(kappa, 2 * n - 2, alternating=False)
    return F0, D, E0, E1


def l2_error_mode(kappa: np.ndarray, n: int, l: int = 0, kind: str = "interp",
                  n_alias: int | None = None) -> np.ndarray:
    """Relative squared L2 error of one Fourier mode (Eqs. l2-error, l2-error-der), l = 0 or 1.

    l = 0: (F(kappa) - 1)^2 + sum_{i != 0} F(kappa + i)^2;
    l = 1: (F(kappa) - 1)^2 + sum_{i != 0} ((kappa + i)/kappa)^2 F(kappa + i)^2.
    If n_alias is given, the alias sum is instead the plain sum over 0 < |i| <= n_alias.
    """
    kappa = np.asarray(kappa, dtype=np.float64)
    if n_alias is not None:
        c = (1.0 / transfer_discrete(kappa, n) if kind == "interp"
             else sinc(kappa) ** n / transfer_discrete(kappa, 2 * n))
        i = np.arange(-n_alias, n_alias + 1, dtype=np.float64)
        i = i[i != 0]
        F0 = c * sinc(kappa) ** n
        Fi = c[..., None] * sinc(kappa[..., None] + i) ** n
        ratio = ((kappa[..., None] + i) / kappa[..., None]) ** (2 * l)
        return (F0 - 1.0) ** 2 + (ratio * Fi ** 2).sum(axis=-1)
    F0, D, E0, E1 = _alias_sums(kappa, n, kind)
    if l == 0:
        return D ** 2 + E0
    if l == 1:
        return D ** 2 + E1 / kappa ** 2
    raise ValueError("closed form only for l = 0, 1")


def l2_error_field(N: int, idx: np.ndarray, val: np.ndarray, n: int, L: float = 2.0 * math.pi,
                   kind: str = "interp") -> tuple[np.ndarray, np.ndarray]:
    """Predicted domain-mean squared interpolation error of u_c and of d u_c / d x_d.

    By the orthogonality Theorem of Section 5 the squared error of a sum of
    modes is the sum of the per-mode squared errors weighted by |u_hat_k|^2.
    In 3D each mode's interpolant is the product of the three 1D interpolants
    (Eq. condition), so its components sit at kappa + (i, j, l) with amplitude
    F_x(i) F_y(j) F_z(l).  The squared error of the value is
    (prod_a F0_a - 1)^2 + [prod_a (F0_a^2 + E0_a) - prod_a F0_a^2]; for the
    derivative along axis d the factor of axis d carries (kappa_d + i)^2, i.e.
    E0_d becomes E1_d and F0_d^2 becomes kappa_d^2 F0_d^2.  Modes of the half
    spectrum with 0 < kz < N/2 count twice.  Returns (mse_u [3], mse_grad [3][3]).
    """
    idx = np.asarray(idx)
    val = np.asarray(val, dtype=np.complex128)
    k = np.stack([_signed(idx[:, 0], N), _signed(idx[:, 1], N), idx[:, 2]], axis=1).astype(np.float64)
    kappa = k / N
    # per-axis factors depend only on the signed wavenumber: tabulate them for -N/2..N/2
    ktab = np.arange(-(N // 2), N // 2 + 1, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        tabs = _alias_sums(ktab / N, n, kind)
    # kappa = 0: the mode is constant along that axis, reproduced exactly (c(0) sinc(i)^n = delta_i0)
    z0 = ktab == 0
    tabs = [np.where(z0, v0, t) for t, v0 in zip(tabs, (1.0, 0.0, 0.0, 0.0))]
    pos = (k + N // 2).astype(np.int64)
    F0, D, E0, E1 = (t[pos] for t in tabs)                    # [M, 3] each
    mult = np.where((idx[:, 2] == 0) | (2 * idx[:, 2] == N), 1.0, 2.0)
    amp2 = np.abs(val) ** 2 * mult[None, :]                   # [3, M]
    # prod F0 - 1 = (1+Dx)(1+Dy)(1+Dz) - 1, expanded
    Dx, Dy, Dz = D[:, 0], D[:, 1], D[:, 2]
    Pm1 = Dx + Dy + Dz + Dx * Dy + Dx * Dz + Dy * Dz + Dx * Dy * Dz
    A = F0 ** 2
    full = A + E0

    def excess(fa, fb, fc, aa, ab, ac):
        # fa fb fc - aa ab ac with f = a + e, e >= 0, as a sum of nonnegative terms
        return (fa - aa) * fb * fc + aa * (fb - ab) * fc + aa * ab * (fc - ac)

    eps_u = Pm1 ** 2 + excess(full[:, 0], full[:, 1], full[:, 2], A[:, 0], A[:, 1], A[:, 2])
    mse_u = (amp2 * eps_u[None, :]).sum(axis=1)
    w = 2.0 * math.pi / L
    mse_g = np.zeros((3, 3))
    for d in range(3):
        o = [a for a in range(3) if a != d]
        kd2A = kappa[:, d] ** 2 * A[:, d]
        full_d = kd2A + E1[:, d]
        ex = excess(full_d, full[:, o[0]], full[:, o[1]], kd2A, A[:, o[0]], A[:, o[1]])
        eps = kappa[:, d] ** 2 * Pm1 ** 2 + ex                  # in units of N^2
        mse_g[:, d] = (w * N) ** 2 * (amp2 * eps[None, :]).sum(axis=1)
    return mse_u, mse_g


def table1_fma_count(n: int) -> int:
    """Cost of u and all first derivatives of a 3-component field per point (Table 1)."""
    return 6 * n ** 3 + 15 * n ** 2 + 12 * n


# ---------------------------------------------------------------------------
# Adjoint of the path (differentiation with respect to u_hat and positions).
# The paper has no adjoint; these are the transposes of the linear maps above
# (Sections 3-4 and 7), written out, plus second-derivative weights for the
# position gradient (the derivative of Eq. interpolation2 in x).
# ---------------------------------------------------------------------------

def weights2(t: np.ndarray, n: int) -> np.ndarray:
    """Second-derivative weights W''[p, j] = sum_i (M D D)[j, i] t_p^i (monomial form)."""
    t = np.asarray(t, dtype=np.float64)
    M = bspline_matrix(n)
    D = derivative_matrix(n)
    xbar = t[..., None] ** np.arange(n, dtype=np.float64)
    return xbar @ (M @ D @ D).T


def _valid_positions(x: np.ndarray) -> np.ndarray:
    return np.all(np.isfinite(x), axis=1)


def hessian(coef: np.ndarray, x: np.ndarray, n: int, L: float = 2.0 * math.pi,
            chunk: int = 4096) -> np.ndarray:
    """H[p][c][d][e] = d^2 u_c / dx_d dx_e of the B-spline interpolant at x (physical units).

    Each entry is the stencil contraction of Eq. interpolation with, per axis,
    W, W' or W'' by how often that axis is differentiated, scaled by (N / L)^2.
    """
    coef = np.asarray(coef, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    N = coef.shape[1]
    P = x.shape[0]
    H = np.empty((P, 3, 3, 3))
    scale2 = (float(N) / float(L)) ** 2
    for p0 in range(0, P, chunk):
        xs = x[p0:p0 + chunk]
        nodes, t = locate(xs, N, n, L)
        W = weights(t, n)
        sets = (W[0], W[1], weights2(t, n))            # derivative order 0, 1, 2 -> [p, 3, n]
        ix = nodes[:, 0, :, None, None]
        iy = nodes[:, 1, None, :, None]
        iz = nodes[:, 2, None, None, :]
        for c in range(3):
            B = coef[c][ix, iy, iz]
            for d in range(3):
                for e in range(3):
                    k = [0, 0, 0]
                    k[d] += 1
                    k[e] += 1
                    H[p0:p0 + chunk, c, d, e] = scale2 * np.einsum(
                        "pabc,pa,pb,pc->p", B, sets[k[0]][:, 0], sets[k[1]][:, 1], sets[k[2]][:, 2])
    return H


def spread(x: np.ndarray, g_u: np.ndarray, g_grad: np.ndarray | None, N: int, n: int,
           L: float = 2.0 * math.pi, chunk: int = 4096) -> np.ndarray:
    """Adjoint of evaluate() in the coefficients: g_coef [3][N][N][N].

    g_coef[c][node] = sum_p g_u[p, c] W_x W_y W_z + (N / L) sum_p sum_e g_grad[p, c, e] (W with W' on axis e),
    summed over every particle whose stencil covers the node.  Particles with
    non-finite positions contribute nothing.
    """
    x = np.asarray(x, dtype=np.float64)
    g_u = np.asarray(g_u, dtype=np.float64)
    g_grad = None if g_grad is None else np.asarray(g_grad, dtype=np.float64)
    out = np.zeros((3, N, N, N))
    scale = float(N) / float(L)
    ok = _valid_positions(x)
    for p0 in range(0, x.shape[0], chunk):
        sel = np.nonzero(ok[p0:p0 + chunk])[0] + p0
        if sel.size == 0:
            continue
        nodes, t = locate(x[sel], N, n, L)
        W, W1 = weights(t, n)
        ix = np.broadcast_to(nodes[:, 0, :, None, None], (sel.size, n, n, n))
        iy = np.broadcast_to(nodes[:, 1, None, :, None], (sel.size, n, n, n))
        iz = np.broadcast_to(nodes[:, 2, None, None, :], (sel.size, n, n, n))
        for c in range(3):
            T = g_u[sel, c, None, None, None] * np.einsum("pa,pb,pc->pabc", W[:, 0], W[:, 1], W[:, 2])
            if g_grad is not None:
                T = T + scale * (
                    g_grad[sel, c, 0, None, None, None] * np.einsum("pa,pb,pc->pabc", W1[:, 0], W[:, 1], W[:, 2])
                    + g_grad[sel, c, 1, None, None, None] * np.einsum("pa,pb,pc->pabc", W[:, 0], W1[:, 1], W[:, 2])
                    + g_grad[sel, c, 2, None, None, None] * np.einsum("pa,pb,pc->pabc", W[:, 0], W[:, 1], W1[:, 2]))
            np.add.at(out[c], (ix, iy, iz), T)
    return out


def position_gradient(coef: np.ndarray, x: np.ndarray, g_u: np.ndarray, g_grad: np.ndarray | None,
                      n: int, L: float = 2.0 * math.pi) -> np.ndarray:
    """g_x[p][d] = sum_c g_u[p, c] du_c/dx_d + sum_{c, e} g_grad[p, c, e] d^2 u_c / dx_e dx_d.

    NaN for non-finite positions.
    """
    x = np.asarray(x, dtype=np.float64)
    g_u = np.asarray(g_u, dtype=np.float64)
    out = np.full((x.shape[0], 3), np.nan)
    ok = _valid_positions(x)
    if not ok.any():
        return out
    xs = x[ok]
    _, grad = evaluate(coef, xs, n, L)
    gx = np.einsum("pc,pcd->pd", g_u[ok], grad)
    if g_grad is not None:
        H = hessian(coef, xs, n, L)
        gx = gx + np.einsum("pce,pced->pd", np.asarray(g_grad, dtype=np.float64)[ok], H)
    out[ok] = gx
    return out


def real_transform_multiplicity(N: int) -> np.ndarray:
    """m(kz) on the half spectrum: 1 for kz = 0 and kz = N/2, 2 otherwise (how often an
    inverse real transform counts the stored mode)."""
    m = np.full(N // 2 + 1, 2.0)
    m[0] = 1.0
    if N % 2 == 0:
        m[N // 2] = 1.0
    return m


def adjoint_transform(g_coef: np.ndarray, n: int, kind: str = "interp") -> np.ndarray:
    """Adjoint of coefficients(): g_u_hat [3][N][N][N//2+1] from g_coef [3][N][N][N].

    coefficients() is u_hat -> inverse real transform of c(kx) c(ky) c(kz) u_hat.
    For a real loss with gradient g_coef, the gradient with respect to the
    half spectrum (real and imaginary parts, as d/dRe + i d/dIm) is
    c(kx) c(ky) c(kz) m(kz) sum_x g_coef(x) exp(-2 pi i k.x / N): the
    unnormalised forward real transform, counted m(kz) times.
    """
    g_coef = np.asarray(g_coef, dtype=np.float64)
    N = g_coef.shape[1]
    c = prefilter(N, n) if kind == "interp" else prefilter_l2(N, n)
    G = np.fft.rfftn(g_coef, axes=(1, 2, 3), norm="backward")
    nh = N // 2 + 1
    f = c[:, None, None] * c[None, :, None] * (c[:nh] * real_transform_multiplicity(N))[None, None, :]
    return G * f[None]


def interpolate_adjoint(u_hat: np.ndarray, x: np.ndarray, g_u: np.ndarray, g_grad: np.ndarray | None,
                        n: int, L: float = 2.0 * math.pi, kind: str = "interp"):
    """Gradients of sum g_u . u + sum g_grad . grad u through the whole path:
    (g_u_hat, g_x, g_coef)."""
    N = np.asarray(u_hat).shape[1]
    g_coef = spread(x, g_u, g_grad, N, n, L)
    g_x = position_gradient(coefficients(u_hat, n, kind), x, g_u, g_grad, n, L)
    return adjoint_transform(g_coef, n, kind), g_x, g_coef
