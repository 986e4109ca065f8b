"""Seeded synthetic inputs for the B-spline interpolation path.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds none of the interpolation method's arithmetic (no
prefilter, no transform, no B-spline weights, no particle location): only the
recipes that draw a periodic Fourier-space velocity field and particle
positions.

Field recipe (stands in for the dealiased pseudo-spectral turbulence fields of
Section 1 and the k_max*dx = 1/3 band of Section 8):

* modes with 1 <= |k| <= k_max, |k| the Euclidean norm of the signed integer
  wavenumber vector, k_max = N // 3 by default (2/3 dealiasing);
* |u_hat(k)|^2 proportional to |k|^(-11/3), i.e. the shell spectrum
  E(k) ~ k^(-5/3);
* a complex Gaussian (independent real and imaginary parts) per component;
* solenoidal projection u_hat <- u_hat - k (k . u_hat) / |k|^2;
* Hermitian symmetry u_hat(-k) = conj(u_hat(k)) on the k_z = 0 plane (the
  only plane of the half spectrum where both k and -k are stored);
* normalised to u_rms = 1 (mean over the three components).

Layout of a dense half spectrum: complex array [3][N][N][N//2+1], index
(c, kx, ky, kz); signed wavenumber k <-> index k mod N; kz >= 0 only.

Particle recipes: uniform in [0, L)^3, or clustered (60 % uniform, 40 % drawn
from isotropic Gaussians of standard deviation sigma around 64 uniform
centres, wrapped into [0, L)).
"""
from __future__ import annotations

import math

import numpy as np

L_DEFAULT = 2.0 * math.pi


class SparseField:
    """Nonzero modes of a half-spectrum field.

    idx: int64 [M, 3] array indices (ix, iy, iz) into [N][N][N//2+1];
    val: complex128 [3, M] mode values per component.
    """

    def __init__(self, N: int, idx: np.ndarray, val: np.ndarray):
        self.N = int(N)
        self.idx = idx
        self.val = val

    @property
    def nhalf(self) -> int:
        return self.N // 2 + 1

    def dense(self, dtype=np.complex128) -> np.ndarray:
        out = np.zeros((3, self.N, self.N, self.nhalf), dtype=dtype)
        ix, iy, iz = self.idx[:, 0], self.idx[:, 1], self.idx[:, 2]
        for c in range(3):
            out[c, ix, iy, iz] = self.val[c].astype(dtype)
        return out

    def rounded(self, dtype) -> "SparseField":
        """Same modes with values rounded to `dtype` and widened back to complex128."""
        return SparseField(self.N, self.idx, self.val.astype(dtype).astype(np.complex128))


def kolmogorov_field(N: int, seed: int, kmax: int | None = None) -> SparseField:
    """Divergence-free random field with E(k) ~ k^(-5/3) on 1 <= |k| <= kmax."""
    if kmax is None:
        kmax = N // 3
    kmax = int(min(kmax, N // 2 - 1))
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.arange(-kmax, kmax + 1, dtype=np.int64)
    rz = np.arange(0, kmax + 1, dtype=np.int64)
    kx, ky, kz = np.meshgrid(r, r, rz, indexing="ij")
    kx, ky, kz = kx.ravel(), ky.ravel(), kz.ravel()
    k2 = kx * kx + ky * ky + kz * kz
    band = (k2 >= 1) & (k2 <= kmax * kmax)
    # independent half of the kz = 0 plane: kx > 0, or kx == 0 and ky > 0
    indep = band & ((kz > 0) | (kx > 0) | ((kx == 0) & (ky > 0)))
    kx, ky, kz, k2 = kx[indep], ky[indep], kz[indep], k2[indep]
    M = kx.size
    kmag = np.sqrt(k2.astype(np.float64))
    amp = kmag ** (-11.0 / 6.0)
    g = rng.standard_normal((2, 3, M))
    v = (g[0] + 1j * g[1]) * amp[None, :]
    # solenoidal projection
    kvec = np.stack([kx, ky, kz]).astype(np.float64)
    kdotv = (kvec * v).sum(axis=0)
    v = v - kvec * (kdotv / k2.astype(np.float64))[None, :]
    # Hermitian mirror of the kz = 0 independent half
    on0 = kz == 0
    mkx, mky, mkz = -kx[on0], -ky[on0], kz[on0]
    mv = np.conj(v[:, on0])
    KX = np.concatenate([kx, mkx])
    KY = np.concatenate([ky, mky])
    KZ = np.concatenate([kz, mkz])
    V = np.concatenate([v, mv], axis=1)
    # normalise u_rms = 1: mean over components of sum over the full spectrum
    w = np.where(KZ == 0, 1.0, 2.0)
    energy = (np.abs(V) ** 2 * w[None, :]).sum() / 3.0
    V = V / math.sqrt(energy)
    idx = np.stack([np.mod(KX, N), np.mod(KY, N), KZ], axis=1).astype(np.int64)
    return SparseField(N, idx, V)


def random_half_spectrum(N: int, seed: int, hermitian: bool = True) -> np.ndarray:
    """Dense random half spectrum with every mode populated (edge-case input).

    With hermitian=True the self-conjugate structure of a real field's
    spectrum is imposed on the kz = 0 and kz = N/2 planes; with False the
    array is arbitrary complex data.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nh = N // 2 + 1
    a = rng.standard_normal((3, N, N, nh)) + 1j * rng.standard_normal((3, N, N, nh))
    if hermitian:
        for iz in ([0, N // 2] if N % 2 == 0 else [0]):
            p = a[:, :, :, iz]
            neg = np.conj(p[:, (-np.arange(N)) % N][:, :, (-np.arange(N)) % N])
            a[:, :, :, iz] = 0.5 * (p + neg)
    return a


def uniform_particles(P: int, seed: int, L: float = L_DEFAULT) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, L, size=(P, 3))


def clustered_particles(P: int, seed: int, L: float = L_DEFAULT, frac_uniform: float = 0.6,
                        n_centres: int = 64, sigma: float = 0.1) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    n_uni = int(round(frac_uniform * P))
    n_clu = P - n_uni
    uni = rng.uniform(0.0, L, size=(n_uni, 3))
    centres = rng.uniform(0.0, L, size=(n_centres, 3))
    which = rng.integers(0, n_centres, size=n_clu)
    clu = centres[which] + sigma * rng.standard_normal((n_clu, 3))
    clu = np.mod(clu, L)
    x = np.concatenate([uni, clu], axis=0)
    return x[rng.permutation(P)]


def sort_by_cell(x: np.ndarray, N: int, L: float = L_DEFAULT) -> np.ndarray:
    """Reorder positions in raster order of the grid cell that contains them (z fastest)."""
    c = np.clip(np.floor(np.mod(x, L) / (L / N)).astype(np.int64), 0, N - 1)
    key = (c[:, 0] * N + c[:, 1]) * N + c[:, 2]
    return x[np.argsort(key, kind="stable")]


def cotangents(P: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """N(0, 1) cotangents on u [P][3] and grad u [P][3][3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((P, 3)), rng.standard_normal((P, 3, 3))


# Workloads of the benchmark and parity suite (field seed 1201 + i, particle seed 4060 + i).
WORKLOADS = {
    "parity32": dict(N=32, order=4, P=10_000, field_seed=1202, particle_seed=4061, particles="uniform"),
    "orders256": dict(N=256, order=(2, 4, 6, 8), P=1_000_000, field_seed=1203, particle_seed=4062,
                      particles="uniform_sorted"),
    "throughput512": dict(N=512, order=6, P=1 << 24, field_seed=1204, particle_seed=4063, particles="clustered"),
    # adjoint (differentiation): N(0, 1) cotangents on u and grad u, seed = particle_seed + 1
    "adjoint256": dict(N=256, order=4, P=1 << 22, field_seed=1206, particle_seed=4065, particles="uniform"),
    # 64 independent small fields (batch_workload), cubic, FP32 coefficients
    "batch64": dict(nfields=64, order=4, field_seed=1205, particle_seed=4064, particles="uniform"),
}


BATCH_GRIDS = (32, 48, 64, 96, 128, 192)


def batch_workload(nfields: int = 64, field_seed: int = 1205, particle_seed: int = 4064,
                   p_range: tuple[float, float] = (1e3, 1e6)) -> list[dict]:
    """Many independent small fields: field i has grid BATCH_GRIDS[i % 6], field seed field_seed + i,
    uniform particles (seed particle_seed + i) whose count is log-uniform over p_range
    (mean (hi - lo) / ln(hi / lo), about 1.45e5 for the default range)."""
    rng = np.random.Generator(np.random.PCG64(particle_seed))
    lo, hi = np.log10(p_range[0]), np.log10(p_range[1])
    counts = np.floor(10.0 ** rng.uniform(lo, hi, nfields)).astype(np.int64)
    return [dict(N=BATCH_GRIDS[i % len(BATCH_GRIDS)], field_seed=field_seed + i, particle_seed=particle_seed + i,
                 P=int(counts[i])) for i in range(nfields)]


def make_particles(kind: str, P: int, seed: int, N: int, L: float = L_DEFAULT) -> np.ndarray:
    if kind == "uniform":
        return uniform_particles(P, seed, L)
    if kind == "uniform_sorted":
        return sort_by_cell(uniform_particles(P, seed, L), N, L)
    if kind == "clustered":
        return clustered_particles(P, seed, L)
    raise ValueError(kind)
