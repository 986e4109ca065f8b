"""The seeded input recipes hold the properties stated for them (no GPU): the Kolmogorov-spectrum field
(band 1 <= |k| <= N/3, divergence-free, Hermitian k_z = 0 plane, u_rms = 1, E(k) ~ k^(-5/3)), the
clustered and uniform particle sets, and the batch workload's particle count."""
import math

import numpy as np

from paper_1201_4060_gb300 import synth


def _signed(i, N):
    return np.where(i <= N // 2, i, i - N)


def test_kolmogorov_field_band_divergence_hermitian_and_unit_rms():
    N = 48
    F = synth.kolmogorov_field(N, seed=1201)
    kx, ky, kz = _signed(F.idx[:, 0], N), _signed(F.idx[:, 1], N), F.idx[:, 2]
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    assert k2.min() >= 1 and k2.max() <= (N // 3) ** 2
    div = kx * F.val[0] + ky * F.val[1] + kz * F.val[2]
    assert np.abs(div).max() <= 1e-12 * np.abs(F.val).max()
    d = F.dense()
    plane = d[:, :, :, 0]
    mirror = np.conj(plane[:, (-np.arange(N)) % N][:, :, (-np.arange(N)) % N])
    assert np.array_equal(plane, mirror)
    # the real field u(x) = sum_k u_hat(k) exp(i k.x): mean of u_c^2 over the grid and the components
    u = np.fft.irfftn(d, s=(N, N, N), axes=(1, 2, 3)) * N ** 3
    assert abs((u ** 2).mean() - 1.0) < 1e-12
    # divergence-free on the grid as well: spectral derivative of the real field
    k = np.fft.fftfreq(N, 1.0 / N)
    ux = np.fft.irfftn(1j * k[:, None, None] * d[0], s=(N, N, N), axes=(0, 1, 2))
    uy = np.fft.irfftn(1j * k[None, :, None] * d[1], s=(N, N, N), axes=(0, 1, 2))
    uz = np.fft.irfftn(1j * np.arange(N // 2 + 1)[None, None, :] * d[2], s=(N, N, N), axes=(0, 1, 2))
    assert np.abs(ux + uy + uz).max() < 1e-12 * np.abs(ux).max()


def test_kolmogorov_shell_spectrum_slope():
    """|u_hat|^2 ~ |k|^(-11/3) on about 4 pi k^2 modes per shell: E(k) ~ k^(-5/3) (a seeded draw)."""
    N = 64
    F = synth.kolmogorov_field(N, seed=1201)
    kx, ky, kz = _signed(F.idx[:, 0], N), _signed(F.idx[:, 1], N), F.idx[:, 2]
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    energy = (np.abs(F.val) ** 2).sum(axis=0) * np.where(kz == 0, 1.0, 2.0)
    E = np.bincount(np.rint(kmag).astype(int), weights=energy)
    shells = np.arange(2, N // 3)
    slope = np.polyfit(np.log(shells), np.log(E[shells]), 1)[0]
    assert abs(slope + 5.0 / 3.0) < 0.15


def _cell_counts(x, cells=16):
    c = np.floor(x / (2 * math.pi / cells)).astype(int)
    return np.bincount((c[:, 0] * cells + c[:, 1]) * cells + c[:, 2], minlength=cells ** 3)


def test_particles_in_the_domain_uniform_and_clustered():
    P = 200_000
    xu = synth.uniform_particles(P, seed=5)
    xc = synth.clustered_particles(P, seed=5)
    for x in (xu, xc):
        assert x.shape == (P, 3) and x.dtype == np.float64
        assert x.min() >= 0.0 and x.max() < 2 * math.pi
    cu, cc = _cell_counts(xu), _cell_counts(xc)
    assert 0.8 < cu.var() / cu.mean() < 1.2          # Poisson: variance = mean
    assert cc.var() / cc.mean() > 20.0                # 40 % in Gaussian clumps of sigma 0.1
    assert np.array_equal(synth.clustered_particles(1000, seed=9), synth.clustered_particles(1000, seed=9))


def test_sort_by_cell_orders_raster_cells():
    N = 16
    x = synth.sort_by_cell(synth.uniform_particles(5000, seed=3), N)
    c = np.floor(x / (2 * math.pi / N)).astype(np.int64)
    key = (c[:, 0] * N + c[:, 1]) * N + c[:, 2]
    assert np.all(np.diff(key) >= 0)


def test_batch_workload_grids_and_particle_count():
    fields = synth.batch_workload()
    assert len(fields) == 64
    assert [f["N"] for f in fields[:6]] == list(synth.BATCH_GRIDS)
    assert all(1000 <= f["P"] < 1_000_000 for f in fields)
    assert sum(f["P"] for f in fields) == 8_380_148
