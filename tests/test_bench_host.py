"""Host-side logic of bench.py (no GPU): the headline workload and the algorithmic bytes that the
roofline's `achieved` figure divides by, each pinned to a count written out from the data layout."""
import bench


def test_headline_workload_is_512_cubed_quintic_with_2_pow_24_particles():
    wl = bench.workload()
    assert (wl["N"], wl["order"], wl["P"]) == (512, 6, 1 << 24)


def test_gather_algorithmic_bytes_at_the_headline():
    # three FP32 coefficient components read once; per particle a 16-byte record (first node, t per
    # axis) and a 4-byte index read, u (3) and grad u (9) FP32 values written
    N, P = 512, 1 << 24
    want = 3 * N ** 3 * 4 + P * (16 + 4) + P * 12 * 4
    assert want == 2_751_463_424
    assert bench.algorithmic_bytes("gather", N, P, "f32", 6) == want


def test_transform_algorithmic_bytes_count_the_unpadded_half_spectrum():
    N = 512
    spec = 3 * N * N * (N // 2 + 1) * 8          # complex64 half spectrum
    assert bench.algorithmic_bytes("fft_x", N, 0, "f32") == 2 * spec
    assert bench.algorithmic_bytes("fft_yz", N, 0, "f32") == spec + 3 * N ** 3 * 4
    # FP64 plans: complex128 spectrum and FP64 coefficients
    assert bench.algorithmic_bytes("fft_yz", N, 0, "f64") == 2 * spec + 3 * N ** 3 * 8


def test_sort_algorithmic_bytes():
    P = 1000
    assert bench.algorithmic_bytes("bin", 64, P, "f32") == 24 * P                 # positions read
    assert bench.algorithmic_bytes("scatter", 64, P, "f32") == 24 * P + 20 * P    # positions, record + index
    assert bench.algorithmic_bytes("scatter", 64, P, "f64") == 24 * P + 36 * P    # FP64 record


def test_scan_bytes_follow_the_brick_grid():
    # FP32, order 6: 16 x 12 x 16 bricks; 512^3 gives 32 * 43 * 32 bricks (the y axis rounds up)
    nb = 32 * 43 * 32
    assert bench.algorithmic_bytes("scan", 512, 0, "f32", 6) == 16 * (nb + 1)
    # order 8: 16 x 8 x 16
    nb8 = 32 * 64 * 32
    assert bench.algorithmic_bytes("scan", 512, 0, "f32", 8) == 16 * (nb8 + 1)


def test_e2e_host_to_device_bytes_full_and_band_box():
    # the full half spectrum, or only the modes of the band box (every signed |kx|, |ky| <= K, 0 <= kz <= K),
    # counted from a mask over the half spectrum's index grid; 8 bytes a complex64 mode, 24 a position
    import numpy as np
    for N, K, P in ((16, 5, 7), (48, 16, 100), (64, 21, 1), (32, 0, 3)):
        idx = np.arange(N)
        k = np.abs(np.where(idx <= N // 2, idx, idx - N))
        kz = np.arange(N // 2 + 1)
        inside = (k[:, None, None] <= K) & (k[None, :, None] <= K) & (kz[None, None, :] <= K)
        modes = 3 * (int(inside.sum()) if K else N * N * (N // 2 + 1))
        assert bench.e2e_h2d_bytes(N, P, K) == modes * 8 + P * 24
    assert bench.e2e_h2d_bytes(512, 1 << 24) == 3 * 512 * 512 * 257 * 8 + (1 << 24) * 24
