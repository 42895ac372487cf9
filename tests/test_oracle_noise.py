"""Pins of the oracle's noise model (Eq. 19, App. D / Eq. 28) -- CPU only."""
import numpy as np

from oracle import noise


def test_white_noise_row_is_inverse_variance():
    # f_knee = 0: the spectrum is flat, N^-1 = I / sigma^2 (closed form).
    for sigma in (1.0, 0.37, 2.5):
        for kind in (noise.WINDOW_GAUSS, noise.WINDOW_RECT):
            t = noise.toeplitz_row(sigma, 0.0, 1.0, 1024, 100.0, 64, kind)
            assert abs(t[0] - 1.0 / sigma**2) <= 1e-15 / sigma**2 * 4
            assert np.abs(t[1:]).max() <= 1e-15 / sigma**2 * 4


def test_row_scales_as_inverse_sigma_squared():
    a = noise.toeplitz_row(1.0, 0.7, 1.4, 2048, 100.0, 100)
    b = noise.toeplitz_row(3.0, 0.7, 1.4, 2048, 100.0, 100)
    np.testing.assert_allclose(b, a / 9.0, rtol=1e-13, atol=1e-17)


def test_direct_and_fft_rows_agree():
    for (L, lam) in ((64, 10), (512, 100), (2048, 300)):
        inv = noise.inverse_psd_grid(1.2, 1.5, 1.3, L, 100.0)
        d = noise.row_direct(inv, L, lam)
        f = noise.row_fft(inv, L, lam)
        assert np.abs(d - f).max() <= 1e-13 * np.abs(d).max()


def test_full_row_sums_to_zero_frequency_value():
    # Inverse DFT evaluated back at j = 0: r_0 + 2 sum_{0<k<L/2} r_k + r_{L/2} = 1/S_0,
    # which is 0 for 1/f noise (the f -> 0 limit) and 1/sigma^2 for white noise.
    L = 1024
    for fk, expect in ((1.0, 0.0), (0.0, 1.0 / 0.25)):
        inv = noise.inverse_psd_grid(0.5, fk, 1.0, L, 100.0)
        r = noise.row_direct(inv, L, L // 2)
        s = r[0] + 2.0 * r[1 : L // 2].sum() + r[L // 2]
        assert abs(s - expect) <= 1e-12 * max(1.0, np.abs(r).max())


def test_inverse_psd_grid_values():
    inv = noise.inverse_psd_grid(2.0, 1.0, 2.0, 8, 8.0)  # f_j = j Hz
    # S_j = 4 (1 + 1/j^2): j=1 -> 8, j=2 -> 5, j=4 -> 4.25
    assert inv[0] == 0.0
    np.testing.assert_allclose(inv[[1, 2, 4]], [1 / 8.0, 1 / 5.0, 1 / 4.25], rtol=1e-15)


def test_window_endpoints():
    w = noise.window(100)
    assert w[0] == 1.0
    assert abs(w[100] - np.exp(-2.0)) < 1e-16
    assert abs(w[50] - np.exp(-0.5)) < 1e-16
    assert np.all(noise.window(7, noise.WINDOW_RECT) == 1.0)


def test_grid_length():
    assert noise.grid_length([65536, 65536]) == 65536
    assert noise.grid_length([40000, 70000]) == 131072
    assert noise.grid_length([3]) == 4


def test_symbol_routes_agree_and_match_definition():
    t = noise.toeplitz_row(1.0, 1.0, 1.0, 4096, 100.0, 40)
    M = noise.symbol_grid_size(40)
    assert M == 512
    a = noise.symbol(t, M)
    b = noise.symbol_fft(t, M)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    # brute force at three frequencies
    for m in (0, 17, 255):
        w = 2 * np.pi * m / M
        ref = t[0] + 2 * sum(t[k] * np.cos(w * k) for k in range(1, 41))
        assert abs(a[m] - ref) <= 1e-13 * np.abs(a).max()


def test_symbol_bounds_finite_section_eigenvalues():
    # Eigenvalues of any finite section lie inside [min symbol, max symbol].
    from oracle.toeplitz import dense_block
    t = noise.toeplitz_row(1.0, 0.8, 1.5, 1024, 100.0, 12)
    s = noise.symbol(t, 4096)
    ev = np.linalg.eigvalsh(dense_block(t, 200))
    assert ev.min() >= s.min() - 1e-12 and ev.max() <= s.max() + 1e-12


def test_configuration_rows_are_spd_and_a_rect_row_is_not():
    # The GAUSS-windowed rows of the workloads pass reading R4 ...
    for (fk, al, lam, L) in ((1.0, 1.0, 1024, 65536), (2.0, 2.0, 4096, 131072), (0.1, 1.0, 4096, 131072)):
        assert noise.is_positive_definite(noise.toeplitz_row(1.0, fk, al, L, 100.0, lam))
    # ... (for alpha <= 2 every off-diagonal r_k is negative, so the symbol is smallest
    # at w = 0 where it equals -2 sum_{k > lambda} r_k > 0), while a hard-truncated
    # (RECT) row of a steeper spectrum has oscillating r_k and a negative symbol.
    bad = noise.toeplitz_row(1.0, 1.0, 4.0, 4096, 100.0, 64, noise.WINDOW_RECT)
    assert not noise.is_positive_definite(bad)
    t = noise.toeplitz_row(1.0, 0.5, 2.0, 4096, 100.0, 64, noise.WINDOW_RECT)
    assert np.all(t[1:] < 0) and noise.is_positive_definite(t)
