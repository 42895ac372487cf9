"""The synthetic inputs follow their stated recipe (CPU).  They stand in for the paper's
simulated scans (Sec. 4.1): a crossing raster at 4 samples per pixel, a polariser angle
that turns through 180 degrees over a detector's run, piecewise-stationary 1/f noise with
the PSD of Eq. 19 (exponent alpha), uneven stationary intervals, and an I/Q/U sky."""
import numpy as np
import pytest

from paper_1408_3048_gb300 import synth


def _raster_brute(W, H, ndet, nper, spp=4):
    """The raster rule written out sample by sample."""
    out = []
    half = nper // 2
    for d in range(ndet):
        for s in range(nper):
            if s < half:                       # rows, boustrophedon
                line, pos = divmod(s, spp * W)
                pos //= spp
                col = pos if line % 2 == 0 else W - 1 - pos
                row = (line + d * H // ndet) % H
            else:                              # columns, boustrophedon
                line, pos = divmod(s - half, spp * H)
                pos //= spp
                row = pos if line % 2 == 0 else H - 1 - pos
                col = (line + d * W // ndet) % W
            out.append(row * W + col)
    return np.array(out)


@pytest.mark.parametrize("W,H,ndet,nper", [(6, 5, 2, 240), (8, 8, 3, 1000), (5, 7, 1, 333)])
def test_raster_pointing_rule(W, H, ndet, nper):
    pix = synth.raster_pointing(W, H, ndet, nper)
    assert pix.dtype == np.int32 and pix.size == ndet * nper
    assert np.array_equal(pix, _raster_brute(W, H, ndet, nper))
    # 4 consecutive samples per pixel along a sweep
    assert np.all(pix[:4] == pix[0]) and pix[4] != pix[0]


def test_polariser_angle_turns_half_a_circle_per_detector():
    ndet, nper = 3, 1000
    w = synth.polariser_weights(ndet, nper, 42)
    np.testing.assert_allclose(w[:, 0] ** 2 + w[:, 1] ** 2, 1.0, atol=1e-14)
    two_phi = np.unwrap(np.arctan2(w[:, 1], w[:, 0]).reshape(ndet, nper), axis=1)
    # 2 phi_t - 2 phi_0 = 2 pi t / T_d
    expect = 2 * np.pi * np.arange(nper) / nper
    for d in range(ndet):
        np.testing.assert_allclose(two_phi[d] - two_phi[d, 0], expect, atol=1e-9)


def test_bench_workload_tables():
    """The 2^24-sample polarised workload: 16 detectors x 2^20 samples, 16 uneven intervals
    per detector (U[2^15, 2^17] rescaled to fill the detector), one PSD per detector with
    sigma = 1, f_knee in [0.1, 2] Hz, alpha in [1, 2]; lambda = 4096; 256 x 256 patch."""
    scan = synth.config(2)
    assert scan.nt == 2 ** 24 and scan.ncomp == 3 and scan.npix_sky == 256 * 256 and scan.lam == 4096
    assert scan.K == 256 and scan.offsets[0] == 0 and scan.offsets[-1] == scan.nt
    lengths = np.diff(scan.offsets).reshape(16, 16)
    assert np.all(lengths.sum(axis=1) == 2 ** 20)
    assert lengths.min() >= 2 ** 14 and lengths.max() <= 2 ** 17 and scan.lam < lengths.min()
    assert np.array_equal(scan.interval_psd.reshape(16, 16), np.repeat(np.arange(16)[:, None], 16, axis=1))
    psds = np.asarray(scan.psds)
    assert np.all(psds[:, 0] == 1.0)
    assert np.all((psds[:, 1] >= 0.1) & (psds[:, 1] <= 2.0)) and np.all((psds[:, 2] >= 1.0) & (psds[:, 2] <= 2.0))
    # every detector's samples sit in its own contiguous run of intervals
    assert np.all(scan.offsets[::16] == np.arange(17) * 2 ** 20)


def test_noise_is_coloured_by_its_psd():
    """Averaged periodogram of many realisations of one interval against
    S(f) = sigma^2 (1 + (f_knee / f)^alpha) (the periodogram of irfft(rfft(xi) sqrt(S))
    has expectation S(f) at every f_j > 0)."""
    m, R = 4096, 64
    offsets = np.array([0, m])
    sigma, fk, al = 1.3, 1.5, 1.4
    P = np.zeros(m // 2 + 1)
    for r in range(R):
        n = synth.noise_realisation(offsets, np.array([0]), np.array([[sigma, fk, al]]), 100.0, r)
        P += np.abs(np.fft.rfft(n)) ** 2 / m
    P /= R
    f = np.arange(m // 2 + 1) * 100.0 / m
    S = sigma ** 2 * (1.0 + (fk / f[1:]) ** al)
    ratio = P[1:-1] / S[:-1]
    # each bin averages R exponential variates (relative sd 1/sqrt(R)); bands of 64 bins
    bands = ratio[: (ratio.size // 64) * 64].reshape(-1, 64).mean(axis=1)
    assert np.all(np.abs(bands - 1.0) < 5.0 / np.sqrt(R * 64))
    # white noise: variance sigma^2 over a long run
    n = synth.noise_realisation(np.array([0, 2 ** 18]), np.array([0]), np.array([[0.7, 0.0, 1.0]]), 100.0, 9)
    assert np.var(n) == pytest.approx(0.49, rel=0.02)


def test_sky_and_data():
    x = synth.sky_map(20000, 3, 5)
    assert np.std(x[:, 0]) == pytest.approx(1.0, rel=0.03)
    assert np.std(x[:, 1]) == pytest.approx(0.1, rel=0.03) and np.std(x[:, 2]) == pytest.approx(0.1, rel=0.03)
    scan = synth.raster_scan(8, 8, 2, 512, 3, 2, 8, [(1.0, 1.0, 1.0)], seed=3)
    sky = synth.sky_map(scan.npix_sky, 3, 1)
    d = synth.tod(scan, sky, np.zeros(scan.nt))
    t = 100
    p = scan.pix[t]
    assert d[t] == pytest.approx(sky[p, 0] + scan.weights[t, 0] * sky[p, 1] + scan.weights[t, 1] * sky[p, 2],
                                 abs=1e-15)


def test_uneven_lengths_sum_and_range():
    rng = np.random.default_rng(0)
    for _ in range(20):
        v = synth.uneven_lengths(2 ** 20, 16, 2 ** 15, 2 ** 17, rng)
        assert v.sum() == 2 ** 20 and v.min() > 0
    v = synth.sequential_lengths(10 ** 6, 2 ** 16, 2 ** 18, rng)
    assert v.sum() == 10 ** 6 and np.all(v[:-1] >= 2 ** 16) and np.all(v[:-1] <= 2 ** 18) and v[-1] >= 2 ** 16
