"""Pins of the oracle's adjoint / PSD gradient (derived from Eq. 3) -- CPU only."""
import numpy as np
import pytest

from oracle import adjoint, noise
from oracle.pcg import dense_solve
from oracle.system import Problem
from paper_1408_3048_gb300 import synth
from problems import tiny_scan


def _problem(scan, psds=None):
    return Problem(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd,
                   scan.psds if psds is None else psds, scan.fsamp, scan.lam, scan.ncomp)


def _loss(prob, d, mref):
    m = dense_solve(prob.dense_A(), prob.rhs(d))
    return 0.5 * np.sum((m - mref) ** 2), m


@pytest.fixture(scope="module", params=[1, 3])
def setup(request):
    ncomp = request.param
    scan = tiny_scan(ncomp=ncomp, psds=((1.0, 2.0, 1.5), (1.3, 0.7, 1.2)), lam=8)
    prob = _problem(scan)
    rng = np.random.default_rng(ncomp)
    d = synth.tod(scan, synth.sky_map(scan.npix_sky, ncomp, 3), rng.standard_normal(scan.nt))
    mref = rng.standard_normal(prob.n)
    return scan, prob, d, mref


def test_row_derivatives_match_finite_differences():
    L, lam = 4096, 40
    th = np.array([1.3, 0.8, 1.4])
    D = adjoint.row_derivatives(*th, L, 100.0, lam)
    for c in range(3):
        h = 1e-5 * th[c]
        tp, tm = th.copy(), th.copy()
        tp[c] += h
        tm[c] -= h
        fd = (noise.toeplitz_row(*tp, L, 100.0, lam) - noise.toeplitz_row(*tm, L, 100.0, lam)) / (2 * h)
        assert np.abs(fd - D[c]).max() <= 1e-7 * np.abs(D[c]).max()
    # closed form: t scales as 1/sigma^2
    t = noise.toeplitz_row(*th, L, 100.0, lam)
    np.testing.assert_allclose(D[0], -2.0 / th[0] * t, rtol=1e-12, atol=1e-15)
    # direct cosine-sum route equals the FFT route
    Dd = adjoint.row_derivatives(*th, L, 100.0, lam, route="direct")
    assert np.abs(Dd - D).max() <= 1e-12 * np.abs(D).max()


def test_lagged_products_equal_dense_form(setup):
    scan, prob, d, mref = setup
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal(prob.nt), rng.standard_normal(prob.nt)
    np.testing.assert_allclose(adjoint.psd_gradient(prob, u, v), adjoint.dense_psd_gradient(prob, u, v),
                               rtol=1e-10, atol=1e-12)


def test_gradient_wrt_data_matches_finite_differences(setup):
    scan, prob, d, mref = setup
    L0, m = _loss(prob, d, mref)
    dLdd, _ = adjoint.gradients(prob, d, m, m - mref, dense=True)
    rng = np.random.default_rng(7)
    for _ in range(3):
        e = rng.standard_normal(prob.nt)
        h = 1e-4
        fd = (_loss(prob, d + h * e, mref)[0] - _loss(prob, d - h * e, mref)[0]) / (2 * h)
        assert fd == pytest.approx(dLdd @ e, rel=1e-7, abs=1e-9)


def test_gradient_wrt_psd_matches_finite_differences(setup):
    scan, prob, d, mref = setup
    L0, m = _loss(prob, d, mref)
    _, G = adjoint.gradients(prob, d, m, m - mref, dense=True)
    for p in range(len(scan.psds)):
        for c in range(3):
            th = np.array(scan.psds, dtype=np.float64)
            h = 1e-4 * th[p, c]
            tp, tm = th.copy(), th.copy()
            tp[p, c] += h
            tm[p, c] -= h
            fd = (_loss(_problem(scan, tp), d, mref)[0] - _loss(_problem(scan, tm), d, mref)[0]) / (2 * h)
            assert fd == pytest.approx(G[p, c], rel=1e-5, abs=1e-8 * np.abs(G).max()), (p, c)


def test_shared_sigma_gradient_is_zero():
    # one PSD for every interval: scaling N^-1 leaves m unchanged, so dL/dsigma = 0
    scan = tiny_scan(ncomp=3, psds=((1.4, 1.5, 1.3),), lam=8)
    prob = _problem(scan)
    rng = np.random.default_rng(2)
    d = rng.standard_normal(prob.nt)
    L0, m = _loss(prob, d, rng.standard_normal(prob.n))
    g = m - rng.standard_normal(prob.n)
    _, G = adjoint.gradients(prob, d, m, g, dense=True)
    assert abs(G[0, 0]) <= 1e-10 * np.abs(G[0, 1:]).max()


def test_white_noise_data_gradient_closed_form():
    # N^-1 = I / sigma^2: m is the per-pixel mean, so dL/dd_t = g_{p_t} / hits_{p_t}
    scan = tiny_scan(ncomp=1, psds=((0.8, 0.0, 1.0),), lam=4)
    prob = _problem(scan)
    g = np.random.default_rng(3).standard_normal(prob.n)
    dLdd = prob.Ninv(prob.P(dense_solve(prob.dense_A(), g)))
    ref = g[prob.pix_c] / prob.hits[prob.pix_c]
    np.testing.assert_allclose(dLdd, ref, rtol=1e-10, atol=1e-12)
