"""Pins of the oracle's pointing, Toeplitz and system operators -- CPU only."""
import numpy as np
import pytest

from oracle import pointing, toeplitz
from oracle.pcg import pcg, dense_solve
from oracle.precond import BlockJacobi
from paper_1408_3048_gb300 import synth
from problems import oracle_problem, tiny_scan


def test_hits_and_observed_set_brute_force():
    rng = np.random.default_rng(3)
    npix = 40
    pix = rng.integers(0, npix, size=300)
    pix[pix == 7] = 8          # pixel 7 never observed
    obs2sky, hits, pix_c = pointing.observed_pixels(pix, npix, 1)
    ref_hits = {}
    for p in pix:
        ref_hits[int(p)] = ref_hits.get(int(p), 0) + 1
    assert list(obs2sky) == sorted(ref_hits)
    assert [int(h) for h in hits] == [ref_hits[int(p)] for p in obs2sky]
    for t, p in enumerate(pix):
        assert obs2sky[pix_c[t]] == p


def test_polarisation_observed_set_brute_force():
    rng = np.random.default_rng(5)
    npix = 30
    pix = rng.integers(0, npix, size=200)
    phi = rng.uniform(0, np.pi, size=200)
    phi[pix == 3] = 0.4          # one angle only -> singular block -> dropped
    pix[:2] = 29                 # pixel 29: force exactly 2 hits -> dropped
    pix[pix == 29] = 28
    pix[:2] = 29
    w = np.stack([np.cos(2 * phi), np.sin(2 * phi)], axis=1)
    obs2sky, hits, pix_c = pointing.observed_pixels(pix, npix, 3, w, 1e-6)
    for p in range(npix):
        sel = pix == p
        keep = False
        if sel.sum() >= 3:
            W3 = np.stack([np.ones(sel.sum()), w[sel, 0], w[sel, 1]], axis=1)
            sv = np.linalg.svd(W3, compute_uv=False)      # B = W3^T W3 -> eig = sv^2
            keep = (sv[-1] / sv[0]) ** 2 >= 1e-6
        assert (p in set(obs2sky.tolist())) == keep, p
    assert 3 not in obs2sky and 29 not in obs2sky
    assert np.all(pix_c[np.isin(pix, [3, 29])] == -1)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_pointing_adjoint_and_dense(ncomp):
    scan = tiny_scan(ncomp=ncomp)
    pr = oracle_problem(scan)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(pr.n)
    y = rng.standard_normal(pr.nt)
    assert abs(y @ pr.P(x) - pr.PT(y) @ x) <= 1e-12 * np.abs(y).sum() * np.abs(x).max() * 3
    P = pr.dense_P()
    np.testing.assert_allclose(pr.P(x), P @ x, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pr.PT(y), P.T @ y, rtol=1e-13, atol=1e-12)
    # brute force gather of one sample
    t = 17
    q = pr.pix_c[t]
    ref = x[q * ncomp] + (scan.weights[t, 0] * x[q * 3 + 1] + scan.weights[t, 1] * x[q * 3 + 2] if ncomp == 3 else 0.0)
    assert abs(pr.P(x)[t] - ref) < 1e-14


def test_toeplitz_direct_equals_dense_and_fft():
    rng = np.random.default_rng(2)
    for n, lam in ((50, 7), (13, 12), (200, 0), (64, 30)):
        t = rng.standard_normal(lam + 1)
        y = rng.standard_normal(n)
        T = toeplitz.dense_block(t, n)
        zd = toeplitz.apply_block_direct(y, t)
        np.testing.assert_allclose(zd, T @ y, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(toeplitz.apply_block_fft(y, t), zd, rtol=1e-10, atol=1e-11)
        # brute force, one output
        k0 = n // 2
        ref = sum(t[abs(k)] * y[k0 + k] for k in range(-lam, lam + 1) if 0 <= k0 + k < n)
        assert abs(zd[k0] - ref) < 1e-12


def test_toeplitz_blocks_do_not_couple_intervals():
    offsets = np.array([0, 40, 100, 130])
    ipsd = np.array([0, 1, 0])
    rows = [np.array([2.0, -0.5, -0.2]), np.array([1.0, -0.3, 0.1])]
    y = np.zeros(130)
    y[39] = 1.0                          # last sample of interval 0
    z = toeplitz.apply_ninv(y, offsets, ipsd, rows)
    assert np.all(z[40:] == 0.0)
    np.testing.assert_allclose(z[37:40], [-0.2, -0.5, 2.0])
    N = toeplitz.dense_ninv(offsets, ipsd, rows)
    yy = np.random.default_rng(0).standard_normal(130)
    np.testing.assert_allclose(toeplitz.apply_ninv(yy, offsets, ipsd, rows), N @ yy, atol=1e-13)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_A_symmetric_positive_and_dense(ncomp):
    scan = tiny_scan(ncomp=ncomp)
    pr = oracle_problem(scan)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(pr.n)
    y = rng.standard_normal(pr.n)
    Ax, Ay = pr.A(x), pr.A(y)
    assert abs(y @ Ax - x @ Ay) <= 1e-13 * np.linalg.norm(Ax) * np.linalg.norm(y) * 10
    for _ in range(5):
        v = rng.standard_normal(pr.n)
        assert v @ pr.A(v) > 0
    A = pr.dense_A()
    np.testing.assert_allclose(Ax, A @ x, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(pr.A(x, route="fft"), Ax, rtol=1e-9, atol=1e-10)
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("ncomp", [1, 3])
def test_white_noise_gls_is_binned_map(ncomp):
    # f_knee = 0: N^-1 = I/sigma^2 and the GLS map is the hit-weighted binned map
    # (per pixel mean for T, per pixel 3x3 solve for I/Q/U), computed here by brute force.
    scan = tiny_scan(ncomp=ncomp, psds=((1.5, 0.0, 1.0),), lam=4)
    pr = oracle_problem(scan)
    d = np.random.default_rng(6).standard_normal(pr.nt)
    b = pr.rhs(d)
    bd = BlockJacobi(pr)
    res = pcg(pr.A, bd.apply, b, 1e-12, 50)
    assert res.iters == 1                 # M_BD = A^-1 for white noise
    ref = np.zeros(pr.n)
    for q, p in enumerate(pr.obs2sky):
        sel = np.nonzero(scan.pix == p)[0]
        if ncomp == 1:
            ref[q] = d[sel].mean()
        else:
            W3 = np.stack([np.ones(sel.size), scan.weights[sel, 0], scan.weights[sel, 1]], axis=1)
            ref[3 * q:3 * q + 3] = np.linalg.solve(W3.T @ W3, W3.T @ d[sel])
    np.testing.assert_allclose(res.x, ref, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_noiseless_data_recovers_sky(ncomp):
    scan = tiny_scan(ncomp=ncomp)
    pr = oracle_problem(scan)
    sky = synth.sky_map(scan.npix_sky, ncomp, 11)
    d = synth.tod(scan, sky, np.zeros(scan.nt))
    b = pr.rhs(d)
    res = pcg(pr.A, BlockJacobi(pr).apply, b, 1e-13, 500)
    assert res.converged
    np.testing.assert_allclose(res.x.reshape(-1, ncomp), sky[pr.obs2sky], rtol=1e-8, atol=1e-8)


def test_pcg_matches_dense_cholesky():
    scan = tiny_scan(ncomp=3)
    pr = oracle_problem(scan)
    d = np.random.default_rng(7).standard_normal(pr.nt)
    b = pr.rhs(d)
    ref = dense_solve(pr.dense_A(), b)
    res = pcg(pr.A, BlockJacobi(pr).apply, b, 1e-12, 1000)
    assert np.linalg.norm(res.x - ref) / np.linalg.norm(ref) < 1e-9


def test_problem_validation():
    scan = tiny_scan()
    with pytest.raises(ValueError):
        oracle_problem(scan.__class__(**{**scan.__dict__, "lam": 10 ** 6}))
    bad = scan.__dict__.copy()
    bad["offsets"] = scan.offsets.copy()
    bad["offsets"][1] = bad["offsets"][2]
    with pytest.raises(ValueError):
        oracle_problem(scan.__class__(**bad))
