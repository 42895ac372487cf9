"""Property tests of the oracle on random tiny problems (hypothesis; CPU only).

Random pointings (any pixel hit any number of times, unobserved and ill-conditioned
I/Q/U pixels included), random interval partitions with lengths from 8 samples, one or
two noise PSDs, and half bandwidths from 0 up to half the shortest interval.  On each the
algebraic facts the paper fixes must hold: P and P^T are adjoint (Eq. 2, Sec. 2), the
matrix-free A equals the dense P^T N^-1 P (Eq. 5, 8), it is symmetric positive definite
(Sec. 3.1), white noise makes the GLS map the hit-weighted binned map (M_BD = A^-1,
Sec. 3.2), PCG reaches the dense solution (Eq. 3), and the two-level operator satisfies
R A Z = 0 and M_2lvl A Z = Z (Eq. 11, 13) for any coarse basis.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, assume, given, settings
from hypothesis import strategies as st

from oracle import precond, toeplitz
from oracle.pcg import dense_solve, pcg
from oracle.system import Problem

SETTINGS = settings(max_examples=50, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])


@st.composite
def problems(draw, white=False):
    ncomp = draw(st.sampled_from([1, 3]))
    npix = draw(st.integers(2, 12))
    lengths = draw(st.lists(st.integers(8, 60), min_size=1, max_size=4))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    nt = int(sum(lengths))
    pix = rng.integers(0, npix, size=nt)
    weights = None
    if ncomp == 3:
        phi = rng.uniform(0.0, np.pi, size=nt)
        weights = np.stack([np.cos(2 * phi), np.sin(2 * phi)], axis=1)
    npsd = draw(st.integers(1, 2))
    psds = [(draw(st.floats(0.5, 2.0)), 0.0 if white else draw(st.floats(0.0, 2.0)), draw(st.floats(1.0, 2.0)))
            for _ in range(npsd)]
    # lambda <= L/2, where every row of a 1/f PSD with alpha <= 2 is positive definite;
    # beyond, the periodic row wraps and the symbol check rejects it (from ~0.84 L on)
    lam = draw(st.integers(0, min(lengths) // 2))
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    ipsd = rng.integers(0, npsd, size=len(lengths))
    pr = Problem(pix, npix, weights, offsets, ipsd, psds, 100.0, lam, ncomp)
    assume(pr.n > 0)
    return pr, rng


@SETTINGS
@given(problems())
def test_operators_match_their_dense_forms(arg):
    pr, rng = arg
    x = rng.standard_normal(pr.n)
    y = rng.standard_normal(pr.nt)
    Pd = pr.dense_P()
    Nd = toeplitz.dense_ninv(pr.offsets, pr.interval_psd, pr.rows)
    # P and P^T are adjoint and equal their dense matrices
    assert abs(y @ pr.P(x) - pr.PT(y) @ x) <= 1e-12 * (np.abs(y).sum() * np.abs(x).max() * 3 + 1)
    np.testing.assert_allclose(pr.P(x), Pd @ x, rtol=1e-13, atol=1e-13)
    # the banded N^-1 is symmetric and equals its dense block-diagonal Toeplitz form
    assert np.array_equal(Nd, Nd.T)
    np.testing.assert_allclose(pr.Ninv(y), Nd @ y, rtol=1e-12, atol=1e-12 * np.abs(Nd).sum(axis=1).max())
    # A x = P^T N^-1 P x by both Toeplitz routes, symmetric positive definite
    A = Pd.T @ Nd @ Pd
    scale = np.abs(A).sum(axis=1).max() * np.abs(x).max()
    np.testing.assert_allclose(pr.A(x), A @ x, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(pr.A(x, route="fft"), A @ x, rtol=0, atol=1e-9 * scale)
    v = rng.standard_normal(pr.n)
    assert v @ pr.A(v) > 0
    assert abs(v @ pr.A(x) - x @ pr.A(v)) <= 1e-12 * scale * np.abs(v).sum()


@SETTINGS
@given(problems(white=True))
def test_white_noise_gls_is_the_binned_map(arg):
    pr, rng = arg
    d = rng.standard_normal(pr.nt)
    m = dense_solve(pr.dense_A(), pr.rhs(d))
    # brute force: per observed pixel, sum over its samples of w w^T / sigma_t^2 m = w d / sigma_t^2
    sig2 = np.empty(pr.nt)
    for i in range(pr.offsets.size - 1):
        sig2[pr.offsets[i]:pr.offsets[i + 1]] = pr.psds[pr.interval_psd[i]][0] ** 2
    ref = np.empty(pr.n)
    for q in range(pr.npix_obs):
        ts = np.flatnonzero(pr.pix_c == q)
        if pr.ncomp == 1:
            W = np.ones((ts.size, 1))
        else:
            W = np.stack([np.ones(ts.size), pr.weights[ts, 0], pr.weights[ts, 1]], axis=1)
        Bq = (W / sig2[ts, None]).T @ W
        ref[q * pr.ncomp:(q + 1) * pr.ncomp] = np.linalg.solve(Bq, (W / sig2[ts, None]).T @ d[ts])
    np.testing.assert_allclose(m, ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())
    # M_BD is A^-1 here: PCG converges in one step
    res = pcg(pr.A, precond.BlockJacobi(pr).apply, pr.rhs(d), 1e-8, 10)
    assert res.converged and res.iters == 1


@SETTINGS
@given(problems())
def test_pcg_reaches_the_dense_solution(arg):
    pr, rng = arg
    b = pr.rhs(rng.standard_normal(pr.nt))
    assume(np.linalg.norm(b) > 0)
    res = pcg(pr.A, precond.BlockJacobi(pr).apply, b, 1e-11, 50 * pr.n + 50)
    assert res.converged
    assert np.linalg.norm(b - pr.A(res.x)) <= 1e-9 * np.linalg.norm(b)
    assert res.rel_hist[0] == 1.0 and res.rel_hist[-1] <= 1e-11
    A = pr.dense_A()
    m = dense_solve(A, b)
    # forward error within the condition number times the residual
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(res.x - m) <= 1e-8 * kappa * np.linalg.norm(m) + 1e-300


@SETTINGS
@given(problems(), st.integers(1, 4))
def test_two_level_identities_for_any_coarse_basis(arg, k):
    pr, rng = arg
    assume(pr.n > k)
    bd = precond.BlockJacobi(pr)
    Z = rng.standard_normal((pr.n, k))
    tl = precond.TwoLevel(pr, bd, Z)
    A = pr.dense_A()
    assume(np.linalg.cond(Z.T @ A @ Z) < 1e10)
    AZ = A @ Z
    RAZ = np.stack([tl.deflate(AZ[:, j]) for j in range(k)], axis=1)
    assert np.linalg.norm(RAZ) <= 1e-8 * np.linalg.norm(AZ)
    MAZ = np.stack([tl.apply(AZ[:, j]) for j in range(k)], axis=1)
    assert np.linalg.norm(MAZ - Z) <= 1e-8 * np.linalg.norm(Z)


@st.composite
def one_over_f_problems(draw):
    """problems() with f_knee > 0 for every PSD (the PSD derivatives need it)."""
    pr, rng = draw(problems())
    psds = [(s, max(fk, 0.1), a) for (s, fk, a) in pr.psds]
    pr = Problem(pr.pix, pr.npix_sky, pr.weights, pr.offsets, pr.interval_psd, psds, pr.fsamp, pr.lam, pr.ncomp)
    assume(pr.n > 0)
    return pr, rng


@SETTINGS
@given(one_over_f_problems())
def test_data_gradient_is_exact_for_the_linear_map(arg):
    """m(d) = A^-1 P^T N^-1 d is linear in d, so for L = g^T m the adjoint gradient
    dL/dd = N^-1 P A^-1 g (A and N^-1 symmetric) gives g^T (m(d + e) - m(d)) exactly."""
    pr, rng = arg
    A = pr.dense_A()
    d, e = rng.standard_normal(pr.nt), rng.standard_normal(pr.nt)
    m0 = dense_solve(A, pr.rhs(d))
    m1 = dense_solve(A, pr.rhs(d + e))
    g = rng.standard_normal(pr.n)
    from oracle import adjoint
    dLdd, _ = adjoint.gradients(pr, d, m0, g, dense=True)
    lhs, rhs = g @ (m1 - m0), dLdd @ e
    assert abs(lhs - rhs) <= 1e-7 * np.linalg.cond(A) * 1e-3 * (np.abs(g) @ np.abs(m1 - m0) + abs(rhs)) + 1e-12


@settings(max_examples=25, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(one_over_f_problems())
def test_psd_gradient_matches_central_differences(arg):
    """dL/d(sigma, f_knee, alpha) of L = 1/2 ||m - m_ref||^2 (the adjoint of R14) against
    central differences of problems rebuilt with the perturbed PSD."""
    pr, rng = arg
    d = rng.standard_normal(pr.nt)
    mref = rng.standard_normal(pr.n)

    def loss(psds):
        q = Problem(pr.pix, pr.npix_sky, pr.weights, pr.offsets, pr.interval_psd, psds, pr.fsamp, pr.lam, pr.ncomp)
        m = dense_solve(q.dense_A(), q.rhs(d))
        return 0.5 * np.sum((m - mref) ** 2), m

    L0, m = loss(pr.psds)
    from oracle import adjoint
    _, G = adjoint.gradients(pr, d, m, m - mref, dense=True)
    kappa = np.linalg.cond(pr.dense_A())
    th = np.array(pr.psds, dtype=np.float64)
    for p in range(th.shape[0]):
        for c in range(3):
            h = 1e-5 * th[p, c]
            tp, tm = th.copy(), th.copy()
            tp[p, c] += h
            tm[p, c] -= h
            fd = (loss([tuple(v) for v in tp])[0] - loss([tuple(v) for v in tm])[0]) / (2 * h)
            # the difference quotient's own rounding floor: kappa eps L / h
            floor = 10 * kappa * np.finfo(float).eps * L0 / h
            assert fd == pytest.approx(G[p, c], rel=1e-4, abs=1e-6 * np.abs(G).max() + floor), (p, c)


@SETTINGS
@given(problems(), st.integers(1, 6))
def test_apriori_rows_sum_to_one(arg, r):
    """Z_S of Eq. 16-17: each observed pixel's T row is its hit fractions over the
    intervals, so it sums to 1; Q/U rows are zero; merging intervals keeps both."""
    pr, _ = arg
    from oracle.precond import deflation_apriori, deflation_apriori_merged
    Z = deflation_apriori(pr)
    K = pr.offsets.size - 1
    nc = pr.ncomp
    np.testing.assert_allclose(Z[0::nc].sum(axis=1), 1.0, rtol=0, atol=1e-14)
    if nc == 3:
        assert np.all(Z[1::3] == 0.0) and np.all(Z[2::3] == 0.0)
    Zm = deflation_apriori_merged(pr, min(r, K))
    np.testing.assert_allclose(Zm[0::nc].sum(axis=1), 1.0, rtol=0, atol=1e-14)
    # brute force: the fraction of pixel q's hits inside interval j
    j = 0
    a, b = int(pr.offsets[j]), int(pr.offsets[j + 1])
    for q in range(min(pr.npix_obs, 5)):
        frac = np.sum(pr.pix_c[a:b] == q) / pr.hits[q]
        assert Z[q * nc, j] == pytest.approx(frac, abs=1e-15)


@SETTINGS
@given(problems())
def test_lanczos_ritz_values_lie_in_the_spectrum(arg):
    """Ritz values of the CG-Lanczos tridiagonal (Sec. 3.3.2) are Rayleigh quotients of
    M_BD A, so they lie in its spectrum's hull [lambda_min, lambda_max]."""
    pr, rng = arg
    bd = precond.BlockJacobi(pr)
    A = pr.dense_A()
    ev = np.sort(np.linalg.eigvals(bd.dense() @ A).real)
    res = pcg(pr.A, bd.apply, rng.standard_normal(pr.n), 1e-10, pr.n)
    assume(len(res.alphas) >= 1)
    T = precond.lanczos_tridiagonal(res.alphas, res.betas[: len(res.alphas) - 1])
    th = np.linalg.eigvalsh(T)
    slack = 1e-8 * ev[-1]
    assert th.min() >= ev[0] - slack and th.max() <= ev[-1] + slack


@SETTINGS
@given(problems(), st.integers(1, 12))
def test_arnoldi_relation(arg, m):
    """Algorithm 1 gives B W_j = W_{j+1} Hbar_j (Eq. A.3), B = M_BD A, with W_j orthonormal;
    w_{j+1} is a unit vector orthogonal to W_j unless h_{j+1,j} is at rounding level (the
    Krylov space is exhausted: then it is noise, and the relation holds through the
    negligible h_{j+1,j})."""
    pr, rng = arg
    bd = precond.BlockJacobi(pr)
    B = lambda x: bd.apply(pr.A(x))
    W, H, beta, _ = precond.arnoldi(B, bd.apply(rng.standard_normal(pr.n)), min(m, pr.n))
    j = H.shape[1]
    assume(j >= 1)
    BW = np.stack([B(W[:, i]) for i in range(j)], axis=1)
    np.testing.assert_allclose(BW, W @ H, rtol=0, atol=1e-10 * np.abs(BW).max())
    np.testing.assert_allclose(W[:, :j].T @ W[:, :j], np.eye(j), atol=1e-10)
    if H[j, j - 1] > 1e-8 * np.abs(H).max():
        np.testing.assert_allclose(W.T @ W, np.eye(j + 1), atol=1e-10)
