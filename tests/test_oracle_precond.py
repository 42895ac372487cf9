"""Pins of the oracle's preconditioners and Ritz construction (Sec. 3, App. A-C) -- CPU."""
import numpy as np
import pytest

from oracle import precond
from paper_1408_3048_gb300 import synth
from oracle.pcg import pcg
from problems import oracle_problem, tiny_scan


@pytest.fixture(scope="module", params=[1, 3])
def prob(request):
    ncomp = request.param
    scan = tiny_scan(ncomp=ncomp, psds=((1.0, 3.0, 1.8), (1.2, 1.5, 1.2)), lam=10)
    return oracle_problem(scan)


def test_bd_equals_dense_inverse(prob):
    bd = precond.BlockJacobi(prob)
    P = prob.dense_P()
    D = np.diag(prob.ninv_diag())
    ref = np.linalg.inv(P.T @ D @ P)
    np.testing.assert_allclose(bd.dense(), ref, rtol=1e-9, atol=1e-9)


def _z_from_eigvecs(prob, bd, k):
    A = prob.dense_A()
    Minv = np.linalg.inv(bd.dense())
    # smallest generalised eigenvectors of M_BD A  (A v = theta M_BD^-1 v)
    import scipy.linalg
    th, V = scipy.linalg.eigh(A, Minv)
    return A, th, V[:, :k]


def test_deflation_and_two_level_identities(prob):
    bd = precond.BlockJacobi(prob)
    rng = np.random.default_rng(0)
    Z = rng.standard_normal((prob.n, 4))
    tl = precond.TwoLevel(prob, bd, Z)
    A = prob.dense_A()
    AZ = A @ Z
    # E = Z^T A Z is SPD (Cholesky succeeds)
    np.linalg.cholesky(0.5 * (tl.E + tl.E.T))
    # T4: R A Z = 0 (Eq. 11)
    RAZ = np.stack([tl.deflate(AZ[:, j]) for j in range(4)], axis=1)
    assert np.linalg.norm(RAZ) <= 1e-10 * np.linalg.norm(AZ)
    # T5: M_2lvl A Z = Z (Eq. 13)
    MAZ = np.stack([tl.apply(AZ[:, j]) for j in range(4)], axis=1)
    assert np.linalg.norm(MAZ - Z) <= 1e-10 * np.linalg.norm(Z)
    # T6: M_2lvl A Y = M_BD A Y when Z^T A Y = 0 (Eq. 14)
    Y = rng.standard_normal((prob.n, 3))
    Y = Y - Z @ np.linalg.solve(Z.T @ A @ Z, Z.T @ A @ Y)      # A-orthogonalise against Z
    assert np.linalg.norm(Z.T @ A @ Y) <= 1e-10 * np.linalg.norm(A @ Y)
    AY = A @ Y
    lhs = np.stack([tl.apply(AY[:, j]) for j in range(3)], axis=1)
    rhs = np.stack([bd.apply(AY[:, j]) for j in range(3)], axis=1)
    assert np.linalg.norm(lhs - rhs) <= 1e-9 * np.linalg.norm(rhs)


def test_two_level_maps_deflated_eigenvalues_to_one(prob):
    bd = precond.BlockJacobi(prob)
    A, th, Z = _z_from_eigvecs(prob, bd, 5)
    tl = precond.TwoLevel(prob, bd, Z)
    M2 = np.stack([tl.apply(e) for e in np.eye(prob.n)], axis=1)
    ev = np.sort(np.linalg.eigvals(M2 @ A).real)
    evbd = np.sort(th)
    # the 5 smallest eigenvalues of M_BD A are replaced by 1, the rest are unchanged
    expect = np.sort(np.concatenate([np.ones(5), evbd[5:]]))
    np.testing.assert_allclose(ev, expect, rtol=1e-7, atol=1e-8)


def test_lanczos_ritz_values_converge_to_the_spectrum(prob):
    # T9 / Eq. 22-23: after CG has converged, the smallest Ritz value of T_m equals the
    # smallest eigenvalue of M_BD A, every Ritz value lies inside the spectrum, and the
    # Ritz vector of the smallest one is an eigenvector (small residual).
    bd = precond.BlockJacobi(prob)
    A, th, V = _z_from_eigvecs(prob, bd, 1)
    b = np.random.default_rng(1).standard_normal(prob.n)
    res = pcg(prob.A, bd.apply, b, 1e-14, 5 * prob.n, record=True)
    T = precond.lanczos_tridiagonal(res.alphas, res.betas)
    rv = np.linalg.eigvalsh(T)
    # (CG stops after ~20 steps on a 90-dim, well clustered spectrum: the smallest
    # Ritz value is converged to a few 1e-6, a wrong T_m would be off by O(1))
    assert rv[0] == pytest.approx(th[0], rel=1e-4)
    assert rv[0] >= th[0] * (1 - 1e-10) and rv[-1] <= th[-1] * (1 + 1e-10)
    Z, theta = precond.ritz_coarse_space(res.alphas, res.betas, res.zs, res.rzs, 3)
    assert np.allclose(Z.T @ Z, np.eye(Z.shape[1]), atol=1e-10)
    np.testing.assert_allclose(theta, rv[:3], rtol=1e-13)
    v = V[:, 0] / np.linalg.norm(V[:, 0])
    assert np.linalg.norm(v - Z @ (Z.T @ v)) < 0.05


def test_lanczos_vectors_are_minv_orthonormal(prob):
    bd = precond.BlockJacobi(prob)
    b = np.random.default_rng(2).standard_normal(prob.n)
    res = pcg(prob.A, bd.apply, b, 1e-10, 20, record=True)
    m = len(res.alphas)
    V = np.stack([((-1.0) ** j) * res.zs[j] / np.sqrt(res.rzs[j]) for j in range(m)], axis=1)
    Minv = np.linalg.inv(bd.dense())
    G = V.T @ Minv @ V
    assert np.abs(G - np.eye(m)).max() < 1e-8
    # M A V = V T + (rank-one remainder in the last column only)
    A = prob.dense_A()
    T = precond.lanczos_tridiagonal(res.alphas, res.betas)
    Rm = bd.dense() @ A @ V - V @ T
    assert np.linalg.norm(Rm[:, :-1]) <= 1e-8 * np.linalg.norm(V)


def test_arnoldi_relation_and_ritz_residuals(prob):
    # Algorithm 1 / Eq. A.2: B W_m = W_{m+1} Hbar_m with orthonormal W; Eq. A.4: the
    # residual of a Ritz pair equals |h_{m+1,m} e_m^T v_i|
    bd = precond.BlockJacobi(prob)
    B = lambda x: bd.apply(prob.A(x))
    b = prob.rhs(np.random.default_rng(8).standard_normal(prob.nt))
    m = min(12, prob.n - 1)
    W, H, beta, rel = precond.arnoldi(B, bd.apply(b), m)
    j = H.shape[1]
    assert j == m and beta > 0
    np.testing.assert_allclose(W.T @ W, np.eye(j + 1), atol=1e-10)
    BW = np.stack([B(W[:, c]) for c in range(j)], axis=1)
    np.testing.assert_allclose(BW, W @ H, atol=1e-10 * np.abs(BW).max())
    lam, V = np.linalg.eig(H[:j, :j])
    for i in range(j):
        y = W[:, :j] @ V[:, i]
        res = np.linalg.norm(B(y.real) + 1j * B(y.imag) - lam[i] * y)
        assert res == pytest.approx(abs(H[j, j - 1] * V[j - 1, i]), rel=1e-6, abs=1e-10)
    # GMRES stopping: the residual estimate is the true left-preconditioned residual
    W2, H2, beta2, rel2 = precond.arnoldi(B, bd.apply(b), prob.n, tol=1e-8)
    j2 = H2.shape[1]
    e1 = np.zeros(j2 + 1)
    e1[0] = beta2
    x = W2[:, :j2] @ np.linalg.lstsq(H2, e1, rcond=None)[0]
    assert rel2 <= 1e-8
    assert np.linalg.norm(bd.apply(b) - B(x)) / beta2 == pytest.approx(rel2, rel=1e-3, abs=1e-12)
    # a full-dimension run reproduces the spectrum of M_BD A: the selected pairs are
    # the smallest eigenpairs, orthonormalised
    W3, H3, _, _ = precond.arnoldi(B, bd.apply(b), prob.n)
    Z, vals = precond.arnoldi_coarse_space(W3, H3, 3, eps_tol=np.inf)
    lam_true = np.sort(np.linalg.eigvals(bd.dense() @ prob.dense_A()).real)
    np.testing.assert_allclose(np.sort(vals)[:3], lam_true[:3], rtol=1e-6)
    np.testing.assert_allclose(Z.T @ Z, np.eye(Z.shape[1]), atol=1e-10)
    # eps_tol keeps only the pairs below the threshold
    _, v2 = precond.arnoldi_coarse_space(W3, H3, 64, eps_tol=0.5 * (lam_true[1] + lam_true[2]))
    assert len(v2) == 2


def test_adef2_spectrum_and_start(prob):
    # App. B: M_2lvl A and M_2lvl^(alt) A have the same spectrum; from x0 = Z E^-1 Z^T b
    # every A-DEF2 residual stays orthogonal to Z, and PCG reaches the dense solution
    b = prob.rhs(np.random.default_rng(4).standard_normal(prob.nt))
    bd = precond.BlockJacobi(prob)
    res = pcg(prob.A, bd.apply, b, 1e-10, 500, record=True)
    Z, _ = precond.ritz_coarse_space(res.alphas, res.betas, res.zs, res.rzs, 3)
    tl = precond.TwoLevel(prob, bd, Z)
    A = prob.dense_A()
    I = np.eye(prob.n)
    M1 = np.stack([tl.apply(I[:, j]) for j in range(prob.n)], axis=1)
    M2 = np.stack([tl.apply_adef2(I[:, j]) for j in range(prob.n)], axis=1)
    e1 = np.sort(np.linalg.eigvals(M1 @ A).real)
    e2 = np.sort(np.linalg.eigvals(M2 @ A).real)
    np.testing.assert_allclose(e2, e1, rtol=1e-7, atol=1e-7 * e1.max())
    x0 = tl.adef2_start(b)
    r0 = b - prob.A(x0)
    assert np.linalg.norm(Z.T @ r0) <= 1e-10 * np.linalg.norm(b)
    out = pcg(prob.A, tl.apply_adef2, b, 1e-10, 500, x0=x0)
    assert out.converged
    np.testing.assert_allclose(out.x, np.linalg.solve(A, b), rtol=1e-7, atol=1e-7 * np.abs(out.x).max())
    # the deflated directions stay deflated along the way
    r = b - prob.A(out.x)
    assert np.linalg.norm(Z.T @ r) <= 1e-8 * np.linalg.norm(b)


def test_ritz_threshold_selection(prob):
    # eps_tol keeps exactly the Ritz pairs below the threshold (at most k), which are the
    # leading columns of the k-smallest selection
    b = prob.rhs(np.random.default_rng(3).standard_normal(prob.nt))
    bd = precond.BlockJacobi(prob)
    res = pcg(prob.A, bd.apply, b, 1e-10, 500, record=True)
    Zall, th = precond.ritz_coarse_space(res.alphas, res.betas, res.zs, res.rzs, 64)
    eps = 0.5 * (th[2] + th[3])
    Ze, the = precond.ritz_coarse_space(res.alphas, res.betas, res.zs, res.rzs, 64, eps_tol=eps)
    assert len(the) == 3 and np.all(the < eps)
    np.testing.assert_allclose(the, th[:3], rtol=0, atol=0)
    np.testing.assert_allclose(np.abs(Ze.T @ Zall[:, :3]), np.eye(3), atol=1e-8)
    assert len(precond.ritz_coarse_space(res.alphas, res.betas, res.zs, res.rzs, 2, eps_tol=eps)[1]) == 2
    with pytest.raises(ValueError):
        precond.ritz_coarse_space(res.alphas, res.betas, res.zs, res.rzs, 64, eps_tol=0.5 * th[0])


def test_apriori_rows_sum_to_one(prob):
    Z = precond.deflation_apriori(prob)
    nc = prob.ncomp
    np.testing.assert_allclose(Z[0::nc].sum(axis=1), 1.0, rtol=0, atol=1e-15)
    if nc == 3:
        assert np.all(Z[1::3] == 0) and np.all(Z[2::3] == 0)


def test_apriori_merged_brute_force(prob):
    # merged Z_S against a direct count over samples: column g = the fraction of each
    # observed pixel's kept samples that fall in group g's intervals (Sec. 3.3.1)
    K = prob.offsets.size - 1
    nc = prob.ncomp
    for r in sorted({1, 2, max(1, K // 2), K}):
        Z = precond.deflation_apriori_merged(prob, r)
        assert Z.shape == (prob.n, r)
        cnt = np.zeros((prob.npix_obs, r))
        for i in range(K):
            g = i * r // K
            for t in range(int(prob.offsets[i]), int(prob.offsets[i + 1])):
                q = prob.pix_c[t]
                if q >= 0:
                    cnt[q, g] += 1.0
        np.testing.assert_array_equal(Z[0::nc], cnt / cnt.sum(axis=1, keepdims=True))
        if nc == 3:
            assert np.all(Z[1::3] == 0) and np.all(Z[2::3] == 0)
        np.testing.assert_allclose(Z[0::nc].sum(axis=1), 1.0, rtol=0, atol=1e-15)
    # r = K is the unmerged Z_S; r = 1 is the temperature vector of ones (Eq. 15)
    np.testing.assert_array_equal(precond.deflation_apriori_merged(prob, K), precond.deflation_apriori(prob))
    ones = np.zeros(prob.n)
    ones[0::nc] = 1.0
    np.testing.assert_allclose(precond.deflation_apriori_merged(prob, 1)[:, 0], ones, rtol=0, atol=1e-15)


def test_apriori_dependent_columns_dropped(prob):
    # every interval of the tiny raster sees each pixel equally often: all columns of Z_S
    # are equal, so one column survives and it spans the temperature ones vector
    Z = precond.deflation_apriori(prob)
    Zk, kept = precond.independent_columns(Z)
    assert kept == [0]
    Z2 = np.column_stack([Z[:, 0], 2.0 * Z[:, 0] + 1e-3 * np.arange(prob.n), Z[:, 0] + Z[:, 0]])
    assert precond.independent_columns(Z2)[1] == [0, 1]


@pytest.mark.parametrize("ncomp", [1, 3])
def test_apriori_two_level_invariants(ncomp):
    # uneven intervals cut the sweeps mid-way, so the columns of Z_S differ; M_2lvl A Z = Z
    # holds for the a priori space (the coarse correction is exact on range Z)
    scan = synth.raster_scan(16, 16, 2, 6000, ncomp, 3, 60, [(1.0, 1.0, 1.0), (0.8, 1.5, 1.5)],
                             det_psd=[0, 1], uneven=(1000, 3000), seed=7)
    prob = oracle_problem(scan)
    K = prob.offsets.size - 1
    Z, kept = precond.independent_columns(precond.deflation_apriori_merged(prob, min(K, 4)))
    assert len(kept) >= 2
    bd = precond.BlockJacobi(prob)
    tl = precond.TwoLevel(prob, bd, Z)
    for j in range(Z.shape[1]):
        np.testing.assert_allclose(tl.apply(prob.A(Z[:, j])), Z[:, j], rtol=0, atol=1e-9 * np.abs(Z[:, j]).max())


def test_ones_near_nullspace_with_one_over_f():
    # Eq. 15: A 1_p is small when the noise has a 1/f excess (N^-1 1_t ~ 0).
    s1 = tiny_scan(ncomp=1, psds=((1.0, 20.0, 1.0),), lam=100, nper=2000)
    s0 = tiny_scan(ncomp=1, psds=((1.0, 0.0, 1.0),), lam=100, nper=2000)
    r = []
    for s in (s1, s0):
        pr = oracle_problem(s)
        one = np.ones(pr.n)
        A = pr.dense_A()
        r.append(np.linalg.norm(A @ one) / (np.linalg.norm(A, 2) * np.linalg.norm(one)))
    assert r[0] < 0.1 * r[1]


def test_cg_iterations_obey_the_condition_number_bound(prob):
    # Eq. 9 for PCG: ||x - x_j||_A <= 2 ||x||_A ((sqrt k - 1)/(sqrt k + 1))^j with k the
    # condition number of M_BD A.
    bd = precond.BlockJacobi(prob)
    A, th, _ = _z_from_eigvecs(prob, bd, 1)
    kappa = th[-1] / th[0]
    b = np.random.default_rng(3).standard_normal(prob.n)
    xs = np.linalg.solve(A, b)
    rate = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    for j in (2, 5, 10):
        res = pcg(prob.A, bd.apply, b, 0.0, j)
        e = xs - res.x
        assert np.sqrt(e @ A @ e) <= 2 * np.sqrt(xs @ A @ xs) * rate ** j * (1 + 1e-8)


def test_two_level_needs_fewer_iterations():
    # T13 (Sec. 5.1): with strong 1/f noise the a posteriori two-level preconditioner
    # converges in fewer iterations than M_BD.
    scan = tiny_scan(ncomp=3, W=8, H=8, ndet=2, nper=1200, K_per_det=2, lam=40,
                     psds=((1.0, 5.0, 2.0), (1.0, 4.0, 1.5)))
    pr = oracle_problem(scan)
    bd = precond.BlockJacobi(pr)
    b = np.random.default_rng(9).standard_normal(pr.n)
    r0 = pcg(pr.A, bd.apply, b, 1e-6, 2000, record=True)
    Z, _ = precond.ritz_coarse_space(r0.alphas, r0.betas, r0.zs, r0.rzs, 8)
    tl = precond.TwoLevel(pr, bd, Z)
    b2 = np.random.default_rng(10).standard_normal(pr.n)
    it_bd = pcg(pr.A, bd.apply, b2, 1e-6, 2000).iters
    it_2l = pcg(pr.A, tl.apply, b2, 1e-6, 2000).iters
    assert it_2l < it_bd


def test_dependence_rule_pins():
    # reading R16: a column is dependent when its part orthogonal to the earlier kept
    # columns is below 1e-10 of the largest column norm.  Exact duplicates, scaled copies,
    # combinations and zero columns go; a near-duplicate 1e-9 away stays, one 1e-11 away
    # goes (both relative to the column norm of ~8)
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((64, 9))
    Y[:, 2] = Y[:, 0]
    Y[:, 3] = -3.0 * Y[:, 1]
    Y[:, 4] = Y[:, 0] - 2.0 * Y[:, 1]
    Y[:, 5] = 0.0
    u = rng.standard_normal(64)
    u /= np.linalg.norm(u)
    Y[:, 6] = Y[:, 1] + 1e-9 * np.linalg.norm(Y[:, 1]) * u
    Y[:, 7] = Y[:, 0] + 1e-11 * np.linalg.norm(Y[:, 0]) * u
    _, kept = precond.independent_columns(Y)
    assert kept == [0, 1, 6, 8]
    Q, kept2 = precond.orthonormal_basis(Y)
    assert kept2 == kept
    np.testing.assert_allclose(Q.T @ Q, np.eye(4), atol=1e-12)
    Yk = Y[:, kept]
    assert np.linalg.norm(Yk - Q @ (Q.T @ Yk)) <= 1e-12 * np.linalg.norm(Yk)


@pytest.mark.parametrize("seed", range(4))
def test_dependence_rule_matches_the_numerical_rank(seed):
    # independent of the Gram-Schmidt route: for a matrix of exact rank r with the other
    # columns random combinations of earlier ones, the kept count equals the number of
    # singular values above 1e-10 of the largest column norm, the first r columns are kept
    # and their span contains every column
    rng = np.random.default_rng(seed)
    n, r, k = 80, 5, 12
    B = rng.standard_normal((n, r))
    C = np.zeros((r, k))
    C[:, :r] = np.eye(r)
    C[:, r:] = rng.standard_normal((r, k - r))
    Y = B @ C
    Y[:, r:] += 1e-14 * rng.standard_normal((n, k - r))
    _, kept = precond.independent_columns(Y)
    s = np.linalg.svd(Y, compute_uv=False)
    assert len(kept) == int(np.sum(s > 1e-10 * np.linalg.norm(Y, axis=0).max())) == r
    assert kept == list(range(r))
    Q, _ = precond.orthonormal_basis(Y)
    assert np.linalg.norm(Y - Q @ (Q.T @ Y)) <= 1e-12 * np.linalg.norm(Y)
