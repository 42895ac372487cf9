"""Parity of the CUDA path (through the C-ABI) against the FP64 oracle -- needs a GPU.

Tolerances: integer outputs (observed pixels, hits) bit-exact; FP64 operators to
1e-12 relative L2 (the FFT Toeplitz product and the oracle's direct sum differ only by
rounding, ~log2(B) * 1e-16 relative to the band norm); FP32 operators to 2e-5 relative
L2 (FP32 FFT rounding, ~log2(B) * 6e-8, times the dynamic range of the 1/f band); maps
to 1e-6 relative L2 with PCG iteration counts within 2 of the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import precond as oprec
from oracle.pcg import pcg
from paper_1408_3048_gb300 import mm, synth
from problems import oracle_problem, tiny_scan

pytestmark = pytest.mark.gpu


def _plan(scan, **kw):
    return mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.lam, scan.fsamp, **kw)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def _converged(pr, b, tol=1e-12):
    """The oracle's converged map m* of A m = b (block-Jacobi PCG to tol) and the error
    amplification kappa_b = ||M_BD|| ||b|| / (theta_1 ||m*||), theta_1 the smallest Ritz
    value of M_BD A from that run's Lanczos tridiagonal: a map with true relative residual
    rho lies within kappa_b (rho + tol) ||m*|| of m* (||A^-1|| <= ||M_BD|| / lambda_min)."""
    bd = oprec.BlockJacobi(pr)
    ref = pcg(pr.A, bd.apply, b, tol, 20000)
    k = len(ref.alphas)
    th1 = np.linalg.eigvalsh(oprec.lanczos_tridiagonal(ref.alphas, ref.betas[: k - 1]))[0]
    mbd = np.linalg.eigvalsh(bd.inv).max()
    return ref.x, mbd * np.linalg.norm(b) / (th1 * np.linalg.norm(ref.x))


SCANS = {
    "T_tiny": lambda: tiny_scan(ncomp=1),
    "P_tiny": lambda: tiny_scan(ncomp=3),
    "T_ragged": lambda: synth.raster_scan(24, 20, 3, 20000, 1, 3, 300, [(1.0, 1.0, 1.0), (0.7, 2.0, 1.7), (1.3, 0.3, 1.2)],
                                          det_psd=[0, 1, 2], uneven=(2000, 12000), seed=4),
    "P_ragged": lambda: synth.raster_scan(24, 24, 4, 24000, 3, 4, 500, [(1.0, 1.0, 1.0), (0.8, 1.5, 1.5)],
                                          det_psd=[0, 1, 0, 1], uneven=(3000, 9000), seed=5),
    "c2_small": lambda: synth.config(2, scale=64),
}


@pytest.fixture(scope="module", params=list(SCANS))
def case(request):
    scan = SCANS[request.param]()
    pr = oracle_problem(scan)
    plan = _plan(scan)
    yield request.param, scan, pr, plan
    plan.close()


def test_pixels_and_hits_bit_exact(case):
    _, scan, pr, plan = case
    o2s, hits = plan.pixels()
    assert plan.npix_obs == pr.npix_obs and plan.n == pr.n
    assert np.array_equal(o2s, pr.obs2sky)
    assert np.array_equal(hits, pr.hits)


def test_rows_match(case):
    _, scan, pr, plan = case
    for p in range(plan.npsd):
        r = plan.row(p)
        assert np.abs(r - pr.rows[p]).max() <= 1e-13 * np.abs(pr.rows[p]).max()


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32])
def test_gather_ninv_scatter(case, prec):
    _, scan, pr, plan = case
    rng = np.random.default_rng(1)
    dt = torch.float64 if prec == mm.MM_FP64 else torch.float32
    tol = 1e-12 if prec == mm.MM_FP64 else 2e-5
    x = rng.standard_normal(pr.n)
    xc = _cuda(x, dt)
    y = plan.gather(xc, prec).cpu().numpy()
    assert _rel(y, pr.P(xc.double().cpu().numpy())) <= (1e-15 if prec == mm.MM_FP64 else 1e-7)
    t = rng.standard_normal(pr.nt)
    tc = _cuda(t, dt)
    z = plan.apply_ninv(tc, prec).cpu().numpy()
    zr = pr.Ninv(tc.double().cpu().numpy())
    assert _rel(z, zr) <= tol
    # element-wise: every output within tol of the band norm scale
    scale = np.abs(pr.rows[0]).sum() * np.abs(t).max()
    assert np.abs(z - zr).max() <= tol * scale * 10
    w = plan.scatter(tc, prec).cpu().numpy()
    assert _rel(w, pr.PT(tc.double().cpu().numpy())) <= (1e-14 if prec == mm.MM_FP64 else 1e-6)


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32])
def test_apply_A(case, prec):
    _, scan, pr, plan = case
    dt = torch.float64 if prec == mm.MM_FP64 else torch.float32
    x = np.random.default_rng(2).standard_normal(pr.n)
    xc = _cuda(x, dt)
    y = plan.apply_A(xc, prec).cpu().numpy()
    assert _rel(y, pr.A(xc.double().cpu().numpy())) <= (1e-12 if prec == mm.MM_FP64 else 3e-5)


def test_A_symmetric_deterministic(case):
    _, scan, pr, plan = case
    rng = np.random.default_rng(3)
    x, y = _cuda(rng.standard_normal(pr.n)), _cuda(rng.standard_normal(pr.n))
    Ax1 = plan.apply_A(x)
    Ax2 = plan.apply_A(x)
    assert torch.equal(Ax1, Ax2)                     # bit-reproducible (no atomics)
    Ay = plan.apply_A(y)
    a, b = float(y @ Ax1), float(x @ Ay)
    assert abs(a - b) <= 1e-12 * float(torch.linalg.norm(Ax1) * torch.linalg.norm(y))
    assert float(x @ Ax1) > 0


def test_rhs_and_bd(case):
    _, scan, pr, plan = case
    rng = np.random.default_rng(4)
    d = rng.standard_normal(pr.nt)
    b = plan.rhs(_cuda(d)).cpu().numpy()
    assert _rel(b, pr.rhs(d)) <= 1e-12
    bd = oprec.BlockJacobi(pr)
    r = rng.standard_normal(pr.n)
    for prec, tol in ((mm.MM_FP64, 1e-12), (mm.MM_FP32, 1e-5)):
        dt = torch.float64 if prec == mm.MM_FP64 else torch.float32
        z = plan.precond(_cuda(r, dt), mm.MM_PREC_BD, prec).cpu().numpy()
        assert _rel(z, bd.apply(r)) <= tol


def _data(scan, real=0):
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 1000)
    n = synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp, 2000 + real)
    return synth.tod(scan, sky, n)


def test_solve_fp64_bd_matches_oracle(case):
    name, scan, pr, plan = case
    d = _data(scan)
    bd = oprec.BlockJacobi(pr)
    ref = pcg(pr.A, bd.apply, pr.rhs(d), 1e-6, 3000)
    m, st, status = plan.solve(_cuda(d), tol=1e-6, maxit=3000)
    assert status == mm.MM_OK and st["converged"] == 1
    assert abs(st["iters"] - ref.iters) <= 2, (st["iters"], ref.iters)
    assert _rel(m.cpu().numpy(), ref.x) <= 1e-6
    assert st["rel_resid"] <= 1.5e-6


@pytest.mark.parametrize("tol", [1e-6, 1e-8])
def test_solve_mixed_reaches_tolerance(case, tol):
    name, scan, pr, plan = case
    d = _data(scan)
    b = pr.rhs(d)
    mstar, kappa_b = _converged(pr, b)
    m, st, status = plan.solve(_cuda(d), tol=tol, maxit=5000, solver=mm.MM_SOLVE_MIXED)
    assert status == mm.MM_OK
    # true FP64 residual of the returned map, recomputed by the oracle
    mm_ = m.cpu().numpy()
    rel = np.linalg.norm(b - pr.A(mm_)) / np.linalg.norm(b)
    assert rel <= tol
    assert st["rel_resid"] <= tol
    # the reported residual (from P^T N^-1 (d - P m), scaled by the FP32 ||b||) is the
    # oracle's b - A m up to FP64 rounding of the residual and FP32 rounding of ||b||
    assert st["rel_resid"] == pytest.approx(rel, rel=1e-5, abs=1e-12)
    # the map against the oracle's converged one, within what its residual allows
    assert _rel(mm_, mstar) <= kappa_b * (tol + 1e-12)


@pytest.mark.parametrize("arith", [mm.MM_RESID_FP64, mm.MM_RESID_DF32])
def test_residual_from_data(case, arith):
    """r = P^T N^-1 (d - P x) (Eq. 5, 7) against the oracle's b - A x: the FP64 band
    product and the double-float one (pairs of FP32 numbers, ~48-bit significands) both
    within 1e-12 of ||b||, x = 0 giving b itself."""
    name, scan, pr, plan = case
    d = _data(scan)
    b = pr.rhs(d, route="fft")
    x = np.random.default_rng(8).standard_normal(pr.n)
    ref = b - pr.A(x, route="fft")
    r = plan.residual(_cuda(d), _cuda(x), arith).cpu().numpy()
    assert np.linalg.norm(r - ref) <= 1e-12 * np.linalg.norm(b)
    assert np.abs(r - ref).max() <= 1e-12 * np.abs(b).max()
    r0 = plan.residual(_cuda(d), _cuda(np.zeros(pr.n)), arith).cpu().numpy()
    assert np.linalg.norm(r0 - b) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("lanes", [32, 16, 8])
def test_scatter_pixel_tiles(lanes):
    # the scatter with 32, 16 or 8 lanes per observed pixel (one, two or four pixels per
    # warp) against the oracle's P^T, FP64 and FP32, and inside A x; the fused p^T q of the
    # PCG scatter through a solve
    scan = SCANS["P_ragged"]()
    pr = oracle_problem(scan)
    plan = _plan(scan, scatter_lanes=lanes)
    assert plan.scatter_config()[0] == lanes
    rng = np.random.default_rng(lanes)
    z = rng.standard_normal(pr.nt)
    ref = pr.PT(z)
    assert _rel(plan.scatter(_cuda(z)).cpu().numpy(), ref) <= 1e-12
    assert _rel(plan.scatter(_cuda(z, torch.float32), mm.MM_FP32).double().cpu().numpy(), ref) <= 2e-5
    x = rng.standard_normal(pr.n)
    assert _rel(plan.apply_A(_cuda(x)).cpu().numpy(), pr.A(x)) <= 1e-12
    d = _data(scan)
    m, st, status = plan.solve(_cuda(d), tol=1e-8, maxit=3000)
    ref_m = pcg(pr.A, oprec.BlockJacobi(pr).apply, pr.rhs(d), 1e-8, 3000)
    assert status == mm.MM_OK and abs(st["iters"] - ref_m.iters) <= 2
    assert _rel(m.cpu().numpy(), ref_m.x) <= 1e-6
    plan.close()


def test_fp32_scatter_weights_from_angles_and_pairs():
    # unit-norm weights: the FP32 scatter forms (cos, sin) from a stored angle; weights
    # of another norm (a polarisation efficiency of 0.9 here) keep the stored pairs.
    # Both against the oracle's P^T and A.
    for eff in (1.0, 0.9):
        scan = SCANS["P_ragged"]()
        scan.weights = np.asarray(scan.weights) * eff
        pr = oracle_problem(scan)
        plan = _plan(scan)
        rng = np.random.default_rng(23)
        z = rng.standard_normal(pr.nt)
        got = plan.scatter(_cuda(z, torch.float32), mm.MM_FP32).double().cpu().numpy()
        assert _rel(got, pr.PT(z)) <= 2e-5, eff
        # against the FP64 scatter of the same FP32-rounded values: the weights formed from
        # the angle (table-driven, ~2e-7) and the FP32 sums stay within 1e-6
        z32 = _cuda(z, torch.float32)
        ref64 = plan.scatter(z32.double(), mm.MM_FP64).cpu().numpy()
        assert _rel(got, ref64) <= 1e-6, eff
        x = rng.standard_normal(pr.n)
        ax = plan.apply_A(_cuda(x, torch.float32), mm.MM_FP32).double().cpu().numpy()
        assert _rel(ax, pr.A(x)) <= 3e-5, eff
        plan.close()


def test_scatter_pixel_tile_autotuned():
    scan = SCANS["c2_small"]()
    plan = _plan(scan, autotune=True)
    lanes, ms = plan.scatter_config()
    assert lanes in (32, 16, 8) and min(ms) > 0
    assert lanes == (32, 16, 8)[int(np.argmin(ms))]
    with pytest.raises(mm.MMError) as e:
        _plan(scan, scatter_lanes=12)
    assert e.value.status == mm.MM_ERR_ARG
    plan.close()


def test_residual_history(case):
    """||r_j|| / ||b|| per step (the Sec. 5.1 convergence measure) against the oracle's
    PCG on the same system: equal start, the stopping rule on the last two entries, and
    the oracle's values wherever the two runs take the same number of steps."""
    name, scan, pr, plan = case
    d = _data(scan)
    tol = 1e-6
    ref = pcg(pr.A, oprec.BlockJacobi(pr).apply, pr.rhs(d), tol, 3000)
    m, st, status = plan.solve(_cuda(d), tol=tol, maxit=3000)
    h = plan.solve_history()
    assert status == mm.MM_OK and h.shape == (st["iters"] + 1,)
    assert h[0] == 1.0 and h[-1] <= tol * (1 + 1e-12) and h[-2] > tol * (1 - 1e-12)
    assert h[-1] == pytest.approx(st["rel_resid_rec"], rel=1e-12)
    ro = np.asarray(ref.rel_hist)
    j = min(10, len(h), len(ro))
    np.testing.assert_allclose(h[:j], ro[:j], rtol=1e-6)
    if len(h) == len(ro):
        assert np.max(np.abs(np.log10(h / ro))) <= 0.1
    # mixed: inner FP32 runs concatenated, each scaled to the outer FP64 residual
    m, st, status = plan.solve(_cuda(d), tol=tol, maxit=5000, solver=mm.MM_SOLVE_MIXED)
    h = plan.solve_history()
    assert status == mm.MM_OK and h.shape == (st["iters"] + 1,)
    assert h[0] == 1.0 and np.all(np.isfinite(h)) and h[-1] <= tol
    j = min(5, len(h), len(ro))
    np.testing.assert_allclose(h[:j], ro[:j], rtol=1e-2)   # FP32 operators, same iteration


def test_nan_data_is_reported():
    """A NaN sample reaches b and the first reduction: both solvers stop with
    MM_ERR_NUMERIC, and the plan solves the repaired data afterwards."""
    scan = tiny_scan(ncomp=3)
    plan = _plan(scan)
    d = _data(scan)
    bad = slice(len(d) // 2, len(d) // 2 + 8)
    d[bad] = np.nan
    for solver in (mm.MM_SOLVE_FP64, mm.MM_SOLVE_MIXED):
        m, st, status = plan.solve(_cuda(d), tol=1e-6, maxit=100, solver=solver, raise_on_error=False)
        assert status == mm.MM_ERR_NUMERIC, (solver, status)
        assert st["converged"] == 0
    d[bad] = 0.0
    m, st, status = plan.solve(_cuda(d), tol=1e-6, maxit=1000)
    assert status == mm.MM_OK and np.all(np.isfinite(plan.solve_history()))
    plan.close()


def test_two_level(case):
    name, scan, pr, plan = case
    k = 8 if pr.n < 2000 else 16
    d0, d1 = _data(scan, 0), _data(scan, 1)
    b0 = pr.rhs(d0)
    bd = oprec.BlockJacobi(pr)
    r0 = pcg(pr.A, bd.apply, b0, 1e-6, 3000, record=True)
    Zo, th = oprec.ritz_coarse_space(r0.alphas, r0.betas, r0.zs, r0.rzs, k)
    tl = oprec.TwoLevel(pr, bd, Zo)
    kk, ritz = plan.build_coarse(k, mm.MM_FP64, bprime=_cuda(b0), tol=1e-6, maxit=3000)
    assert kk >= 1
    # converged (smallest) Ritz values agree with the oracle's Lanczos
    np.testing.assert_allclose(ritz[:3], th[:3], rtol=1e-6)
    ref = pcg(pr.A, tl.apply, pr.rhs(d1), 1e-6, 3000)
    m, st, status = plan.solve(_cuda(d1), tol=1e-6, maxit=3000, kind=mm.MM_PREC_TWOLEVEL)
    assert status == mm.MM_OK
    assert abs(st["iters"] - ref.iters) <= 2, (st["iters"], ref.iters)
    assert _rel(m.cpu().numpy(), ref.x) <= 1e-6
    # M_2lvl application (Eq. 12) against the oracle's operator built on the library's Z
    Zl = plan.coarse_vectors()
    assert np.allclose(Zl.T @ Zl, np.eye(kk), atol=1e-10)
    tl_lib = oprec.TwoLevel(pr, bd, Zl)
    r = np.random.default_rng(5).standard_normal(pr.n)
    z = plan.precond(_cuda(r), mm.MM_PREC_TWOLEVEL, mm.MM_FP64).cpu().numpy()
    assert _rel(z, tl_lib.apply(r)) <= 1e-9
    z32 = plan.precond(_cuda(r, torch.float32), mm.MM_PREC_TWOLEVEL, mm.MM_FP32).cpu().numpy()
    assert _rel(z32, tl_lib.apply(r)) <= 1e-4
    # T5 on the library operator: M_2lvl A Z = Z
    AZ0 = plan.apply_A(_cuda(Zl[:, 0]))
    mz = plan.precond(AZ0, mm.MM_PREC_TWOLEVEL, mm.MM_FP64).cpu().numpy()
    assert _rel(mz, Zl[:, 0]) <= 1e-8
    # mixed two-level reaches the tolerance in the true residual, and its map is within
    # what that residual allows of the oracle's converged map
    m2, st2, status2 = plan.solve(_cuda(d1), tol=1e-6, maxit=3000, kind=mm.MM_PREC_TWOLEVEL,
                                  solver=mm.MM_SOLVE_MIXED)
    assert status2 == mm.MM_OK
    b1 = pr.rhs(d1)
    assert np.linalg.norm(b1 - pr.A(m2.cpu().numpy())) / np.linalg.norm(b1) <= 1e-6
    mstar, kappa_b = _converged(pr, b1)
    assert _rel(m2.cpu().numpy(), mstar) <= kappa_b * (1e-6 + 1e-12)


def test_coarse_threshold_and_import(case):
    # eps_tol selection (Sec. 5) against the oracle's Lanczos, and a basis carried over
    # to a second plan of the same scan gives the same two-level solve
    name, scan, pr, plan = case
    d0, d1 = _data(scan, 0), _data(scan, 1)
    b0 = pr.rhs(d0)
    bd = oprec.BlockJacobi(pr)
    r0 = pcg(pr.A, bd.apply, b0, 1e-6, 3000, record=True)
    _, th = oprec.ritz_coarse_space(r0.alphas, r0.betas, r0.zs, r0.rzs, 8)
    eps = 0.5 * (th[2] + th[3])
    kk, ritz = plan.build_coarse_eps(eps, kmax=64, precision=mm.MM_FP64, bprime=_cuda(b0), tol=1e-6, maxit=3000)
    assert kk == 3
    np.testing.assert_allclose(ritz[:3], th[:3], rtol=1e-6)
    with pytest.raises(mm.MMError) as e:
        plan.build_coarse_eps(0.5 * th[0], precision=mm.MM_FP64, bprime=_cuda(b0), tol=1e-6, maxit=3000)
    assert e.value.status == mm.MM_ERR_STATE
    assert plan.coarse_vectors().shape[1] == 3          # the failed build kept the space
    m1, st1, _ = plan.solve(_cuda(d1), tol=1e-6, maxit=3000, kind=mm.MM_PREC_TWOLEVEL)
    other = _plan(scan)
    assert other.coarse_import(plan.coarse_vectors()) == 3
    m2, st2, _ = other.solve(_cuda(d1), tol=1e-6, maxit=3000, kind=mm.MM_PREC_TWOLEVEL)
    assert st2["iters"] == st1["iters"]
    assert _rel(m2.cpu().numpy(), m1.cpu().numpy()) <= 1e-12
    other.close()


def test_coarse_import_drops_dependent_columns():
    # reading R16 in the library against the oracle's rule: an imported basis is
    # orthonormalised in order and a column whose part orthogonal to the kept ones is
    # below 1e-10 of the largest column norm is dropped.  Exact duplicates, scaled copies,
    # combinations and zero columns go; a near-duplicate 1e-9 away stays, one 1e-11 away
    # goes; the kept basis spans the oracle's kept columns.
    scan = tiny_scan(ncomp=3)
    pr = oracle_problem(scan)
    plan = _plan(scan)
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((pr.n, 9))
    Y[:, 2] = Y[:, 0]
    Y[:, 3] = -3.0 * Y[:, 1]
    Y[:, 4] = Y[:, 0] - 2.0 * Y[:, 1]
    Y[:, 5] = 0.0
    u = rng.standard_normal(pr.n)
    u /= np.linalg.norm(u)
    Y[:, 6] = Y[:, 1] + 1e-9 * np.linalg.norm(Y[:, 1]) * u
    Y[:, 7] = Y[:, 0] + 1e-11 * np.linalg.norm(Y[:, 0]) * u
    Yo, kept = oprec.independent_columns(Y)
    assert kept == [0, 1, 6, 8]
    assert plan.coarse_import(Y) == len(kept)
    Zl = plan.coarse_vectors()
    np.testing.assert_allclose(Zl.T @ Zl, np.eye(len(kept)), atol=1e-12)
    assert np.linalg.norm(Yo - Zl @ (Zl.T @ Yo)) <= 1e-12 * np.linalg.norm(Yo)
    # the installed space acts as the oracle's M_2lvl (Eq. 12) on the library's basis, and
    # on the oracle's own basis of the kept columns up to the conditioning of that basis:
    # the direction of the 1e-9 near-duplicate's orthogonal part is fixed only to
    # ~eps / 1e-9 ~ 2e-7, in both implementations
    bd = oprec.BlockJacobi(pr)
    r = rng.standard_normal(pr.n)
    z = plan.precond(_cuda(r), mm.MM_PREC_TWOLEVEL, mm.MM_FP64).cpu().numpy()
    assert _rel(z, oprec.TwoLevel(pr, bd, Zl).apply(r)) <= 1e-9
    assert _rel(z, oprec.TwoLevel(pr, bd, oprec.orthonormal_basis(Y)[0]).apply(r)) <= 1e-6
    # non-finite columns are reported and the previous space stays
    Y[3, 4] = np.nan
    with pytest.raises(mm.MMError) as e:
        plan.coarse_import(Y)
    assert e.value.status == mm.MM_ERR_NUMERIC
    assert plan.coarse_vectors().shape[1] == len(kept)
    plan.close()


def test_coarse_arnoldi(case):
    # the paper's Ritz source (Algorithm 1 on M_BD A) with eps_tol selection
    name, scan, pr, plan = case
    d0, d1 = _data(scan, 0), _data(scan, 1)
    b0 = pr.rhs(d0)
    bd = oprec.BlockJacobi(pr)
    B = lambda x: bd.apply(pr.A(x))
    W, H, _, _ = oprec.arnoldi(B, bd.apply(b0), 400, tol=1e-8)
    lam = np.sort(np.linalg.eigvals(H[:H.shape[1], :]).real)
    eps = 0.5 * (lam[2] + lam[3])
    Zo, vo = oprec.arnoldi_coarse_space(W, H, 64, eps)
    kk, vals = plan.build_coarse_arnoldi(eps, kmax=64, bprime=_cuda(b0), tol=1e-8, maxit=400)
    assert kk == Zo.shape[1] == 3
    np.testing.assert_allclose(np.sort(vals), np.sort(vo), rtol=1e-6)
    Zl = plan.coarse_vectors()
    np.testing.assert_allclose(Zl.T @ Zl, np.eye(kk), atol=1e-10)
    assert np.linalg.norm(Zl - Zo @ (Zo.T @ Zl)) <= 1e-5 * np.sqrt(kk)   # same span
    ref = pcg(pr.A, oprec.TwoLevel(pr, bd, Zo).apply, pr.rhs(d1), 1e-6, 3000)
    m, st, status = plan.solve(_cuda(d1), tol=1e-6, maxit=3000, kind=mm.MM_PREC_TWOLEVEL)
    assert status == mm.MM_OK and abs(st["iters"] - ref.iters) <= 2, (st["iters"], ref.iters)
    assert _rel(m.cpu().numpy(), ref.x) <= 1e-6
    with pytest.raises(mm.MMError) as e:
        plan.build_coarse_arnoldi(0.5 * lam[0], bprime=_cuda(b0), tol=1e-8, maxit=400)
    assert e.value.status == mm.MM_ERR_STATE


def test_adef2(case):
    # the A-DEF2 form of App. B on the library's a posteriori space, from its starting
    # vector, against the oracle's operator and PCG
    name, scan, pr, plan = case
    d0, d1 = _data(scan, 0), _data(scan, 1)
    kk, _ = plan.build_coarse(8, mm.MM_FP64, bprime=_cuda(pr.rhs(d0)), tol=1e-6, maxit=3000)
    Zl = plan.coarse_vectors()
    bd = oprec.BlockJacobi(pr)
    tl = oprec.TwoLevel(pr, bd, Zl)
    r = np.random.default_rng(9).standard_normal(pr.n)
    z = plan.precond(_cuda(r), mm.MM_PREC_ADEF2, mm.MM_FP64).cpu().numpy()
    assert _rel(z, tl.apply_adef2(r)) <= 1e-9
    z32 = plan.precond(_cuda(r, torch.float32), mm.MM_PREC_ADEF2, mm.MM_FP32).cpu().numpy()
    assert _rel(z32, tl.apply_adef2(r)) <= 1e-4
    b1 = pr.rhs(d1)
    ref = pcg(pr.A, tl.apply_adef2, b1, 1e-6, 3000, x0=tl.adef2_start(b1))
    m, st, status = plan.solve(_cuda(d1), tol=1e-6, maxit=3000, kind=mm.MM_PREC_ADEF2)
    assert status == mm.MM_OK
    assert abs(st["iters"] - ref.iters) <= 2, (st["iters"], ref.iters)
    assert _rel(m.cpu().numpy(), ref.x) <= 1e-6
    m2, st2, status2 = plan.solve(_cuda(d1), tol=1e-6, maxit=3000, kind=mm.MM_PREC_ADEF2, solver=mm.MM_SOLVE_MIXED)
    assert status2 == mm.MM_OK
    assert np.linalg.norm(b1 - pr.A(m2.cpu().numpy())) / np.linalg.norm(b1) <= 1e-6
    mstar, kappa_b = _converged(pr, b1)
    assert _rel(m2.cpu().numpy(), mstar) <= kappa_b * (1e-6 + 1e-12)


def test_two_level_apriori(case):
    # a priori coarse space Z_S (Sec. 3.3.1) merged into r interval groups
    name, scan, pr, plan = case
    K = pr.offsets.size - 1
    r = min(K, 8)
    Zo, kept = oprec.independent_columns(oprec.deflation_apriori_merged(pr, r))
    kk = plan.build_coarse_apriori(r)
    assert kk == len(kept)
    Zl = plan.coarse_vectors()
    # the library keeps an orthonormal basis of the range of the merged hit fractions
    np.testing.assert_allclose(Zl.T @ Zl, np.eye(kk), atol=1e-10)
    assert np.linalg.norm(Zo - Zl @ (Zl.T @ Zo)) <= 1e-10 * np.linalg.norm(Zo)
    bd = oprec.BlockJacobi(pr)
    tl = oprec.TwoLevel(pr, bd, Zo)
    d1 = _data(scan, 1)
    ref = pcg(pr.A, tl.apply, pr.rhs(d1), 1e-6, 3000)
    m, st, status = plan.solve(_cuda(d1), tol=1e-6, maxit=3000, kind=mm.MM_PREC_TWOLEVEL)
    assert status == mm.MM_OK
    assert abs(st["iters"] - ref.iters) <= 2, (st["iters"], ref.iters)
    assert _rel(m.cpu().numpy(), ref.x) <= 1e-6
    r_ = np.random.default_rng(6).standard_normal(pr.n)
    z = plan.precond(_cuda(r_), mm.MM_PREC_TWOLEVEL, mm.MM_FP64).cpu().numpy()
    assert _rel(z, tl.apply(r_)) <= 1e-9
    mz = plan.precond(plan.apply_A(_cuda(Zo[:, 0])), mm.MM_PREC_TWOLEVEL, mm.MM_FP64).cpu().numpy()
    assert _rel(mz, Zo[:, 0]) <= 1e-8
    with pytest.raises(mm.MMError) as e:
        plan.build_coarse_apriori(K + 1 if K < 64 else 65)
    assert e.value.status == mm.MM_ERR_ARG
    assert plan.build_coarse_apriori(r) == kk     # a failed build left the space usable


def test_errors_are_reported():
    scan = tiny_scan()
    with pytest.raises(mm.MMError) as e:
        mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                10 ** 6, scan.fsamp)
    assert e.value.status == mm.MM_ERR_ARG
    bad = scan.pix.copy()
    bad[3] = scan.npix_sky
    with pytest.raises(mm.MMError) as e:
        mm.Plan(bad, scan.npix_sky, None, scan.offsets, scan.interval_psd, scan.psds, scan.lam)
    assert e.value.status == mm.MM_ERR_ARG
    # a hard-truncated steep spectrum has a negative symbol (the oracle's noise pin)
    s2 = synth.raster_scan(8, 8, 1, 8192, 1, 2, 64, [(1.0, 1.0, 4.0)], seed=1)
    with pytest.raises(mm.MMError) as e:
        mm.Plan(s2.pix, s2.npix_sky, None, s2.offsets, s2.interval_psd, s2.psds, 64, window=mm.MM_WINDOW_RECT)
    assert e.value.status == mm.MM_ERR_NOT_SPD
    plan = _plan(scan)
    with pytest.raises(mm.MMError) as e:
        plan.precond(_cuda(np.ones(plan.n)), mm.MM_PREC_TWOLEVEL)
    assert e.value.status == mm.MM_ERR_STATE
    d = _data(scan)
    m, st, status = plan.solve(_cuda(d), tol=1e-12, maxit=2, raise_on_error=False)
    assert status == mm.MM_ERR_NOT_CONVERGED and st["iters"] == 2
    plan.close()


def test_host_buffers_e2e():
    scan = tiny_scan(ncomp=3)
    pr = oracle_problem(scan)
    plan = _plan(scan)
    d = _data(scan)
    out = np.zeros(plan.n)
    st = mm.mm_solve(plan.handle, d, 1e-8, 1000, mm.MM_PREC_BD, mm.MM_SOLVE_FP64, out)[1]
    ref = pcg(pr.A, oprec.BlockJacobi(pr).apply, pr.rhs(d), 1e-8, 1000)
    assert _rel(out, ref.x) <= 1e-6 and st.converged == 1
    plan.close()


@pytest.mark.parametrize("ncomp", [1, 3])
@pytest.mark.parametrize("cl", [2, 4])
def test_cluster_fft_blocks_forced(ncomp, cl):
    # blocks one and two sizes above the single-CTA maximum run on 2- and 4-CTA clusters
    scan = SCANS["T_ragged" if ncomp == 1 else "P_ragged"]()
    pr = oracle_problem(scan)
    lb = 14 + cl // 2
    plan = _plan(scan, fft_log2=(lb, lb + 1))
    assert plan.fft_block_f64 == 2 ** lb and plan.fft_block_f32 == 2 ** (lb + 1)
    rng = np.random.default_rng(8)
    t = rng.standard_normal(pr.nt)
    x = rng.standard_normal(pr.n)
    for prec, dt, tol in ((mm.MM_FP64, torch.float64, 1e-12), (mm.MM_FP32, torch.float32, 2e-5)):
        tc = _cuda(t, dt)
        z = plan.apply_ninv(tc, prec).cpu().numpy()
        assert _rel(z, pr.Ninv(tc.double().cpu().numpy())) <= tol
        xc = _cuda(x, dt)
        y = plan.apply_A(xc, prec).cpu().numpy()
        assert _rel(y, pr.A(xc.double().cpu().numpy())) <= (tol if prec == mm.MM_FP64 else 3e-5)
    plan.close()


@pytest.mark.parametrize("case", ["P_ragged", "c2_small"])
def test_autotuned_blocks(case):
    # the autotuner times the cheapest admissible blocks and keeps the fastest; the
    # operator stays within the same tolerances as with cost-model blocks
    scan = SCANS[case]()
    pr = oracle_problem(scan)
    plan = _plan(scan, autotune=True)
    ms64, ms32 = plan.autotune_ms()
    for ms, block in ((ms64, plan.fft_block_f64), (ms32, plan.fft_block_f32)):
        if len(ms) >= 2:   # the kept block is a fastest one (ties keep the cheaper model cost)
            assert ms[block.bit_length() - 1] == min(ms.values())
        assert 1 <= len(ms) <= 3 or len(ms) == 0
    rng = np.random.default_rng(21)
    x = rng.standard_normal(pr.n)
    ref = pr.A(x)
    for prec, dt, tol in ((mm.MM_FP64, torch.float64, 1e-12), (mm.MM_FP32, torch.float32, 3e-5)):
        xc = _cuda(x, dt)
        y = plan.apply_A(xc, prec).cpu().numpy()
        assert _rel(y, pr.A(xc.double().cpu().numpy())) <= tol
    plan.close()


@pytest.mark.parametrize("lam", [8192, 16384, 40000])
def test_long_band_uses_cluster_blocks(lam):
    # lambda = 8192 (the large polarised workload's band) needs a cluster FP64 block,
    # lambda = 16384 (the longest batched band) the four-CTA FP64 block, and
    # lambda = 40000 exceeds every FP64 block (2^16 reals) but fits the four-CTA FP32 one
    scan = synth.raster_scan(64, 64, 1, 4 * 2 ** 17, 1, 4, lam, [(1.0, 1.0, 1.0)], seed=9)
    pr = oracle_problem(scan)
    plan = _plan(scan)
    assert plan.fft_block_f64 in {8192: (2 ** 15, 2 ** 16), 16384: (2 ** 16,), 40000: (0,)}[lam]
    assert plan.fft_block_f32 in {8192: (2 ** 15, 2 ** 16, 2 ** 17), 16384: (2 ** 16, 2 ** 17), 40000: (2 ** 17,)}[lam]
    if lam == 40000:
        with pytest.raises(mm.MMError) as e:
            plan.apply_ninv(_cuda(np.ones(pr.nt)), mm.MM_FP64)
        assert e.value.status == mm.MM_ERR_ARG
    rng = np.random.default_rng(lam)
    t = rng.standard_normal(pr.nt)
    ref = pr.Ninv(t, route="fft")
    if lam != 40000:
        z = plan.apply_ninv(_cuda(t), mm.MM_FP64).cpu().numpy()
        assert _rel(z, ref) <= 1e-12
    tc = _cuda(t, torch.float32)
    z32 = plan.apply_ninv(tc, mm.MM_FP32).cpu().numpy()
    assert _rel(z32, pr.Ninv(tc.double().cpu().numpy(), route="fft")) <= 2e-5
    plan.close()


@pytest.mark.parametrize("ncomp", [1, 3])
def test_white_noise_is_binned_map(ncomp):
    # white noise with lambda = 0 (N diagonal, Sec. 2): the GLS map is the per-pixel
    # noise-weighted binned map, written here directly from the data (no oracle), and
    # M_BD is A^-1, so PCG converges in one step.  Intervals include a single sample.
    rng = np.random.default_rng(30 + ncomp)
    npix, nt = 40, 5000
    pix = rng.integers(0, npix, nt).astype(np.int32)
    offsets = np.array([0, 1, 7, 1200, 3000, nt], dtype=np.int64)
    sig = np.array([1.0, 0.5, 2.0])
    ipsd = np.array([0, 1, 2, 0, 1], dtype=np.int32)
    psds = [(s, 0.0, 1.0) for s in sig]
    phi = rng.uniform(0, np.pi, nt)
    w = np.stack([np.cos(2 * phi), np.sin(2 * phi)], axis=1) if ncomp == 3 else None
    d = rng.standard_normal(nt)
    plan = mm.Plan(pix, npix, w, offsets, ipsd, psds, 0, 100.0)
    m, st, status = plan.solve(_cuda(d), tol=1e-12, maxit=10)
    assert status == mm.MM_OK and st["iters"] <= 1
    inv = np.repeat(1.0 / sig[ipsd] ** 2, np.diff(offsets))
    o2s, _ = plan.pixels()
    mh = m.cpu().numpy().reshape(-1, ncomp)
    for q, p in enumerate(o2s):
        sel = pix == p
        if ncomp == 1:
            ref = np.sum(inv[sel] * d[sel]) / np.sum(inv[sel])
            assert abs(mh[q, 0] - ref) <= 1e-12 * max(1.0, abs(ref))
        else:
            W = np.column_stack([np.ones(sel.sum()), w[sel]])
            Bp = (W * inv[sel, None]).T @ W
            ref = np.linalg.solve(Bp, (W * inv[sel, None]).T @ d[sel])
            np.testing.assert_allclose(mh[q], ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    plan.close()
