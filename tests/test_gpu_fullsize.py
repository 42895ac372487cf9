"""Full-size workloads on the GPU against oracle results stored by the golden scripts
(tests/golden/make_c2_oracle.py, make_c3_oracle.py -- oracle only) and against
properties that hold at any size.  Needs a GPU; each test takes seconds to a minute.

Tolerances:
  * iteration counts at tolerance within 2 of the oracle's (same algorithm, FP64);
  * whole maps, when both run the same FP64 algorithm to the same tolerance, within 1e-6
    relative L2 of the oracle's map (reading R11);
  * every map at residual target tol against the oracle's converged map m* (PCG to 1e-10):
    relative L2 error <= kappa_b tol, kappa_b = ||M_BD|| ||b|| / (theta_1 ||m*||) stored
    by the golden script (||m - m*|| <= ||A^-1|| rho ||b|| for a true residual rho ||b||,
    ||A^-1|| <= ||M_BD|| / lambda_min(M_BD A), lambda_min estimated by the smallest Ritz
    value theta_1 of the oracle's 1e-10 run), with tol + 1e-10 for m*'s own residual;
  * the overlap-save operators at the benchmark kernel's shape element by element:
    FP64 1e-12, FP32 2e-5 (N^-1) / 3e-5 (A) of the largest output.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1408_3048_gb300 import mm, synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    p = os.path.join(GOLDEN, name)
    if not os.path.exists(p):
        pytest.skip(f"{name} not generated")
    if name.endswith(".npz"):
        with np.load(p) as z:
            return {k: z[k] for k in z.files}
    with open(p) as f:
        return json.load(f)


def _plan(scan, **kw):
    return mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.lam, scan.fsamp, **kw)


def _tod(scan, sky_seed, noise_seed):
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, sky_seed)
    return synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp,
                                                        noise_seed))


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_polarised_2e24_matches_oracle_iterations_and_map():
    g = _load("c2_oracle.json")
    maps = _load("c2_maps.npz")
    mstar = maps["m_star"]
    m_bd_or = mstar + maps["d_bd"].astype(np.float64)
    m_2l_or = mstar + maps["d_2lvl"].astype(np.float64)
    bound = g["kappa_b"] * (1e-6 + 1e-10)
    scan = synth.config(2)
    plan = _plan(scan)
    assert plan.n == g["n"] and plan.npix_obs == g["npix_obs"]
    d0 = torch.from_numpy(_tod(scan, 1002, 2200)).cuda()
    d1 = torch.from_numpy(_tod(scan, 1002, 2201)).cuda()
    errs = {}
    m, st, status = plan.solve(d1, tol=1e-6, maxit=5000, kind=mm.MM_PREC_BD)
    assert status == mm.MM_OK and abs(st["iters"] - g["iters_bd"]) <= 2
    errs["fp64_bd_vs_oracle_bd"] = _rel(m.cpu().numpy(), m_bd_or)
    assert errs["fp64_bd_vs_oracle_bd"] <= 1e-6
    kk, ritz = plan.build_coarse(g["k"], mm.MM_FP64, bprime=plan.rhs(d0), tol=1e-6, maxit=5000)
    assert kk == g["k_kept"]
    np.testing.assert_allclose(ritz[:4], g["ritz"][:4], rtol=1e-4)
    m2, st2, status2 = plan.solve(d1, tol=1e-6, maxit=5000, kind=mm.MM_PREC_TWOLEVEL)
    assert status2 == mm.MM_OK and abs(st2["iters"] - g["iters_2lvl"]) <= 2
    errs["fp64_2lvl_vs_oracle_2lvl"] = _rel(m2.cpu().numpy(), m_2l_or)
    assert errs["fp64_2lvl_vs_oracle_2lvl"] <= 1e-6
    # the converged FP64 map and every 1e-6 map against the oracle's m*
    m3, st3, _ = plan.solve(d1, tol=1e-10, maxit=5000, kind=mm.MM_PREC_BD)
    assert abs(st3["iters"] - g["iters_bd_1e-10"]) <= 2
    errs["fp64_bd_1e-10_vs_m*"] = _rel(m3.cpu().numpy(), mstar)
    assert errs["fp64_bd_1e-10_vs_m*"] <= g["kappa_b"] * 2e-10
    for kind, name in ((mm.MM_PREC_TWOLEVEL, "mixed_2lvl"), (mm.MM_PREC_BD, "mixed_bd")):
        mx, stx, sx = plan.solve(d1, tol=1e-6, maxit=5000, kind=kind, solver=mm.MM_SOLVE_MIXED)
        assert sx == mm.MM_OK and stx["rel_resid"] <= 1e-6
        errs[f"{name}_vs_m*"] = _rel(mx.cpu().numpy(), mstar)
        assert errs[f"{name}_vs_m*"] <= bound, (name, errs, bound)
    for nm in ("fp64_bd", "fp64_2lvl"):
        assert g[f"err_{nm.split('_')[1]}_vs_star"] <= bound      # the oracle's own maps obey it too
    if "iters_2lvl_z1e-10" in g:
        # the bench's coarse space: Ritz vectors from the first solve run to 1e-10 in FP64
        kk, ritz = plan.build_coarse(g["k"], mm.MM_FP64, bprime=plan.rhs(d0), tol=1e-10, maxit=5000)
        np.testing.assert_allclose(ritz[:3], g["ritz_z1e-10"][:3], rtol=1e-4)
        m4, st4, status4 = plan.solve(d1, tol=1e-6, maxit=5000, kind=mm.MM_PREC_TWOLEVEL)
        assert status4 == mm.MM_OK and abs(st4["iters"] - g["iters_2lvl_z1e-10"]) <= 2
        errs["fp64_2lvl_z1e-10_vs_oracle"] = _rel(m4.cpu().numpy(), mstar + maps["d_2lvl_z1e10"].astype(np.float64))
        errs["fp64_2lvl_z1e-10_vs_m*"] = _rel(m4.cpu().numpy(), mstar)
        assert errs["fp64_2lvl_z1e-10_vs_m*"] <= bound
        mx, stx, sx = plan.solve(d1, tol=1e-6, maxit=5000, kind=mm.MM_PREC_TWOLEVEL, solver=mm.MM_SOLVE_MIXED)
        assert sx == mm.MM_OK and stx["rel_resid"] <= 1e-6
        errs["mixed_2lvl_z1e-10_vs_m*"] = _rel(mx.cpu().numpy(), mstar)
        assert errs["mixed_2lvl_z1e-10_vs_m*"] <= bound
    print(f"\nmap errors (bound {bound:.2e}): {errs}")
    plan.close()


@pytest.mark.parametrize("prec", [mm.MM_FP64, mm.MM_FP32])
def test_operators_at_the_benchmark_kernel_shape(prec):
    # the bench's dominant launches: I/Q/U, lambda = 4096, overlap-save block B = 2^15
    # (FP32: one CTA per tile; FP64: the 2-CTA cluster form), compared element by element
    # with the oracle's FFT route on the polarised scan at 1/4 of its samples (2^22,
    # intervals 6813 .. 29440 samples, several tiles each and ragged last tiles)
    from oracle.system import Problem
    scan = synth.config(2, scale=4)
    scan.lam = 4096
    pr = Problem(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                 scan.fsamp, scan.lam, scan.ncomp)
    plan = _plan(scan, fft_log2=(15, 15))
    assert plan.fft_block_f32 == 2 ** 15 and plan.fft_block_f64 == 2 ** 15
    dt = torch.float64 if prec == mm.MM_FP64 else torch.float32
    tol_n, tol_a = (1e-12, 1e-12) if prec == mm.MM_FP64 else (2e-5, 3e-5)
    rng = np.random.default_rng(21)
    y = rng.standard_normal(scan.nt)
    z = plan.apply_ninv(torch.as_tensor(y, dtype=dt).cuda(), prec).double().cpu().numpy()
    zr = pr.Ninv(y, route="fft")
    assert np.abs(z - zr).max() <= tol_n * np.abs(zr).max()
    assert _rel(z, zr) <= tol_n
    x = rng.standard_normal(pr.n)
    ax = plan.apply_A(torch.as_tensor(x, dtype=dt).cuda(), prec).double().cpu().numpy()
    ar = pr.A(x, route="fft")
    assert np.abs(ax - ar).max() <= tol_a * np.abs(ar).max()
    assert _rel(ax, ar) <= tol_a
    if prec == mm.MM_FP64:
        # the refinement residual of the mixed solver at this shape: double-float and FP64
        # band products against the oracle's b - A x, within 1e-12 of ||b||
        d = y + pr.P(rng.standard_normal(pr.n))
        b = pr.rhs(d, route="fft")
        ref = b - ar
        for arith in (mm.MM_RESID_DF32, mm.MM_RESID_FP64):
            r = plan.residual(torch.from_numpy(d).cuda(), torch.from_numpy(x).cuda(), arith).cpu().numpy()
            assert np.linalg.norm(r - ref) <= 1e-12 * np.linalg.norm(b), arith
    plan.close()


def test_temperature_2e27_mixed_precision_error_vs_oracle():
    # the 2^27-sample temperature workload: mixed-precision maps at tolerances 1e-6 and
    # 1e-8, block-Jacobi and two-level (k = 64, FP64 E), against the oracle's m*
    g = _load("c3_oracle.json")
    mstar = _load("c3_map.npz")["m_star"]
    scan = synth.config(3)
    plan = _plan(scan)
    assert plan.n == g["n"]
    d = torch.from_numpy(_tod(scan, 1003, 2301)).cuda()
    m64, st64, _ = plan.solve(d, tol=1e-6, maxit=5000)
    assert abs(st64["iters"] - g["iters_1e-6"]) <= 2
    errs = {}

    def check(name):
        for tol in (1e-6, 1e-8):
            kind = mm.MM_PREC_BD if name == "bd" else mm.MM_PREC_TWOLEVEL
            m, st, status = plan.solve(d, tol=tol, maxit=5000, kind=kind, solver=mm.MM_SOLVE_MIXED)
            assert status == mm.MM_OK and st["rel_resid"] <= tol
            errs[(name, tol)] = _rel(m.cpu().numpy(), mstar)
            assert errs[(name, tol)] <= g["kappa_b"] * (tol + 1e-10), (name, tol, errs, g["kappa_b"])

    check("bd")
    # two-level with up to k = 64 Ritz vectors of M_BD A and an FP64 E.  A CG-Lanczos run
    # yields at most one Ritz pair per step and block-Jacobi PCG meets 1e-10 here in about
    # 54 steps, so the first solve runs in FP64 to 1e-13 to offer 64 of them.  (The a
    # priori space does not apply: every group of consecutive intervals of this raster
    # covers the patch exactly once per cycle, so all merged hit-fraction columns agree.)
    kk, _ = plan.build_coarse(64, mm.MM_FP64, bprime=plan.rhs(d), tol=1e-13, maxit=5000)
    assert kk >= 48
    check(f"2lvl_ritz_k{kk}")
    print(f"\nmixed-precision error vs FP64 oracle m* (kappa_b {g['kappa_b']:.1f}): {errs}")
    plan.close()


def test_differentiable_2e29_solve_and_gradient():
    # (takes a few minutes: 2^29 samples, five plans)
    # 1024 x 768 grid, 64 detectors x 2^23 samples, lambda 8192, two-level k = 64:
    # properties that hold at any size (the oracle cannot run this size)
    scan = synth.config(5)
    assert scan.nt == 2 ** 29
    plan = _plan(scan, stream=torch.cuda.Stream())
    frac = plan.npix_obs / scan.npix_sky
    assert 0.55 <= frac <= 0.65
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.standard_normal(plan.n)).cuda()
    y = torch.from_numpy(rng.standard_normal(plan.n)).cuda()
    Ax, Ay = plan.apply_A(x), plan.apply_A(y)
    assert abs(float(y @ Ax) - float(x @ Ay)) <= 1e-11 * float(torch.linalg.norm(Ax) * torch.linalg.norm(y))
    d = torch.from_numpy(_tod(scan, 1005, 2501)).cuda()
    kk, _ = plan.build_coarse(64, mm.MM_FP32, bprime=plan.rhs(d), tol=1e-6, maxit=5000)
    assert kk == 64
    _, st_bd, s1 = plan.solve(d, tol=1e-6, maxit=10000, kind=mm.MM_PREC_BD, solver=mm.MM_SOLVE_MIXED)
    _, st_2l, s2 = plan.solve(d, tol=1e-6, maxit=10000, kind=mm.MM_PREC_TWOLEVEL, solver=mm.MM_SOLVE_MIXED)
    assert s1 == s2 == mm.MM_OK and st_2l["iters"] < st_bd["iters"]
    # adjoint data gradient of L = 1/2 ||m - m_ref||^2 against a central difference
    mref = torch.from_numpy(rng.standard_normal(plan.n)).cuda()
    kw = dict(tol=1e-10, maxit=20000, kind=mm.MM_PREC_TWOLEVEL, solver=mm.MM_SOLVE_MIXED)
    m, _, _ = plan.solve(d, **kw)
    dd, dp, _ = plan.grad(d, m, m - mref, **kw)
    assert np.all(np.isfinite(dp))
    e = torch.from_numpy(rng.standard_normal(plan.nt)).cuda()
    h = 1e-4 * float(torch.linalg.norm(d)) / float(torch.linalg.norm(e))

    def loss(dv):
        mm_, _, _ = plan.solve(dv, **kw)
        return 0.5 * float(torch.sum((mm_ - mref) ** 2))

    fd = (loss(d + h * e) - loss(d - h * e)) / (2 * h)
    assert fd == pytest.approx(float(dd @ e), rel=1e-3)
    # noise-PSD gradient (f_knee, alpha of PSD 0) against central differences of
    # re-planned problems, relative step 1e-4 (the loss depends on m only, so the
    # perturbed solves need no coarse space)
    psds = np.array(scan.psds, dtype=np.float64).reshape(-1, 3)
    for comp in (1, 2):
        th = psds[0, comp]
        hp = 1e-4 * th
        Ls = []
        for sgn in (1.0, -1.0):
            ps = psds.copy()
            ps[0, comp] = th + sgn * hp
            p2 = mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, ps, scan.lam,
                         scan.fsamp, stream=plan.stream)
            m2, _, _ = p2.solve(d, tol=1e-11, maxit=20000, kind=mm.MM_PREC_BD, solver=mm.MM_SOLVE_MIXED)
            Ls.append(0.5 * float(torch.sum((m2 - mref) ** 2)))
            p2.close()
        assert (Ls[0] - Ls[1]) / (2 * hp) == pytest.approx(float(dp[0][comp]), rel=1e-3)
    plan.close()


@pytest.fixture(scope="module")
def realisations_2e24():
    scan = synth.config(2)
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 1002)
    return np.stack([synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds,
                                                                  scan.fsamp, 2400 + r)) for r in range(64)])


@pytest.mark.parametrize("lam", [1024, 16384])
def test_batched_2e24_64_realisations(lam, realisations_2e24):
    # the batched Monte-Carlo workload: 64 noise realisations of the 2^24-sample polarised
    # scan in one batched solve; every checked column's true residual, recomputed with the
    # FP64 operator (a separate code path from the batched FP32 one), meets the
    # tolerance, and one column's map matches its single-RHS mixed solve
    scan = synth.config(2)
    scan.lam = lam
    plan = _plan(scan, stream=torch.cuda.Stream())
    Dc = torch.from_numpy(realisations_2e24).cuda()
    M, st, status = plan.solve_batch(Dc, tol=1e-6, maxit=5000)
    assert status == mm.MM_OK and all(x["converged"] == 1 for x in st)
    for r in (0, 17, 63):
        b = plan.rhs(Dc[r].contiguous())
        res = b - plan.apply_A(M[r].contiguous())
        assert float(torch.linalg.norm(res) / torch.linalg.norm(b)) <= 1e-6
    m1, _, _ = plan.solve(Dc[5].contiguous(), tol=1e-6, maxit=5000, solver=mm.MM_SOLVE_MIXED)
    assert float(torch.linalg.norm(M[5] - m1) / torch.linalg.norm(m1)) <= 1e-4
    plan.close()
