"""Adjoint / noise-PSD gradient of the CUDA path vs the oracle and finite differences (GPU).

Tolerances: FP64 solves at tol 1e-13; the data gradient to 1e-8 and the PSD gradient
to 1e-6 relative against the oracle (both solve to ~1e-13, so the map error is ~1e-12
times the condition number); finite differences (central, step 1e-4 relative) to 1e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as oadj
from oracle import precond as oprec
from paper_1408_3048_gb300 import mm, synth
from problems import oracle_problem, tiny_scan

pytestmark = pytest.mark.gpu


def _plan(scan, psds=None):
    return mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd,
                   scan.psds if psds is None else psds, scan.lam, scan.fsamp)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _case(ncomp, ragged):
    if ragged:
        return synth.raster_scan(24, 24, 4, 24000, ncomp, 4, 500, [(1.0, 1.0, 1.0), (0.8, 1.5, 1.5)],
                                 det_psd=[0, 1, 0, 1], uneven=(3000, 9000), seed=5)
    return tiny_scan(ncomp=ncomp, psds=((1.0, 2.0, 1.5), (1.3, 0.7, 1.2)), lam=8)


@pytest.mark.parametrize("ncomp", [1, 3])
@pytest.mark.parametrize("ragged", [False, True])
def test_gradients_match_oracle(ncomp, ragged):
    scan = _case(ncomp, ragged)
    pr = oracle_problem(scan)
    rng = np.random.default_rng(ncomp + 10 * ragged)
    d = synth.tod(scan, synth.sky_map(scan.npix_sky, ncomp, 3), rng.standard_normal(scan.nt))
    mref = rng.standard_normal(pr.n)
    plan = _plan(scan)
    dc = torch.from_numpy(d).cuda()
    m, st, _ = plan.solve(dc, tol=1e-13, maxit=20000)
    g = m - torch.from_numpy(mref).cuda()
    dd, dp, gst = plan.grad(dc, m, g, tol=1e-13, maxit=20000)
    mo = m.cpu().numpy()
    go = g.cpu().numpy()
    if ragged:
        ref_d, ref_p = oadj.gradients(pr, d, mo, go, apply_M=oprec.BlockJacobi(pr).apply, tol=1e-13)
    else:
        ref_d, ref_p = oadj.gradients(pr, d, mo, go, dense=True)
    assert _rel(dd.cpu().numpy(), ref_d) <= 1e-8
    assert np.abs(dp - ref_p).max() <= 1e-6 * np.abs(ref_p).max()
    plan.close()


def test_psd_gradient_matches_finite_differences():
    scan = _case(3, False)
    rng = np.random.default_rng(4)
    d = synth.tod(scan, synth.sky_map(scan.npix_sky, 3, 3), rng.standard_normal(scan.nt))
    dc = torch.from_numpy(d).cuda()
    plan = _plan(scan)
    m, _, _ = plan.solve(dc, tol=1e-13, maxit=20000)
    mref = torch.from_numpy(rng.standard_normal(plan.n)).cuda()
    _, dp, _ = plan.grad(dc, m, m - mref, tol=1e-13, maxit=20000, want_d=False)
    plan.close()

    def loss(psds):
        p = _plan(scan, psds)
        mm_, _, _ = p.solve(dc, tol=1e-13, maxit=20000)
        p.close()
        return 0.5 * float(torch.sum((mm_ - mref) ** 2))

    th = np.array(scan.psds, dtype=np.float64)
    for p in range(th.shape[0]):
        for c in range(3):
            h = 1e-4 * th[p, c]
            tp, tm = th.copy(), th.copy()
            tp[p, c] += h
            tm[p, c] -= h
            fd = (loss(tp) - loss(tm)) / (2 * h)
            assert fd == pytest.approx(dp[p, c], rel=1e-4, abs=1e-7 * np.abs(dp).max()), (p, c, fd, dp[p, c])


def test_shared_sigma_gradient_vanishes():
    scan = tiny_scan(ncomp=3, psds=((1.4, 1.5, 1.3),), lam=8)
    rng = np.random.default_rng(2)
    d = torch.from_numpy(rng.standard_normal(scan.nt)).cuda()
    plan = _plan(scan)
    m, _, _ = plan.solve(d, tol=1e-13, maxit=20000)
    _, dp, _ = plan.grad(d, m, m - torch.from_numpy(rng.standard_normal(plan.n)).cuda(), tol=1e-13,
                         maxit=20000, want_d=False)
    assert abs(dp[0, 0]) <= 1e-8 * np.abs(dp[0, 1:]).max()
    plan.close()


def test_autograd_wrapper():
    scan = _case(3, True)
    rng = np.random.default_rng(6)
    d = torch.from_numpy(synth.tod(scan, synth.sky_map(scan.npix_sky, 3, 3),
                                   rng.standard_normal(scan.nt))).cuda().requires_grad_(True)
    theta = torch.tensor(np.array(scan.psds), dtype=torch.float64, requires_grad=True)
    plan = _plan(scan)
    mref = torch.from_numpy(rng.standard_normal(plan.n)).cuda()
    m = mm.map_solve(plan, d, theta, tol=1e-12)
    L = 0.5 * torch.sum((m - mref) ** 2)
    gd, gth = torch.autograd.grad(L, [d, theta])
    dd, dp, _ = plan.grad(d.detach(), m.detach(), (m - mref).detach(), tol=1e-12)
    assert torch.allclose(gd, dd, rtol=1e-10, atol=0)
    assert np.allclose(gth.numpy(), dp, rtol=1e-10, atol=0)
    # directional derivative in d by central differences through the forward op
    e = torch.from_numpy(rng.standard_normal(scan.nt)).cuda()
    h = 1e-3
    with torch.no_grad():
        Lp = 0.5 * torch.sum((mm.map_solve(plan, d + h * e, theta, tol=1e-13) - mref) ** 2)
        Lm = 0.5 * torch.sum((mm.map_solve(plan, d - h * e, theta, tol=1e-13) - mref) ** 2)
    fd = float((Lp - Lm) / (2 * h))
    assert fd == pytest.approx(float(gd @ e), rel=1e-6)
    plan.close()
