"""Batched right-hand sides (many noise realisations through one plan) -- needs a GPU.

Each column must match its single-RHS counterpart: the batched FP32 operator to the FP32
operator tolerance (3e-5 relative vs the FP64 oracle), and every batched solve must
reach the requested relative residual in the oracle's FP64 arithmetic.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1408_3048_gb300 import mm, synth
from problems import oracle_problem, tiny_scan

pytestmark = pytest.mark.gpu

CASES = {
    "T": lambda: synth.raster_scan(24, 20, 3, 20000, 1, 3, 300, [(1.0, 1.0, 1.0), (0.7, 2.0, 1.7), (1.3, 0.3, 1.2)],
                                   det_psd=[0, 1, 2], uneven=(2000, 12000), seed=4),
    "P": lambda: synth.raster_scan(24, 24, 4, 24000, 3, 4, 500, [(1.0, 1.0, 1.0), (0.8, 1.5, 1.5)],
                                   det_psd=[0, 1, 0, 1], uneven=(3000, 9000), seed=5),
}


def _plan(scan, stream=None):
    return mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.lam, scan.fsamp, stream=stream)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("R", [1, 2, 5, 64])
def test_batched_operator(name, R):
    scan = CASES[name]()
    pr = oracle_problem(scan)
    plan = _plan(scan)
    X = torch.randn(R, plan.n, dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(R))
    Y = plan.apply_A_batch(X).cpu().numpy()
    Xh = X.double().cpu().numpy()
    for r in range(R):
        ref = pr.A(Xh[r])
        assert np.linalg.norm(Y[r] - ref) / np.linalg.norm(ref) <= 3e-5, r
    plan.close()


def _data(scan, R, seed0):
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 7)
    return np.stack([synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds,
                                                                  scan.fsamp, seed0 + r)) for r in range(R)])


@pytest.mark.parametrize("name", list(CASES))
def test_batched_solve_reaches_tol_per_column(name):
    scan = CASES[name]()
    pr = oracle_problem(scan)
    R = 5
    D = _data(scan, R, 100)
    s = torch.cuda.Stream()
    plan = _plan(scan, stream=s)          # private stream: iterations replayed from a graph
    M, st, status = plan.solve_batch(torch.from_numpy(D).cuda(), tol=1e-6, maxit=5000)
    assert status == mm.MM_OK
    Mh = M.cpu().numpy()
    single = _plan(scan)
    for r in range(R):
        b = pr.rhs(D[r])
        assert np.linalg.norm(b - pr.A(Mh[r])) / np.linalg.norm(b) <= 1e-6, r
        assert st[r]["converged"] == 1 and st[r]["rel_resid"] <= 1e-6
        m1, st1, _ = single.solve(torch.from_numpy(D[r]).cuda(), tol=1e-6, maxit=5000, solver=mm.MM_SOLVE_MIXED)
        m1 = m1.cpu().numpy()
        assert np.linalg.norm(Mh[r] - m1) / np.linalg.norm(m1) <= 1e-4
        assert abs(st[r]["iters"] - st1["iters"]) <= 3
    plan.close()
    single.close()


def test_batched_solve_graph_and_direct_paths_agree_and_groups():
    scan = CASES["P"]()
    R = 70                                 # two groups of at most 64 columns
    D = torch.from_numpy(_data(scan, R, 300)).cuda()
    a = _plan(scan, stream=torch.cuda.Stream())
    b = _plan(scan)                        # legacy default stream: direct launches
    Ma, sta, _ = a.solve_batch(D, tol=1e-6)
    Mb, stb, _ = b.solve_batch(D, tol=1e-6)
    assert torch.equal(Ma, Mb)
    assert [x["iters"] for x in sta] == [x["iters"] for x in stb]
    assert all(x["converged"] == 1 for x in sta)
    a.close()
    b.close()


def test_batched_rejects_unsupported_options():
    scan = tiny_scan()
    plan = _plan(scan)
    D = torch.zeros(2, scan.nt, dtype=torch.float64, device="cuda")
    o = mm.mm_solve_opts(tol=1e-6, maxit=10, kind=mm.MM_PREC_BD, solver=mm.MM_SOLVE_FP64)
    M = torch.empty(2, plan.n, dtype=torch.float64, device="cuda")
    with pytest.raises(mm.MMError) as e:
        mm.mm_solve_batch(plan.handle, D, 2, o, M)
    assert e.value.status == mm.MM_ERR_ARG
    plan.close()
