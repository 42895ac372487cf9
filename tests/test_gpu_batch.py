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


def _plan(scan, stream=None, **kw):
    return mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.lam, scan.fsamp, stream=stream, **kw)


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("R", [1, 2, 5, 64])
def test_batched_operator(name, R, kind):
    # kind 0: two columns per complex FFT; kind 1: one real FFT per column; kind 2: the
    # band product on the tensor cores (FP16 split operands, FP32 accumulators)
    scan = CASES[name]()
    pr = oracle_problem(scan)
    plan = _plan(scan)
    assert plan.batch_config(R, kind)[0] == kind
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


def test_batched_nan_column_is_reported():
    """NaN samples in one column's data: MM_ERR_NUMERIC, that column not converged with a
    NaN residual (never a converged zero map), the other columns still solved to tol."""
    scan = CASES["P"]()
    pr = oracle_problem(scan)
    D = _data(scan, 3, 300)
    D[1, 5000:5008] = np.nan
    plan = _plan(scan, stream=torch.cuda.Stream())
    M, st, status = plan.solve_batch(torch.from_numpy(D).cuda(), tol=1e-6, maxit=5000, raise_on_error=False)
    assert status == mm.MM_ERR_NUMERIC
    assert st[1]["converged"] == 0 and np.isnan(st[1]["rel_resid"])
    Mh = M.cpu().numpy()
    for r in (0, 2):
        b = pr.rhs(D[r])
        assert st[r]["converged"] == 1, r
        assert np.linalg.norm(b - pr.A(Mh[r])) / np.linalg.norm(b) <= 1e-6, r
    plan.close()


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


def test_batched_form_autotuned_and_fixed():
    scan = CASES["P"]()
    plan = _plan(scan, autotune=True)
    kind, lb, ms = plan.batch_config(8)
    assert kind in (0, 1, 2) and ms[0] > 0 and ms[1] > 0 and ms[2] > 0
    assert kind == int(np.argmin(ms))
    with pytest.raises(mm.MMError) as e:          # the form is fixed once chosen
        plan.batch_config(8, (kind + 1) % 3)
    assert e.value.status == mm.MM_ERR_ARG
    assert plan.batch_config(8, kind)[0] == kind
    plan.close()


@pytest.mark.parametrize("name", list(CASES))
def test_batched_solve_tensor_form(name):
    # the batched solver on the tensor-core operator: every column reaches the tolerance
    # in the oracle's FP64 arithmetic
    scan = CASES[name]()
    pr = oracle_problem(scan)
    R = 5
    D = _data(scan, R, 300)
    plan = _plan(scan, stream=torch.cuda.Stream())
    assert plan.batch_config(R, 2)[0] == 2
    M, st, status = plan.solve_batch(torch.from_numpy(D).cuda(), tol=1e-6, maxit=5000)
    assert status == mm.MM_OK
    Mh = M.cpu().numpy()
    for r in range(R):
        b = pr.rhs(D[r])
        assert st[r]["converged"] == 1
        assert np.linalg.norm(b - pr.A(Mh[r])) / np.linalg.norm(b) <= 1e-6, r
    plan.close()


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


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("lam", [8192, 16384])
def test_batched_operator_cluster_blocks(lam, kind):
    # bands beyond the single-CTA complex block (2^14 points) take the 2-CTA (2^15) and
    # 4-CTA (2^16) cluster blocks in the pair form, the real form the FP32 cluster blocks;
    # R = 3 leaves the last column pair half empty
    scan = synth.raster_scan(64, 48, 2, 3 * 2 ** 16, 3, 2, lam, [(1.0, 1.0, 1.0), (0.8, 1.5, 1.5)],
                             det_psd=[0, 1], uneven=(2 ** 16 + 5, 2 ** 17 - 7), seed=11)
    pr = oracle_problem(scan)
    plan = _plan(scan)
    R = 3
    k, lb, _ = plan.batch_config(R, kind)
    assert k == kind and (lb >= (15 if lam == 8192 else 16) if kind != 2 else lb == 7)
    X = torch.randn(R, plan.n, dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(lam))
    Y = plan.apply_A_batch(X).cpu().numpy()
    Xh = X.double().cpu().numpy()
    for r in range(R):
        ref = pr.A(Xh[r], route="fft")
        assert np.linalg.norm(Y[r] - ref) / np.linalg.norm(ref) <= 3e-5, r
    D = torch.from_numpy(_data(scan, R, 500)).cuda()
    M, st, status = plan.solve_batch(D, tol=1e-6, maxit=3000)
    assert status == mm.MM_OK
    Mh = M.cpu().numpy()
    for r in range(R):
        b = pr.rhs(D[r].cpu().numpy(), route="fft")
        assert st[r]["converged"] == 1
        assert np.linalg.norm(b - pr.A(Mh[r], route="fft")) / np.linalg.norm(b) <= 1e-6, r
    plan.close()
