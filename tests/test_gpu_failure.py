"""Failure detection on the GPU without a GPU fault -- needs a GPU.

Every grid-barrier wait of the persistent PCG kernels is bounded in time.  The
diagnostic mm_pcg_barrier_check runs the solver's own start kernel with a barrier that
waits for blocks that are never launched (a flag nothing sets) and a 10 ms limit: the
wait runs out, the kernel records MM_ERR_TIMEOUT and returns, the host reads the status,
and the context and the plan stay usable -- a normal solve afterwards matches the oracle.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import precond as oprec
from oracle.pcg import pcg
from paper_1408_3048_gb300 import mm, synth
from problems import oracle_problem, tiny_scan

pytestmark = pytest.mark.gpu


def _plan(scan):
    return mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.lam, scan.fsamp)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_barrier_wait_runs_out_and_plan_stays_usable(ncomp):
    scan = tiny_scan(ncomp=ncomp, nper=2000, lam=40)
    pr = oracle_problem(scan)
    plan = _plan(scan)
    assert plan.barrier_check(0, 1.0) == mm.MM_OK
    t0 = time.perf_counter()
    status = plan.barrier_check(1, 0.01)
    dt = time.perf_counter() - t0
    assert status == mm.MM_ERR_TIMEOUT
    assert "barrier" in mm.mm_last_error(plan.handle)
    assert dt < 5.0
    # twice in a row: the counter left by the first timeout is zeroed before the next run
    assert plan.barrier_check(3, 0.01) == mm.MM_ERR_TIMEOUT
    assert plan.barrier_check(0, 1.0) == mm.MM_OK
    # the plan solves normally afterwards (FP64 block-Jacobi, then two-level mixed)
    sky = synth.sky_map(scan.npix_sky, ncomp, 1)
    d = synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp, 3))
    dc = torch.from_numpy(d).cuda()
    m, st, s1 = plan.solve(dc, tol=1e-8, maxit=500)
    ref = pcg(pr.A, oprec.BlockJacobi(pr).apply, pr.rhs(d), 1e-8, 500)
    assert s1 == mm.MM_OK and abs(st["iters"] - ref.iters) <= 2
    assert np.linalg.norm(m.cpu().numpy() - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
    # and a timeout in between two-level solves leaves them working too
    plan.build_coarse(4, mm.MM_FP64, bprime=plan.rhs(dc), tol=1e-6, maxit=500)
    assert plan.barrier_check(2, 0.01) == mm.MM_ERR_TIMEOUT
    m2, st2, s2 = plan.solve(dc, tol=1e-6, maxit=500, kind=mm.MM_PREC_TWOLEVEL, solver=mm.MM_SOLVE_MIXED)
    b = pr.rhs(d)
    assert s2 == mm.MM_OK
    assert np.linalg.norm(b - pr.A(m2.cpu().numpy())) <= 1e-6 * np.linalg.norm(b)
    plan.close()


def test_barrier_check_rejects_bad_arguments():
    plan = _plan(tiny_scan(ncomp=1))
    for absent, wait in ((-1, 0.01), (2000, 0.01), (0, 0.0), (0, 11.0)):
        assert plan.barrier_check(absent, wait) == mm.MM_ERR_ARG
    plan.close()
