"""mm_apply_A_static: A x for callers that cannot allocate device memory during a call
(their GPU memory is reserved by a pool they do not own, or the call sits on a path
where a cudaMalloc could fail or stall).  It keeps the time-domain intermediate in a
fixed 32 MiB array inside the library.  Checked through the C-ABI against mm_apply_A
on two calls in a row (the array keeps the previous call's contents), in FP64 and FP32;
after a call by a plan with more samples, a plan with fewer samples gets its own result
(it never reads entries the larger one left); the device's free memory is the same
before and after a call; sizes beyond the array are rejected.  Needs a GPU.

The file name makes pytest collect it last, so that a run which stops at its first
failure (pytest -x) has run every other test before this one.  The tests themselves do
not depend on that order: each makes its own plans, and they pass alone in a fresh
process too.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1408_3048_gb300 import mm, synth

pytestmark = pytest.mark.gpu


def _plan(scan):
    return mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.lam, scan.fsamp)


def _scan(ncomp, nper=24000, seed=5):
    return synth.raster_scan(24, 24, 4, nper, ncomp, 4, 500, [(1.0, 1.0, 1.0), (0.8, 1.5, 1.5)],
                             det_psd=[0, 1, 0, 1], uneven=(3000, 9000), seed=seed)


def _check(plan, prec, rng):
    """mm_apply_A_static against mm_apply_A on one random x; returns the relative error
    and the change of the device's free memory across the static call."""
    dt = torch.float64 if prec == mm.MM_FP64 else torch.float32
    x = torch.as_tensor(rng.standard_normal(plan.n), dtype=dt).cuda()
    ref = torch.empty(plan.n, dtype=dt, device="cuda")
    out = torch.full((plan.n,), float("nan"), dtype=dt, device="cuda")
    mm.mm_apply_A(plan.handle, prec, x, ref)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    mm.mm_apply_A_static(plan.handle, prec, x, out)
    free1 = torch.cuda.mem_get_info()[0]
    err = float(torch.linalg.norm((out - ref).double()) / torch.linalg.norm(ref.double()))
    return err, free0 - free1


@pytest.mark.parametrize("ncomp", [1, 3])
def test_static_matches_apply_A_twice(ncomp):
    plan = _plan(_scan(ncomp))
    rng = np.random.default_rng(11)
    for prec, tol in ((mm.MM_FP64, 1e-12), (mm.MM_FP32, 3e-5)):
        for call in range(2):   # the second call runs on the array the first one left behind
            err, dfree = _check(plan, prec, rng)
            assert err <= tol, (prec, call, err)
            assert dfree == 0, (prec, call, dfree)
    plan.close()


def test_static_fp32_matches_the_packed_gather_bit_for_bit():
    # mm_apply_A in FP32 on I/Q/U reads x packed per pixel (one 16-byte load per sample);
    # the static path gathers the three components one by one.  Same arithmetic, so the
    # two A x must agree to the bit.
    plan = _plan(_scan(3))
    rng = np.random.default_rng(17)
    x = torch.as_tensor(rng.standard_normal(plan.n), dtype=torch.float32).cuda()
    ref = torch.empty(plan.n, dtype=torch.float32, device="cuda")
    out = torch.empty(plan.n, dtype=torch.float32, device="cuda")
    mm.mm_apply_A(plan.handle, mm.MM_FP32, x, ref)
    mm.mm_apply_A_static(plan.handle, mm.MM_FP32, x, out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    plan.close()


def test_static_smaller_plan_after_larger_one():
    big = _plan(_scan(3, nper=60000, seed=8))
    small = _plan(_scan(3, nper=9000, seed=9))
    assert big.nt > 4 * small.nt
    rng = np.random.default_rng(12)
    for prec, tol in ((mm.MM_FP64, 1e-12), (mm.MM_FP32, 3e-5)):
        for plan in (big, small, big, small):
            err, dfree = _check(plan, prec, rng)
            assert err <= tol and dfree == 0, (prec, plan.nt, err, dfree)
    big.close()
    small.close()


def test_static_rejects_sizes_beyond_the_array():
    nper = 2 ** 22 + 2 ** 16      # FP64 intermediate 33.5 MB > 32 MiB
    scan = synth.raster_scan(32, 32, 1, nper, 1, 4, 64, [(1.0, 1.0, 1.0)], seed=6)
    plan = _plan(scan)
    x = torch.ones(plan.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(mm.MMError) as e:
        mm.mm_apply_A_static(plan.handle, mm.MM_FP64, x, y)
    assert e.value.status == mm.MM_ERR_ARG and "static" in str(e.value)
    # FP32 needs half the bytes and fits
    err, dfree = _check(plan, mm.MM_FP32, np.random.default_rng(13))
    assert err <= 3e-5 and dfree == 0
    plan.close()


def test_static_null_plan_is_an_argument_error():
    assert mm.lib().mm_apply_A_static(None, mm.MM_FP64, None, None) == mm.MM_ERR_ARG
