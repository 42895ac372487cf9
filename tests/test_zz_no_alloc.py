"""mm_apply_A_static: A x for callers that cannot allocate device memory during a call
(their GPU memory is reserved by a pool they do not own, or the call sits on a path
where a cudaMalloc could fail or stall).  It keeps the time-domain intermediate in a
fixed 32 MiB array inside the library.  Checked through the C-ABI against mm_apply_A
on two calls in a row (the array keeps the previous call's contents), in FP64 and FP32,
plus the size limit.  Needs a GPU; this file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1408_3048_gb300 import mm, synth

pytestmark = pytest.mark.gpu


def _plan(scan):
    return mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.lam, scan.fsamp)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_static_matches_apply_A_twice(ncomp):
    scan = synth.raster_scan(24, 24, 4, 24000, ncomp, 4, 500, [(1.0, 1.0, 1.0), (0.8, 1.5, 1.5)],
                             det_psd=[0, 1, 0, 1], uneven=(3000, 9000), seed=5)
    plan = _plan(scan)
    rng = np.random.default_rng(11)
    for prec, dt, tol in ((mm.MM_FP64, torch.float64, 1e-12), (mm.MM_FP32, torch.float32, 3e-5)):
        for call in range(2):   # second call runs on the array the first one left behind
            x = torch.as_tensor(rng.standard_normal(plan.n), dtype=dt).cuda()
            ref = torch.empty(plan.n, dtype=dt, device="cuda")
            out = torch.full((plan.n,), float("nan"), dtype=dt, device="cuda")
            mm.mm_apply_A(plan.handle, prec, x, ref)
            mm.mm_apply_A_static(plan.handle, prec, x, out)
            err = float(torch.linalg.norm((out - ref).double()) / torch.linalg.norm(ref.double()))
            assert err <= tol, (prec, call, err)
    plan.close()


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
    x32 = torch.ones(plan.n, dtype=torch.float32, device="cuda")
    ref = torch.empty_like(x32)
    out = torch.empty_like(x32)
    mm.mm_apply_A(plan.handle, mm.MM_FP32, x32, ref)
    mm.mm_apply_A_static(plan.handle, mm.MM_FP32, x32, out)
    assert float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref)) <= 3e-5
    plan.close()
