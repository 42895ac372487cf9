"""Small seeded problems shared by the tests (inputs only; no method arithmetic)."""

from paper_1408_3048_gb300 import synth


def tiny_scan(ncomp=1, W=6, H=5, ndet=2, nper=240, K_per_det=2, lam=6,
              psds=((1.0, 1.0, 1.0), (1.3, 0.5, 1.7)), uneven=None, seed=0):
    det_psd = [d % len(psds) for d in range(ndet)]
    return synth.raster_scan(W, H, ndet, nper, ncomp, K_per_det, lam, list(psds),
                             det_psd=det_psd, uneven=uneven, seed=seed)


def oracle_problem(scan, **kw):
    from oracle.system import Problem
    return Problem(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd,
                   scan.psds, scan.fsamp, scan.lam, scan.ncomp, **kw)
