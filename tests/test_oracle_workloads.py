"""The oracle on the workloads themselves (CPU): the 2^18-sample temperature raster at full
size and the polarised workload at 1/64 of its samples, against facts the paper fixes:
noiseless data give back the sky (the GLS estimate is unbiased, Eq. 3), white noise makes
M_BD the inverse of A and the map the hit-weighted binned map (Sec. 3.2), and the
two-level preconditioner needs fewer PCG iterations than block-Jacobi at 1e-6 under 1/f
noise (Sec. 5)."""
import copy

import numpy as np
import pytest

from oracle import precond
from oracle.pcg import pcg
from oracle.system import Problem
from paper_1408_3048_gb300 import synth


def _problem(scan):
    return Problem(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.fsamp, scan.lam, scan.ncomp)


WORKLOADS = {"T_2e18": lambda: synth.config(1), "IQU_2e24_over_64": lambda: synth.config(2, scale=64)}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def workload(request):
    scan = WORKLOADS[request.param]()
    return scan, _problem(scan)


def test_noiseless_data_give_back_the_sky(workload):
    scan, pr = workload
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 11)
    x_true = sky[pr.obs2sky].reshape(-1)
    d = synth.tod(scan, sky, np.zeros(scan.nt))
    res = pcg(lambda x: pr.A(x, route="fft"), precond.BlockJacobi(pr).apply, pr.rhs(d, route="fft"), 1e-10, 5000)
    assert res.converged
    assert np.linalg.norm(res.x - x_true) <= 1e-7 * np.linalg.norm(x_true)


def test_white_noise_map_is_the_binned_map(workload):
    scan = copy.copy(workload[0])       # same pointing and intervals, one white-noise PSD
    scan.psds = np.array([[1.3, 0.0, 1.0]])
    scan.interval_psd = np.zeros_like(scan.interval_psd)
    pr = _problem(scan)
    d = synth.tod(scan, synth.sky_map(scan.npix_sky, scan.ncomp, 12),
                  synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp, 3))
    res = pcg(lambda x: pr.A(x, route="fft"), precond.BlockJacobi(pr).apply, pr.rhs(d, route="fft"), 1e-12, 100)
    assert res.iters == 1
    nc = pr.ncomp
    if nc == 1:
        binned = np.bincount(pr.pix_c, weights=d, minlength=pr.npix_obs) / pr.hits
    else:
        kept = pr.pix_c >= 0
        W = np.stack([np.ones(scan.nt), scan.weights[:, 0], scan.weights[:, 1]], axis=1)[kept]
        q = pr.pix_c[kept]
        Bm = np.zeros((pr.npix_obs, 3, 3))
        np.add.at(Bm, q, W[:, :, None] * W[:, None, :])
        rhs = np.zeros((pr.npix_obs, 3))
        np.add.at(rhs, q, W * d[kept, None])
        binned = np.linalg.solve(Bm, rhs[:, :, None])[:, :, 0].reshape(-1)
    assert np.linalg.norm(res.x - binned) <= 1e-10 * np.linalg.norm(binned)


def test_two_level_beats_block_jacobi_under_one_over_f_noise(workload):
    scan, pr = workload
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 13)
    d0, d1 = (synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds,
                                                           scan.fsamp, s)) for s in (21, 22))
    A = lambda x: pr.A(x, route="fft")
    bd = precond.BlockJacobi(pr)
    first = pcg(A, bd.apply, pr.rhs(d0, route="fft"), 1e-6, 5000, record=True)
    Z, theta = precond.ritz_coarse_space(first.alphas, first.betas, first.zs, first.rzs, 8)
    assert theta[0] < 0.5            # 1/f noise leaves small eigenvalues in M_BD A (= I for white noise)
    b = pr.rhs(d1, route="fft")
    it_bd = pcg(A, bd.apply, b, 1e-6, 5000).iters
    it_2l = pcg(A, precond.TwoLevel(pr, bd, Z).apply, b, 1e-6, 5000).iters
    assert it_2l < it_bd, (it_2l, it_bd)
