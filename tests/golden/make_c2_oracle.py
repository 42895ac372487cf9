"""Write tests/golden/c2_oracle.json and c2_maps.npz: the FP64 oracle's solves of the
full-size polarised workload (256 x 256 patch, 16 detectors x 2^20 samples, 256 uneven
intervals, lambda 4096; inputs from paper_1408_3048_gb300.synth.config(2)).

Recorded (all computed by oracle/ only):
  * iteration counts of block-Jacobi PCG and of two-level PCG (coarse space: 32 Ritz
    vectors of M_BD A from a block-Jacobi solve of b' = P^T N^-1 d_0 run to 1e-6, and
    the same from that solve run to 1e-10) at relative residual 1e-6, right-hand side
    b = P^T N^-1 d_1, and of block-Jacobi PCG to 1e-10;
  * the k smallest Ritz values;
  * the whole maps: m* (block-Jacobi PCG to 1e-10, float64) and the 1e-6 block-Jacobi and
    two-level maps (both coarse spaces) as float32 differences from m* (c2_maps.npz; a
    difference of relative size ~1e-5 keeps ~1e-12 of ||m|| in float32);
  * the error amplification kappa_b = ||M_BD||_2 ||b|| / (theta_1 ||m*||), theta_1 the
    smallest Ritz value of M_BD A from the 1e-10 run's Lanczos tridiagonal: a map whose
    true residual is rho ||b|| lies within about rho kappa_b ||m*|| of m*
    (||A^-1|| <= ||M_BD|| / lambda_min(M_BD A)), and the oracle's own maps' errors.

Realisation r uses the sky seed 1002 and the noise seed 2200 + r.  Run time: tens of
minutes on a few CPU cores (the oracle applies N^-1 by scipy FFT convolution).

    python tests/golden/make_c2_oracle.py [--scale S]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import precond  # noqa: E402
from oracle.pcg import pcg  # noqa: E402
from oracle.system import Problem  # noqa: E402
from paper_1408_3048_gb300 import synth  # noqa: E402


def smallest_ritz(res):
    """Smallest eigenvalue of the Lanczos tridiagonal of a PCG run (Sec. 3.3.2)."""
    m = len(res.alphas)
    T = precond.lanczos_tridiagonal(res.alphas, res.betas[: m - 1])
    return float(np.linalg.eigvalsh(T)[0])


def mbd_norm(bd):
    """||M_BD||_2: the largest eigenvalue over the per-pixel block inverses (Eq. 10)."""
    return float(np.linalg.eigvalsh(bd.inv).max())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=1)
    ap.add_argument("--k", type=int, default=32)
    here = os.path.dirname(os.path.abspath(__file__))
    ap.add_argument("--out", default=os.path.join(here, "c2_oracle.json"))
    ap.add_argument("--maps", default=os.path.join(here, "c2_maps.npz"))
    a = ap.parse_args()
    t0 = time.time()
    scan = synth.config(2, scale=a.scale)
    pr = Problem(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                 scan.fsamp, scan.lam, scan.ncomp)
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 1002)
    d = [synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp,
                                                      2200 + r)) for r in (0, 1)]

    def A(x):
        return pr.A(x, route="fft")

    b0 = pr.rhs(d[0], route="fft")
    b1 = pr.rhs(d[1], route="fft")
    bd = precond.BlockJacobi(pr)
    r0 = pcg(A, bd.apply, b0, 1e-6, 5000, record=True)
    Z, theta = precond.ritz_coarse_space(r0.alphas, r0.betas, r0.zs, r0.rzs, a.k)
    del r0
    tl = precond.TwoLevel(pr, bd, Z, route="fft")
    res_bd = pcg(A, bd.apply, b1, 1e-6, 5000)
    res_2l = pcg(A, tl.apply, b1, 1e-6, 5000)
    # the same construction from a first solve run to 1e-10: a longer Lanczos run whose
    # small Ritz pairs have converged (Sec. 3.3.2, App. A)
    r0 = pcg(A, bd.apply, b0, 1e-10, 5000, record=True)
    Z10, theta10 = precond.ritz_coarse_space(r0.alphas, r0.betas, r0.zs, r0.rzs, a.k)
    del r0
    res_2l10 = pcg(A, precond.TwoLevel(pr, bd, Z10, route="fft").apply, b1, 1e-6, 5000)
    del Z10
    res_star = pcg(A, bd.apply, b1, 1e-10, 5000)
    ms = res_star.x
    bn, mn = float(np.linalg.norm(b1)), float(np.linalg.norm(ms))
    th1 = smallest_ritz(res_star)
    mb = mbd_norm(bd)

    def rel(x):
        return float(np.linalg.norm(x - ms) / mn)

    def true_resid(x):
        return float(np.linalg.norm(b1 - A(x)) / bn)

    out = {
        "workload": f"synth.config(2, scale={a.scale})",
        "tol": 1e-6,
        "k": a.k,
        "n": int(pr.n),
        "npix_obs": int(pr.npix_obs),
        "b_norm": bn,
        "iters_bd": int(res_bd.iters),
        "iters_2lvl": int(res_2l.iters),
        "iters_bd_1e-10": int(res_star.iters),
        "k_kept": int(Z.shape[1]),
        "ritz": [float(v) for v in theta],
        "iters_2lvl_z1e-10": int(res_2l10.iters),
        "ritz_z1e-10": [float(v) for v in theta10],
        "m_bd_norm": float(np.linalg.norm(res_bd.x)),
        "m_2lvl_norm": float(np.linalg.norm(res_2l.x)),
        "m_star_norm": mn,
        "err_bd_vs_star": rel(res_bd.x),
        "err_2lvl_vs_star": rel(res_2l.x),
        "err_2lvl_z1e-10_vs_star": rel(res_2l10.x),
        "true_resid_bd": true_resid(res_bd.x),
        "true_resid_2lvl": true_resid(res_2l.x),
        "theta_1": th1,
        "mbd_norm": mb,
        "kappa_b": mb * bn / (th1 * mn),
        "seconds": time.time() - t0,
    }
    np.savez_compressed(a.maps, m_star=ms, d_bd=(res_bd.x - ms).astype(np.float32),
                        d_2lvl=(res_2l.x - ms).astype(np.float32),
                        d_2lvl_z1e10=(res_2l10.x - ms).astype(np.float32))
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
