"""Write tests/golden/c3_oracle.json and c3_map.npz: the FP64 oracle's solve of the large
temperature workload (512 x 512 patch, 1 detector, 2^27 samples, 2048 intervals of 2^16,
lambda 1024; inputs from paper_1408_3048_gb300.synth.config(3), sky seed 1003, noise seed
2301).

Recorded (computed by oracle/ only): block-Jacobi PCG on b = P^T N^-1 d run to relative
residual 1e-10 (the reference map m*, stored whole as float64 in c3_map.npz), the first
iterations at which the residual is below 1e-6 and 1e-8, ||b||, ||m*||, and the error
amplification kappa_b = ||M_BD||_2 ||b|| / (theta_1 ||m*||) with theta_1 the smallest
Ritz value of M_BD A from that run's Lanczos tridiagonal (Sec. 3.3.2): a map whose true
residual is rho ||b|| lies within about rho kappa_b ||m*|| of m*.  The mixed-precision
GPU maps at tolerances 1e-6 and 1e-8 are compared with m*.  Takes tens of minutes.

    python tests/golden/make_c3_oracle.py [--scale S]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=1)
    here = os.path.dirname(os.path.abspath(__file__))
    ap.add_argument("--out", default=os.path.join(here, "c3_oracle.json"))
    ap.add_argument("--maps", default=os.path.join(here, "c3_map.npz"))
    a = ap.parse_args()
    t0 = time.time()
    scan = synth.config(3, scale=a.scale)
    pr = Problem(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                 scan.fsamp, scan.lam, scan.ncomp)
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 1003)
    d = synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp, 2301))
    b = pr.rhs(d, route="fft")
    bd = precond.BlockJacobi(pr)
    res = pcg(lambda x: pr.A(x, route="fft"), bd.apply, b, 1e-10, 5000)
    rel = np.asarray(res.rel_hist)
    m = len(res.alphas)
    th1 = float(np.linalg.eigvalsh(precond.lanczos_tridiagonal(res.alphas, res.betas[: m - 1]))[0])
    mb = float(bd.inv.max()) if pr.ncomp == 1 else float(np.linalg.eigvalsh(bd.inv).max())
    bn, mn = float(np.linalg.norm(b)), float(np.linalg.norm(res.x))
    out = {
        "workload": f"synth.config(3, scale={a.scale})",
        "n": int(pr.n),
        "b_norm": bn,
        "iters_1e-6": int(np.argmax(rel <= 1e-6)),
        "iters_1e-8": int(np.argmax(rel <= 1e-8)),
        "iters_1e-10": int(res.iters),
        "m_norm": mn,
        "theta_1": th1,
        "mbd_norm": mb,
        "kappa_b": mb * bn / (th1 * mn),
        "seconds": time.time() - t0,
    }
    np.savez_compressed(a.maps, m_star=res.x)
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
