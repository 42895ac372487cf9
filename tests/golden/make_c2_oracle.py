"""Write tests/golden/c2_oracle.json: the FP64 oracle's solves of the full-size polarised
workload (256 x 256 patch, 16 detectors x 2^20 samples, 256 uneven intervals, lambda
4096; inputs from paper_1408_3048_gb300.synth.config(2)).

Recorded (all computed by oracle/ only):
  * iteration counts of block-Jacobi PCG and of two-level PCG (coarse space: 32 Ritz
    vectors of M_BD A from a block-Jacobi solve of b' = P^T N^-1 d_0) at relative
    residual 1e-6, right-hand side b = P^T N^-1 d_1;
  * the k smallest Ritz values;
  * ||b||, ||m||, and the map values at 256 fixed sample indices of each solution.

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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=1)
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle.json"))
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
    idx = np.linspace(0, pr.n - 1, 256).astype(np.int64)
    out = {
        "workload": f"synth.config(2, scale={a.scale})",
        "tol": 1e-6,
        "k": a.k,
        "n": int(pr.n),
        "npix_obs": int(pr.npix_obs),
        "b_norm": float(np.linalg.norm(b1)),
        "iters_bd": int(res_bd.iters),
        "iters_2lvl": int(res_2l.iters),
        "k_kept": int(Z.shape[1]),
        "ritz": [float(v) for v in theta],
        "m_bd_norm": float(np.linalg.norm(res_bd.x)),
        "m_2lvl_norm": float(np.linalg.norm(res_2l.x)),
        "sample_index": idx.tolist(),
        "m_bd_sample": res_bd.x[idx].tolist(),
        "m_2lvl_sample": res_2l.x[idx].tolist(),
        "seconds": time.time() - t0,
    }
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if "sample" not in k}))


if __name__ == "__main__":
    main()
