"""Write tests/golden/c3_oracle.json: the FP64 oracle's solve of the large temperature
workload (512 x 512 patch, 1 detector, 2^27 samples, 2048 intervals of 2^16, lambda
1024; inputs from paper_1408_3048_gb300.synth.config(3), sky seed 1003, noise seed 2301).

Recorded (computed by oracle/ only): block-Jacobi PCG on b = P^T N^-1 d run to relative
residual 1e-10 (the reference map m*), the first iterations at which the residual is
below 1e-6 and 1e-8, ||b||, ||m*||, and m* at 4096 fixed indices.  The mixed-precision
GPU maps at tolerances 1e-6 and 1e-8 are compared with it.  Takes tens of minutes.

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
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_oracle.json"))
    a = ap.parse_args()
    t0 = time.time()
    scan = synth.config(3, scale=a.scale)
    pr = Problem(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                 scan.fsamp, scan.lam, scan.ncomp)
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 1003)
    d = synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp, 2301))
    b = pr.rhs(d, route="fft")
    res = pcg(lambda x: pr.A(x, route="fft"), precond.BlockJacobi(pr).apply, b, 1e-10, 5000)
    rel = np.asarray(res.rel_hist)
    idx = np.linspace(0, pr.n - 1, 4096).astype(np.int64)
    out = {
        "workload": f"synth.config(3, scale={a.scale})",
        "n": int(pr.n),
        "b_norm": float(np.linalg.norm(b)),
        "iters_1e-6": int(np.argmax(rel <= 1e-6)),
        "iters_1e-8": int(np.argmax(rel <= 1e-8)),
        "iters_1e-10": int(res.iters),
        "m_norm": float(np.linalg.norm(res.x)),
        "sample_index": idx.tolist(),
        "m_sample": res.x[idx].tolist(),
        "seconds": time.time() - t0,
    }
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if "sample" not in k}))


if __name__ == "__main__":
    main()
