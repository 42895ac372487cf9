#!/usr/bin/env python
"""Benchmark: GLS map-making time-to-solution on one GB300.

Workload (one "step" = one full map solve): the polarised I/Q/U raster scan of
paper_1408_3048_gb300.synth.config(2) -- 256 x 256 patch, 16 detectors x 2^20 = 2^24
samples, 256 stationary intervals of uneven length, per-detector 1/f noise
(f_knee in [0.1, 2] Hz, alpha in [1, 2]), Toeplitz half bandwidth lambda = 4096.

A step computes b = P^T N^-1 d and solves (P^T N^-1 P) m = b to relative residual 1e-6
with the two-level preconditioner (32 Ritz vectors of M_BD A from an FP64 block-Jacobi
solve of another noise realisation run to 1e-10, built once and reported separately) in
mixed precision (FP32 operators and PCG vectors, double-float dots, FP64 scalars and E,
refinement residual on FP64 data with a double-float band product).  The FP64 block-Jacobi
solve of the same data is timed beside it (``fp64_bj``).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the
same workload and extrapolates to a full solve (see "cpu_baseline" in the output).
N > 1 (torchrun): every rank solves its own noise realisation on its own GPU (replicas,
no collective on the data path); the time is the max over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TOL = 1e-6
K_COARSE = 32
# The Ritz pairs of the coarse space come from the Lanczos tridiagonal of a first
# block-Jacobi solve (Sec. 3.3.2); stopped at 1e-6 (44 steps) only the few smallest of the
# 32 requested pairs have converged and the two-level solve takes 43 inner iterations,
# run to 1e-10 in FP64 (92 steps) about twenty have and it takes 31.
COARSE_TOL = 1e-10
CONFIG = 2
GOLDEN = os.path.join(ROOT, "tests", "golden", "c2_oracle.json")
WORKLOAD = ("polarised I/Q/U raster, 256x256 patch, 16 detectors x 2^20 = 2^24 samples, 256 uneven "
            "intervals, 1/f noise fknee U[0.1,2] Hz alpha U[1,2], lambda=4096, tol 1e-6, two-level k=32 "
            "(Ritz vectors of M_BD A from an FP64 block-Jacobi solve of another realisation to 1e-10)")
METRIC = "time-to-solution @1e-6 resid (2-level mixed vs FP64 BJ, 1 GPU); A·x HBM GB/s"
ARITHMETIC = ("mixed solve: FP32 gather, Toeplitz N^-1, scatter and PCG vectors; CG dot products as "
              "double-float FP32 pairs (~48-bit significand, not FP64); FP64 step scalars and FP64 E^-1; "
              "iterative-refinement residual P^T N^-1 (d - P m) on FP64 data with the band product in "
              "double-float arithmetic (agrees with FP64 to 1e-12 of ||b||, tested)")
# bandwidth and knee-frequency cases of the secondary sweep (the paper's Sec. 5 studies)
SWEEP_CASES = [(1024, 1.0), (4096, 1.0), (16384, 1.0), (4096, 0.25), (4096, 4.0)]
BATCH_R = 64
L2_NOTE = "inputs larger than L2 (d 134 MB, pointing 335 MB)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary measurements after the timed region (coarse-space variants, "
                         "bandwidth / knee sweep, batched right-hand sides)")
    ap.add_argument("--sweep", action="store_true",
                    help="iteration counts of block-Jacobi and two-level PCG over Toeplitz bandwidths "
                         "and knee frequencies on the 2^24-sample workload (one JSON line per case; no "
                         "bench line)")
    ap.add_argument("--batched-forms", type=int, nargs="*", metavar="LAMBDA",
                    help="time one 64-column batched A X in each batched form (pair FFT, real FFT, "
                         "tensor cores) on the 2^24-sample scan at the given bandwidths; one JSON line each")
    ap.add_argument("--profile", action="store_true",
                    help="build, warm up, then run one step between cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off); prints a one-line JSON summary only")
    return ap.parse_args()


# ------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------- inputs
def make_inputs(realisations):
    from paper_1408_3048_gb300 import synth
    scan = synth.config(CONFIG)
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 1000 + CONFIG)
    ds = [synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp,
                                                       2000 + 100 * CONFIG + r)) for r in realisations]
    return scan, ds


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return j.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# -------------------------------------------------------------------- rooflines
# FP64: the recipe's nominal GB300 rate (an FMA-chain probe measured 1.253 TFLOP/s);
# FP32: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (the probe measured 78.3).
ALU_PEAK = {"f64": 1.25e12, "f32": 152 * 128 * 2 * 2.07e9}


def fft_tiles(scan, B, max_segments=3):
    """Overlap-save tiles of B-sample blocks as the plan lays them out: consecutive
    intervals with the same PSD are packed into one sequence with lambda zeros between
    them when that needs fewer tiles (and no tile holds more than `max_segments`
    intervals), else every interval is tiled on its own."""
    lam = int(scan.lam)
    Lv = B - 2 * lam
    lens = np.diff(np.asarray(scan.offsets, dtype=np.int64))
    psd = np.asarray(getattr(scan, "interval_psd", np.arange(lens.size)))
    total, i0 = 0, 0
    while i0 < lens.size:
        i1 = i0 + 1
        while i1 < lens.size and psd[i1] == psd[i0]:
            i1 += 1
        single = int(np.sum((lens[i0:i1] + Lv - 1) // Lv))
        starts = np.concatenate([[0], np.cumsum(lens[i0:i1] + lam)[:-1]])
        vlen = int(lens[i0:i1].sum() + (i1 - i0 - 1) * lam)
        packed = (vlen + Lv - 1) // Lv
        ok = True
        for k in range(packed):
            w0 = k * Lv - lam
            seg = np.sum((starts < w0 + B) & (starts + lens[i0:i1] > w0))
            if seg > max_segments:
                ok = False
                break
        total += packed if (i1 - i0 > 1 and ok and packed < single) else single
        i0 = i1
    return total


# Sources whose text fixes each profiled kernel: the DRAM traffic recorded from an ncu capture
# (a "traffic:" line in profiles/*.md) is reported only while their hash is unchanged.
KERNEL_SOURCES = {
    "toeplitz_f32": ["toeplitz.cuh", "toeplitz_f32.cu"],
    "toeplitz_f64": ["toeplitz.cuh", "toeplitz_f64.cu"],
    "toeplitz_df": ["toeplitz.cuh", "dfloat.cuh", "toeplitz_df.cu", "toeplitz_df_cluster.cu"],
    "scatter_f32": ["pointing.cu"],
    "scatter_f64": ["pointing.cu"],
    "pcg_f32": ["pcg.cu", "pcg.cuh"],
    "pcg_f64": ["pcg.cu", "pcg.cuh"],
}


def recorded_traffic(kernel):
    """(bytes per launch, profile file) from profiles/*.md, or (None, why)."""
    import glob
    import hashlib
    files = KERNEL_SOURCES.get(kernel)
    if not files:
        return None, "no source map"
    d = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1408_3048_gb300", "csrc", f), "rb") as fh:
            d.update(fh.read())
    cur = d.hexdigest()
    for md in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(md) as fh:
            for line in fh:
                parts = line.split()
                if len(parts) == 4 and parts[0] == "traffic:" and parts[1] == kernel:
                    kv = dict(x.split("=", 1) for x in parts[2:])
                    if kv.get("source_sha256") == cur:
                        return int(kv["dram_bytes_per_launch"]), os.path.relpath(md, ROOT)
                    return None, f"{os.path.relpath(md, ROOT)} predates the current kernel source"
    return None, "no ncu capture recorded"


def ax_bytes(plan, s):
    """Algorithmic bytes of one A x (Eq. 8) at s bytes per value: pointing (4 B index) and
    weights (2 s, I/Q/U) per sample, x read and y written (n s each).  Time-domain
    intermediates are excluded: a fully fused A x never writes them."""
    return plan.nt * (4 + (2 * s if plan.ncomp == 3 else 0)) + 2 * plan.n * s


def roofline(kernel, ms, plan, scan, hbm, peak_src):
    """Algorithmic bytes and flops of one launch of `kernel` over its measured duration;
    the bound is whichever of HBM or ALU the launch uses the larger fraction of.  The
    Toeplitz and scatter kernels are the two launches of one A x: each is charged the
    algorithmic bytes of the whole A x (the stage it belongs to), so their fractions are
    the fraction of the A x roofline they would reach if they were the whole A x."""
    nt, n = plan.nt, plan.n
    key = "f32" if kernel.endswith("f32") else "f64"
    s = 4 if key == "f32" else 8
    flops = None
    if kernel.startswith("toeplitz"):
        byts = ax_bytes(plan, s)
        B = plan.fft_block_f32 if key == "f32" else plan.fft_block_f64
        N = B // 2
        tiles = fft_tiles(scan, B)
        # two N-point complex FFTs (5 N log2 N each), real-FFT split/merge and spectrum
        # product (20 N), I/Q/U de-pointing (2 FMA per sample)
        flops = tiles * (2 * 5 * N * np.log2(N) + 20 * N) + (4 * nt if plan.ncomp == 3 else 0)
    elif kernel.startswith("scatter"):
        byts = ax_bytes(plan, s)
    else:
        byts = 8 * n * s
    t = ms * 1e-3
    gbs = byts / t / 1e9
    traffic, tsrc = recorded_traffic(kernel)
    out = {"bound": "hbm", "kernel": kernel, "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
           "frac": round(gbs / hbm, 4), "traffic": traffic, "traffic_source": tsrc,
           "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)", "bytes_per_launch": int(byts),
           "ms_per_launch": round(ms, 4)}
    if flops is not None:
        tf = flops / t / 1e12
        frac_alu = tf * 1e12 / ALU_PEAK[key]
        out["alu"] = {"achieved": round(tf, 3), "peak": ALU_PEAK[key] / 1e12, "unit": "TFLOP/s",
                      "frac": round(frac_alu, 4), "flops_per_launch": int(flops)}
        if frac_alu > out["frac"]:
            out = {"bound": "alu", "kernel": kernel, "achieved": round(tf, 3), "peak": ALU_PEAK[key] / 1e12,
                   "unit": "TFLOP/s", "frac": round(frac_alu, 4), "traffic": traffic, "traffic_source": tsrc,
                   "peak_source": ("recipe nominal GB300 FP64 rate" if key == "f64" else
                                   "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"),
                   "flops_per_launch": int(flops), "ms_per_launch": round(ms, 4),
                   "hbm": {"achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4),
                           "bytes_per_launch": int(byts)}}
    return out


# ------------------------------------------------------------------ CPU oracle
ORACLE_SNIPPET = r"""
import json, os, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from paper_1408_3048_gb300 import synth
from oracle.system import Problem
from oracle.precond import BlockJacobi
from oracle.pcg import pcg
steps, iters = {steps}, {iters}
scan = synth.config({cfg})
sky = synth.sky_map(scan.npix_sky, scan.ncomp, {sky_seed})
d = synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp, {noise_seed}))
t = time.perf_counter()
pr = Problem(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds, scan.fsamp,
             scan.lam, scan.ncomp)
bd = BlockJacobi(pr)
t_plan = time.perf_counter() - t
rng = np.random.default_rng(0)
Z = np.linalg.qr(rng.standard_normal((pr.n, {k})))[0]
AZ = rng.standard_normal((pr.n, {k}))
import scipy.linalg
lu = scipy.linalg.lu_factor(Z.T @ AZ + {k} * np.eye({k}))
A = lambda x: pr.A(x, route="fft")
def m2(r):
    v = scipy.linalg.lu_solve(lu, Z.T @ r)
    return bd.apply(r - AZ @ v) + Z @ v
out, samples = [], []
for s in range(steps):
    t0 = time.perf_counter()
    b = pr.rhs(d, route="fft")
    t1 = time.perf_counter()
    res = pcg(A, m2, b, 0.0, {sample_iters})
    t2 = time.perf_counter()
    per_it = (t2 - t1) / {sample_iters}
    out.append((t1 - t0) + iters * per_it)
    samples.append(t2 - t0)
print(json.dumps({{"values": out, "samples": samples, "t_plan": t_plan, "per_iter": per_it, "rhs": t1 - t0}}))
"""


# PCG iterations timed in the default run's CPU baseline (about 10 s of oracle work on the
# GPU machine's host cores; the reference arm's steps time two each)
CPU_SAMPLE_ITERS = 10


def oracle_time_to_solution(steps, iters, sample_iters=2):
    """Run the oracle, as it stands, in a fresh process on the host cores; each step times
    b = P^T N^-1 d and `sample_iters` two-level PCG iterations of the full workload and
    extrapolates to `iters` iterations.  Returns (extrapolated values, info)."""
    code = ORACLE_SNIPPET.format(root=ROOT, steps=steps, iters=iters, cfg=CONFIG, sky_seed=1000 + CONFIG,
                                 noise_seed=2000 + 100 * CONFIG + 1, k=K_COARSE, sample_iters=sample_iters)
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    j = json.loads(r.stdout.strip().splitlines()[-1])
    j["threads"] = os.cpu_count() or 1
    j["sample_iters"] = sample_iters
    j["sample_s"] = float(np.mean(j["samples"]))
    return j["values"], j


def oracle_iterations():
    """(two-level iteration count, its source, the golden record) of the oracle's own solve."""
    if os.path.exists(GOLDEN):
        with open(GOLDEN) as f:
            g = json.load(f)
        if "iters_2lvl_z1e-10" in g:   # the coarse space the bench builds (first solve to 1e-10)
            return (int(g["iters_2lvl_z1e-10"]), "oracle two-level PCG iteration count, coarse space from a "
                    "first solve to 1e-10 (tests/golden/c2_oracle.json)", g)
        return int(g["iters_2lvl"]), "oracle two-level PCG iteration count (tests/golden/c2_oracle.json)", g
    return None, None, None


GOLDEN_MAPS = os.path.join(ROOT, "tests", "golden", "c2_maps.npz")


def oracle_map():
    """The oracle's converged map m* (block-Jacobi PCG to 1e-10) of the bench's data, as
    written by tests/golden/make_c2_oracle.py (same scan, sky seed 1002, noise seed 2201),
    or None."""
    if not os.path.exists(GOLDEN_MAPS):
        return None
    with np.load(GOLDEN_MAPS) as z:
        return z["m_star"]


# ---------------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    """The reference arm: the FP64 oracle on the host cores.  Each of the W + K steps is a
    bounded sample of the workload (b plus two two-level PCG iterations); ms_per_step is
    the measured time of one such sample, `value` the time-to-solution it extrapolates to
    (the oracle's own two-level iteration count)."""
    if rank != 0:
        return
    iters, src, g = oracle_iterations()
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration count file missing"}))
        return
    vals, info = oracle_time_to_solution(a.warmup + a.steps, iters)
    v = float(np.mean(vals[a.warmup:]))
    sample_ms = float(np.mean(info["samples"][a.warmup:])) * 1e3
    line = {
        "impl": "reference", "metric": METRIC,
        "value": v, "unit": "s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": sample_ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "value_is": (f"time-to-solution extrapolated from each step's measured sample (b = P^T N^-1 d plus "
                     f"{info['sample_iters']} two-level PCG iterations, {sample_ms / 1e3:.2f} s) to {iters} "
                     f"iterations ({src}); ms_per_step is the sample's measured time"),
        "config": {"workload": WORKLOAD, "nt": 1 << 24, "n": int(g["n"]), "npix_obs": int(g["npix_obs"]),
                   "k_kept": int(g["k_kept"]), "l2": L2_NOTE, "parallelism": "one host process (FP64 oracle)"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": info["threads"], "kind": "oracle",
                         "sample": f"per step: b = P^T N^-1 d plus {info['sample_iters']} two-level PCG "
                                   f"iterations of the full workload (FP64 NumPy/SciPy; FFTs on one thread, BLAS "
                                   f"on {info['threads']}), extrapolated to {iters} iterations ({src})"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# -------------------------------------------------------------------- GPU arm
def replica_realisations(rank):
    """Noise realisations of one rank: 0 builds the coarse space, 1 + rank is solved (each
    replica solves its own realisation; no data crosses ranks)."""
    return [0, 1 + rank]


def max_over_ranks(x, world, device):
    """The largest value of x (float) over the ranks; the collective is timing only."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


class PlanInfo:
    """The plan figures the roofline needs, kept after the plan is closed."""

    def __init__(self, nt, n, ncomp, fft_block_f32, fft_block_f64):
        self.nt, self.n, self.ncomp = nt, n, ncomp
        self.fft_block_f32, self.fft_block_f64 = fft_block_f32, fft_block_f64


def coarse_variants(plan, b0, dc1, m):
    """The paper's other coarse spaces on the bench data (each replaces the previous one):
    the a priori Z_S merged into 32 interval groups (Sec. 3.3.1), the Arnoldi (Algorithm 1)
    and CG-Lanczos a posteriori spaces keeping the Ritz values below eps_tol = 0.2 (Sec. 5),
    and the A-DEF2 form (App. B) on the last one."""
    import torch
    from paper_1408_3048_gb300 import mm
    out = {}
    for name, build in (("apriori_r32", lambda: plan.build_coarse_apriori(K_COARSE)),
                        ("arnoldi_eps0.2", lambda: plan.build_coarse_arnoldi(
                            0.2, 64, bprime=b0, tol=TOL, maxit=400)[0]),
                        ("aposteriori_eps0.2", lambda: plan.build_coarse_eps(
                            0.2, 64, mm.MM_FP32, bprime=b0, tol=TOL, maxit=3000)[0])):
        torch.cuda.synchronize()
        t = time.perf_counter()
        try:
            kc = build()
        except mm.MMError as e:
            out[name] = {"error": str(e)}
            continue
        torch.cuda.synchronize()
        tb = time.perf_counter() - t
        _, s64, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_FP64, out=m)
        _, smx, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_MIXED, out=m)
        out[name] = {"k": kc, "build_s": round(tb, 4), "fp64_s": s64["ms_total"] / 1e3,
                     "fp64_iters": s64["iters"], "mixed_s": smx["ms_total"] / 1e3,
                     "mixed_iters": smx["iters"], "mixed_rel_resid": smx["rel_resid"]}
    if "error" not in out.get("aposteriori_eps0.2", {"error": 1}):
        _, s64, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_ADEF2, mm.MM_SOLVE_FP64, out=m)
        _, smx, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_ADEF2, mm.MM_SOLVE_MIXED, out=m)
        out["aposteriori_eps0.2_adef2"] = {
            "k": out["aposteriori_eps0.2"]["k"], "fp64_s": s64["ms_total"] / 1e3, "fp64_iters": s64["iters"],
            "mixed_s": smx["ms_total"] / 1e3, "mixed_iters": smx["iters"], "mixed_rel_resid": smx["rel_resid"]}
    return out


def run_ours(a, rank, world, local_rank):
    import torch
    from paper_1408_3048_gb300 import mm
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    scan, (d0, d1) = make_inputs(replica_realisations(rank))
    plan = mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.lam, scan.fsamp, stream=stream)
    pinfo = PlanInfo(plan.nt, plan.n, plan.ncomp, plan.fft_block_f32, plan.fft_block_f64)
    dc0 = torch.from_numpy(d0).to(dev)
    dc1 = torch.from_numpy(d1).to(dev)
    m = torch.empty(plan.n, dtype=torch.float64, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # coarse space (a posteriori, from realisation 0), built once and timed separately
    b0 = plan.rhs(dc0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    kk, ritz = plan.build_coarse(K_COARSE, mm.MM_FP64, bprime=b0, tol=COARSE_TOL, maxit=3000)
    torch.cuda.synchronize()
    t_coarse = time.perf_counter() - t

    def step():
        return plan.solve(dc1, TOL, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_MIXED, out=m)[1]

    if a.profile:
        for _ in range(max(1, a.warmup)):
            step()
        torch.cuda.synchronize()
        n0 = mm.mm_launch_count()
        torch.cuda.profiler.start()
        st = step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        if rank == 0:
            print(json.dumps({"profiled_step": st, "gpu_launches": mm.mm_launch_count() - n0}))
        plan.close()
        return

    # maps compared: the oracle's converged map of this data (rank 0's realisation) and a
    # converged FP64 GPU map (two-level, 1e-10)
    mstar = oracle_map() if rank == 0 else None
    mstar_t = torch.from_numpy(mstar).to(dev) if mstar is not None and mstar.size == plan.n else None
    _, st_ref, _ = plan.solve(dc1, 1e-10, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_FP64, out=m)
    m_conv = m.clone()

    def errs(x):
        e = {"vs_fp64_gpu_1e-10": float(torch.linalg.norm(x - m_conv) / torch.linalg.norm(m_conv))}
        if mstar_t is not None:
            e["vs_oracle_1e-10"] = float(torch.linalg.norm(x - mstar_t) / torch.linalg.norm(mstar_t))
        return e

    def solve_rec(tol, kind, solver):
        _, st_, _ = plan.solve(dc1, tol, 20000, kind, solver, out=m)
        rec = {"s": st_["ms_total"] / 1e3, "iters": st_["iters"], "rel_resid": st_["rel_resid"],
               "map_rel_err": errs(m)}
        if solver == mm.MM_SOLVE_MIXED:
            rec["outer"] = st_["outer"]
        return rec

    # FP64 block-Jacobi (the baseline of the metric), FP64 two-level, mixed block-Jacobi
    # (what the FP32 arithmetic alone gives), mixed two-level at the second tolerance;
    # one untimed solve of each form first (first launches load the kernels' modules)
    for kind in (mm.MM_PREC_BD, mm.MM_PREC_TWOLEVEL):
        for solver in (mm.MM_SOLVE_FP64, mm.MM_SOLVE_MIXED):
            plan.solve(dc1, TOL, 20000, kind, solver, out=m)
    fp64_bj = solve_rec(TOL, mm.MM_PREC_BD, mm.MM_SOLVE_FP64)
    fp64_2l = solve_rec(TOL, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_FP64)
    mixed_bj = solve_rec(TOL, mm.MM_PREC_BD, mm.MM_SOLVE_MIXED)
    mixed_2l_1e8 = solve_rec(1e-8, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_MIXED)

    for _ in range(a.warmup):
        step()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    n0 = mm.mm_launch_count()
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [step() for _ in range(a.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_total = e0.elapsed_time(e1)
    launches = (mm.mm_launch_count() - n0) // max(a.steps, 1)
    clk = clocks.stop()
    ms_step = max_over_ranks(ms_total, world, dev) / a.steps
    st = stats[-1]
    solve_errs = errs(m)

    # per-kernel profile of one more step (events around every launch)
    plan.profile(True)
    pst = step()
    prof = plan.profile_read()
    plan.profile(False)
    # launches that did work in that step: the PCG loop launches a few steps past
    # convergence (each exits at once on the done flag), counted but not averaged over
    work = {"toeplitz_f32": pst["iters"] + 1, "scatter_f32": pst["iters"] + 1, "pcg_f32": pst["iters"],
            "toeplitz_df": pst["outer"], "scatter_f64": pst["fp64_products"]}
    # A x alone, FP32 and FP64 (CUDA events, inputs already resident)
    x32 = torch.randn(plan.n, dtype=torch.float32, device=dev)
    x64 = x32.double()
    y32 = torch.empty_like(x32)
    y64 = torch.empty_like(x64)
    ax = {}
    for prec, x, y in ((mm.MM_FP32, x32, y32), (mm.MM_FP64, x64, y64)):
        for _ in range(3):
            plan.apply_A(x, prec, out=y)
        plan.profile(True)
        reps = 20 if prec == mm.MM_FP32 else 5
        for _ in range(reps):
            plan.apply_A(x, prec, out=y)
        p = plan.profile_read()
        plan.profile(False)
        key = "f32" if prec == mm.MM_FP32 else "f64"
        ax[key] = {"toeplitz_ms": p[f"toeplitz_{key}"][0] / reps, "scatter_ms": p[f"scatter_{key}"][0] / reps}

    # e2e through the C-ABI with host buffers (pinned d in, host m out)
    dh = torch.from_numpy(d1).pin_memory()
    mh = torch.empty(plan.n, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    barrier()
    t = time.perf_counter()
    for _ in range(a.steps):
        mm.mm_solve(plan.handle, dh, TOL, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_MIXED, mh)
    torch.cuda.synchronize()
    barrier()
    e2e_s = (time.perf_counter() - t) / a.steps

    extras = {}
    if not a.no_extras:
        extras["coarse_variants"] = coarse_variants(plan, b0, dc1, m)
        plan.close()
        plan = None
        del dc0, x32, x64, y32, y64
        torch.cuda.empty_cache()
        extras["sweep"] = run_sweep(cases=SWEEP_CASES, d_base=(d0, d1))
        extras["batched"] = run_batched(scan, dev)
    if plan is not None:
        plan.close()

    if rank != 0:
        return
    # roofline of the dominant kernel of the step
    hbm, peak_src = peaks()
    nt = pinfo.nt
    stages = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(stages, key=lambda k: stages[k][0])
    n_work = min(stages[dom][1], work.get(dom, stages[dom][1]))
    roof = roofline(dom, stages[dom][0] / max(n_work, 1), pinfo, scan, hbm, peak_src)
    roof["launches"] = {"in_step": stages[dom][1], "with_work": n_work,
                        "note": "ms_per_launch = the stage's total over the launches that did work"}
    # A x against the HBM roofline (algorithmic bytes of Eq. 8 over the two launches)
    ax_roof = {}
    for key, sz in (("f32", 4), ("f64", 8)):
        t_ax = (ax[key]["toeplitz_ms"] + ax[key]["scatter_ms"]) * 1e-3
        byts = ax_bytes(pinfo, sz)
        ax_roof[key] = {"achieved": round(byts / t_ax / 1e9, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(byts / t_ax / 1e9 / hbm, 4), "bytes": int(byts),
                        "ms": round(t_ax * 1e3, 4)}
    line = {
        "metric": METRIC,
        "value": ms_step / 1e3, "unit": "s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nt": nt, "n": pinfo.n, "npix_obs": pinfo.n // scan.ncomp,
                   "k_kept": kk, "fft_block_f64": pinfo.fft_block_f64, "fft_block_f32": pinfo.fft_block_f32,
                   "arithmetic": ARITHMETIC, "l2": L2_NOTE,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gpu_launches": int(launches),
        "solve": {"iters": st["iters"], "outer": st["outer"], "fp64_products": st["fp64_products"],
                  "rel_resid": st["rel_resid"], "map_rel_err": solve_errs},
        "fp64_bj": fp64_bj,
        "fp64_2lvl": fp64_2l,
        "mixed_bj": mixed_bj,
        "mixed_2lvl_tol1e-8": mixed_2l_1e8,
        "fp64_2lvl_tol1e-10": {"s": st_ref["ms_total"] / 1e3, "iters": st_ref["iters"],
                               "map_rel_err_vs_oracle_1e-10": errs(m_conv).get("vs_oracle_1e-10")},
        "speedup_vs_fp64_bj": fp64_bj["s"] / (ms_step / 1e3),
        "speedup_split": {"fp32_arithmetic": fp64_bj["s"] / mixed_bj["s"],
                          "two_level_given_fp32": mixed_bj["s"] / (ms_step / 1e3)},
        "coarse_build_s": t_coarse,
        "ax_roofline": ax_roof,
        "ax_ms": ax,
        "profile_ms": {k: [round(v[0], 4), v[1]] for k, v in stages.items()},
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(nt * 8), "d2h_bytes_per_step": int(pinfo.n * 8)},
    }
    line.update(extras)
    if world == 1 and not a.no_cpu_baseline:
        iters, src, _ = oracle_iterations()
        if iters is None:
            iters, src = fp64_2l["iters"], "FP64 two-level PCG iteration count of this run"
        try:
            vals, info = oracle_time_to_solution(1, iters, sample_iters=CPU_SAMPLE_ITERS)
            line["cpu_baseline"] = {"value": vals[0], "unit": "s", "cores": info["threads"], "kind": "oracle",
                                    "sample": f"b = P^T N^-1 d plus {info['sample_iters']} two-level PCG iterations "
                                              f"of the full workload (FP64 NumPy/SciPy; FFTs on one thread, BLAS on "
                                              f"{info['threads']}; coarse space of k = {K_COARSE} random orthonormal "
                                              f"columns, as costly per iteration as the Ritz space), measured "
                                              f"{info['sample_s']:.1f} s, scaled to {iters} iterations ({src}); "
                                              f"plan time {info['t_plan']:.1f} s excluded"}
        except Exception as ex:  # the GPU number stands; say why the baseline is missing
            line["cpu_baseline"] = {"value": None, "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {str(ex)[:200]}"}
    print(json.dumps(line))


def run_sweep(cases=None, d_base=None, emit=False):
    """Bandwidth and knee-frequency sweeps (the paper's Sec. 5 studies of lambda_T and
    f_knee, on the synthetic 2^24-sample polarised scan): iterations and times to 1e-6 of
    FP64 block-Jacobi, mixed block-Jacobi, two-level a priori (Z_S, 32 interval groups)
    and two-level a posteriori (Ritz values below eps_tol = 0.2) PCG.  Cases at the
    workload's own knee frequencies reuse the bench's two realisations (d_base); scaled
    knees draw new ones (seeds 2200, 2201).  Returns the records (emit: also one JSON
    line each)."""
    import torch
    from paper_1408_3048_gb300 import mm, synth
    base = synth.config(CONFIG)
    sky = synth.sky_map(base.npix_sky, base.ncomp, 1000 + CONFIG)
    if cases is None:
        cases = [(lam, 1.0) for lam in (1024, 2048, 4096, 8192, 16384)] + [(4096, f) for f in (0.25, 4.0)]
    recs = []
    for lam, fk in cases:
        psds = np.array(base.psds, dtype=np.float64).reshape(-1, 3).copy()
        psds[:, 1] *= fk
        scan = synth.config(CONFIG)
        scan.lam = lam
        scan.psds = psds
        if fk == 1.0 and d_base is not None:
            d0, d1 = d_base
        else:
            d0, d1 = (synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, psds, scan.fsamp,
                                                                   2200 + r)) for r in (0, 1))
        plan = mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, psds, lam, scan.fsamp)
        dc0, dc1 = torch.from_numpy(d0).cuda(), torch.from_numpy(d1).cuda()
        m = torch.empty(plan.n, dtype=torch.float64, device="cuda")
        out = {"lambda": lam, "fknee_scale": fk}
        if plan.fft_block_f64:
            _, st, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_BD, mm.MM_SOLVE_FP64, out=m)
            out["bd_fp64"] = {"iters": st["iters"], "s": st["ms_total"] / 1e3}
        _, st, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_BD, mm.MM_SOLVE_MIXED, out=m)
        out["bd_mixed"] = {"iters": st["iters"], "s": st["ms_total"] / 1e3}
        b0 = plan.rhs(dc0)
        for name, build in (("apriori_r32", lambda: plan.build_coarse_apriori(K_COARSE)),
                            ("aposteriori_eps0.2", lambda: plan.build_coarse_eps(
                                0.2, 64, mm.MM_FP32, bprime=b0, tol=TOL, maxit=5000)[0])):
            try:
                k = build()
            except mm.MMError as e:
                out[name] = {"error": str(e)}
                continue
            rec = {"k": k}
            if plan.fft_block_f64:
                _, st, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_FP64, out=m)
                rec["fp64"] = {"iters": st["iters"], "s": st["ms_total"] / 1e3}
            _, st, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_MIXED, out=m)
            rec["mixed"] = {"iters": st["iters"], "s": st["ms_total"] / 1e3, "rel_resid": st["rel_resid"]}
            out[name] = rec
        if emit:
            print(json.dumps(out), flush=True)
        recs.append(out)
        plan.close()
        del dc0, dc1, m
        torch.cuda.empty_cache()
    return recs


def run_batched(scan, dev, lams=(1024, 4096, 16384), R=BATCH_R, nbase=4):
    """Many right-hand sides through one plan (the batched Monte-Carlo workload): R noise
    realisations of the bench scan solved together to 1e-6 (mixed precision, block-Jacobi,
    per-column refinement) at each bandwidth.  The R noise vectors are unit-norm random
    combinations (seed 2400) of `nbase` seeded realisations (seeds 2400..): a unit-norm
    combination of independent realisations of one Gaussian noise is again a realisation
    of it, and drawing R full realisations on the host would take minutes.  Reports the
    time per map, the batched operator's form, and one A X per column."""
    import torch
    from paper_1408_3048_gb300 import mm, synth
    sky = synth.sky_map(scan.npix_sky, scan.ncomp, 1000 + CONFIG)
    signal = torch.from_numpy(synth.tod(scan, sky, np.zeros(scan.nt))).to(dev)
    base = torch.stack([torch.from_numpy(synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds,
                                                                 scan.fsamp, 2400 + j)).to(dev)
                        for j in range(nbase)])
    C = np.random.default_rng(2400).standard_normal((R, nbase))
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    D = signal[None, :] + torch.from_numpy(C).to(dev) @ base
    del base
    out = {"R": R, "tol": TOL, "noise": f"unit-norm combinations of {nbase} realisations (seeds 2400..)",
           "forms": "the plan autotunes: one batched A X timed per form (0 pair FFT, 1 real FFT, 2 tensor-core "
                    "band product), the fastest kept"}
    for lam in lams:
        sc = synth.config(CONFIG)
        sc.lam = lam
        plan = mm.Plan(sc.pix, sc.npix_sky, sc.weights, sc.offsets, sc.interval_psd, sc.psds, lam, sc.fsamp,
                       autotune=True)
        kind, logb, tm = plan.batch_config(R)
        M = torch.empty((R, plan.n), dtype=torch.float64, device=dev)
        plan.solve_batch(D, tol=TOL, maxit=5000, out=M)     # warm-up (graph capture)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, st, status = plan.solve_batch(D, tol=TOL, maxit=5000, out=M)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t
        X = torch.randn((R, plan.n), dtype=torch.float32, device=dev)
        Y = torch.empty_like(X)
        plan.apply_A_batch(X, out=Y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            plan.apply_A_batch(X, out=Y)
        e1.record()
        torch.cuda.synchronize()
        ax_ms = e0.elapsed_time(e1) / 3
        out[f"lambda_{lam}"] = {"s_per_map": ts / R, "s_total": ts, "status": int(status),
                                "converged": int(sum(x["converged"] for x in st)),
                                "iters_max": int(max(x["iters"] for x in st)),
                                "form": ["pair", "real", "tensor"][kind], "log2_block": int(logb),
                                "form_ax_ms": {"pair": round(tm[0], 3), "real": round(tm[1], 3),
                                               "tensor": round(tm[2], 3)},
                                "ax_batch_ms_per_column": ax_ms / R}
        plan.close()
        del M, X, Y
        torch.cuda.empty_cache()
    return out


def run_batched_forms(lams, R=BATCH_R):
    """One batched A X (R columns) timed in each batched form, CUDA events, 3 calls after
    2 warm-up calls, on the bench scan at each bandwidth."""
    import torch
    from paper_1408_3048_gb300 import mm, synth
    for lam in lams:
        sc = synth.config(CONFIG)
        sc.lam = lam
        rec = {"lambda": lam, "R": R}
        for kind, name in ((0, "pair"), (1, "real"), (2, "tensor")):
            plan = mm.Plan(sc.pix, sc.npix_sky, sc.weights, sc.offsets, sc.interval_psd, sc.psds, lam, sc.fsamp)
            plan.batch_config(R, kind)
            X = torch.randn(R, plan.n, dtype=torch.float32, device="cuda")
            Y = torch.empty_like(X)
            for _ in range(2):
                plan.apply_A_batch(X, out=Y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                plan.apply_A_batch(X, out=Y)
            e1.record()
            torch.cuda.synchronize()
            rec[f"{name}_ms"] = e0.elapsed_time(e1) / 3
            plan.close()
            del X, Y
            torch.cuda.empty_cache()
        print(json.dumps(rec), flush=True)


def main():
    a = parse()
    if a.sweep:
        run_sweep(emit=True)
        return
    if a.batched_forms:
        run_batched_forms(a.batched_forms)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_ours(a, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
