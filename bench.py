#!/usr/bin/env python
"""Benchmark: GLS map-making time-to-solution on one GB300.

Workload (one "step" = one full map solve): the polarised I/Q/U raster scan of
paper_1408_3048_gb300.synth.config(2) -- 256 x 256 patch, 16 detectors x 2^20 = 2^24
samples, 256 stationary intervals of uneven length, per-detector 1/f noise
(f_knee in [0.1, 2] Hz, alpha in [1, 2]), Toeplitz half bandwidth lambda = 4096.

A step computes b = P^T N^-1 d and solves (P^T N^-1 P) m = b to relative residual 1e-6
with the two-level preconditioner (32 Ritz vectors of M_BD A, built once from another
noise realisation and reported separately) in mixed precision (FP32 operators inside
PCG, FP64 dots, E factor and iterative-refinement residual).  The FP64 block-Jacobi
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
CONFIG = 2
GOLDEN = os.path.join(ROOT, "tests", "golden", "c2_oracle.json")
WORKLOAD = ("polarised I/Q/U raster, 256x256 patch, 16 detectors x 2^20 = 2^24 samples, 256 uneven "
            "intervals, 1/f noise fknee U[0.1,2] Hz alpha U[1,2], lambda=4096, tol 1e-6, two-level k=32")
METRIC = "time-to-solution @1e-6 resid (2-level mixed vs FP64 BJ, 1 GPU); A·x HBM GB/s"
L2_NOTE = "inputs larger than L2 (d 134 MB, pointing 335 MB)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="iteration counts of block-Jacobi and two-level PCG over Toeplitz bandwidths "
                         "and knee frequencies on the 2^24-sample workload (one JSON line per case; no "
                         "bench line)")
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


def fft_tiles(scan, B):
    Lv = B - 2 * scan.lam
    lens = np.diff(scan.offsets)
    return int(np.sum((lens + Lv - 1) // Lv))


# Sources whose text fixes each profiled kernel: the DRAM traffic recorded from an ncu capture
# (a "traffic:" line in profiles/*.md) is reported only while their hash is unchanged.
KERNEL_SOURCES = {
    "toeplitz_f32": ["toeplitz.cuh", "toeplitz_f32.cu"],
    "toeplitz_f64": ["toeplitz.cuh", "toeplitz_f64.cu"],
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


def roofline(kernel, ms, plan, scan, hbm, peak_src):
    """Algorithmic bytes and flops of one launch of `kernel` over its measured duration;
    the bound is whichever of HBM or ALU the launch uses the larger fraction of."""
    nt, n = plan.nt, plan.n
    key = "f32" if kernel.endswith("f32") else "f64"
    s = 4 if key == "f32" else 8
    w = 2 * s if plan.ncomp == 3 else 0
    flops = None
    if kernel.startswith("toeplitz"):
        # pointing (4 B) + weights read, time-domain output written per sample; map read
        byts = nt * (4 + w + s) + n * s
        B = plan.fft_block_f32 if key == "f32" else plan.fft_block_f64
        N = B // 2
        tiles = fft_tiles(scan, B)
        # two N-point complex FFTs (5 N log2 N each), real-FFT split/merge and spectrum
        # product (20 N), I/Q/U de-pointing (2 FMA per sample)
        flops = tiles * (2 * 5 * N * np.log2(N) + 20 * N) + (4 * nt if plan.ncomp == 3 else 0)
    elif kernel.startswith("scatter"):
        byts = nt * (4 + w + s) + n * s
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
out = []
for s in range(steps):
    t0 = time.perf_counter()
    b = pr.rhs(d, route="fft")
    t1 = time.perf_counter()
    res = pcg(A, m2, b, 0.0, {sample_iters})
    t2 = time.perf_counter()
    per_it = (t2 - t1) / {sample_iters}
    out.append((t1 - t0) + iters * per_it)
print(json.dumps({{"values": out, "t_plan": t_plan, "per_iter": per_it, "rhs": t1 - t0}}))
"""


def oracle_time_to_solution(steps, iters, sample_iters=2):
    """Run the oracle in a fresh single-threaded process; return (values, info)."""
    code = ORACLE_SNIPPET.format(root=ROOT, steps=steps, iters=iters, cfg=CONFIG, sky_seed=1000 + CONFIG,
                                 noise_seed=2000 + 100 * CONFIG + 1, k=K_COARSE, sample_iters=sample_iters)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    j = json.loads(r.stdout.strip().splitlines()[-1])
    return j["values"], j


def oracle_iterations():
    """(two-level iteration count, its source, the golden record) of the oracle's own solve."""
    if os.path.exists(GOLDEN):
        with open(GOLDEN) as f:
            g = json.load(f)
        return int(g["iters_2lvl"]), "oracle two-level PCG iteration count (tests/golden/c2_oracle.json)", g
    return None, None, None


# ---------------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    if rank != 0:
        return
    iters, src, g = oracle_iterations()
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration count file missing"}))
        return
    vals, info = oracle_time_to_solution(a.warmup + a.steps, iters)
    v = float(np.mean(vals[a.warmup:]))
    line = {
        "impl": "reference", "metric": METRIC,
        "value": v, "unit": "s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nt": 1 << 24, "n": int(g["n"]), "npix_obs": int(g["npix_obs"]),
                   "k_kept": int(g["k_kept"]), "l2": L2_NOTE, "parallelism": "one host process (FP64 oracle)"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: b = P^T N^-1 d plus 2 two-level PCG iterations of the full "
                                   f"workload, extrapolated to {iters} iterations ({src})"},
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


def run_ours(a, rank, world, local_rank):
    import torch
    from paper_1408_3048_gb300 import mm
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    scan, (d0, d1) = make_inputs(replica_realisations(rank))
    plan = mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, scan.psds,
                   scan.lam, scan.fsamp, stream=stream)
    dc0 = torch.from_numpy(d0).to(dev)
    dc1 = torch.from_numpy(d1).to(dev)
    m = torch.empty(plan.n, dtype=torch.float64, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # coarse space (a posteriori, from realisation 0), timed separately
    b0 = plan.rhs(dc0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    kk, ritz = plan.build_coarse(K_COARSE, mm.MM_FP32, bprime=b0, tol=TOL, maxit=3000)
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

    # FP64 block-Jacobi and FP64 two-level references (one solve each)
    _, st_bj, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_BD, mm.MM_SOLVE_FP64, out=m)
    _, st_2f, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_FP64, out=m)
    m_ref64 = m.clone()

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
    err_vs_fp64 = float(torch.linalg.norm(m - m_ref64) / torch.linalg.norm(m_ref64))

    # per-kernel profile of one more step (events around every launch)
    plan.profile(True)
    step()
    prof = plan.profile_read()
    plan.profile(False)
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

    # the paper's other coarse spaces, after the timed region (each replaces the one
    # above): the a priori Z_S merged into 32 interval groups (Sec. 3.3.1), the Arnoldi
    # (Algorithm 1) and CG-Lanczos a posteriori spaces keeping the Ritz values below
    # eps_tol = 0.2 (Sec. 5)
    coarse_variants = {}
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
            coarse_variants[name] = {"error": str(e)}
            continue
        torch.cuda.synchronize()
        tb = time.perf_counter() - t
        _, s64, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_FP64, out=m)
        _, smx, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_TWOLEVEL, mm.MM_SOLVE_MIXED, out=m)
        coarse_variants[name] = {"k": kc, "build_s": round(tb, 4), "fp64_s": s64["ms_total"] / 1e3,
                                 "fp64_iters": s64["iters"], "mixed_s": smx["ms_total"] / 1e3,
                                 "mixed_iters": smx["iters"], "mixed_rel_resid": smx["rel_resid"]}
    # the A-DEF2 form (App. B) on the last coarse space
    plan.build_coarse_eps(0.2, 64, mm.MM_FP32, bprime=b0, tol=TOL, maxit=3000)
    _, s64, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_ADEF2, mm.MM_SOLVE_FP64, out=m)
    _, smx, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_ADEF2, mm.MM_SOLVE_MIXED, out=m)
    coarse_variants["aposteriori_eps0.2_adef2"] = {
        "k": coarse_variants.get("aposteriori_eps0.2", {}).get("k"), "fp64_s": s64["ms_total"] / 1e3, "fp64_iters": s64["iters"],
        "mixed_s": smx["ms_total"] / 1e3, "mixed_iters": smx["iters"], "mixed_rel_resid": smx["rel_resid"]}

    if rank != 0:
        return
    # roofline of the dominant kernel of the step
    hbm, peak_src = peaks()
    nt, n = plan.nt, plan.n
    stages = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(stages, key=lambda k: stages[k][0])
    roof = roofline(dom, stages[dom][0] / stages[dom][1], plan, scan, hbm, peak_src)
    # A x HBM GB/s (algorithmic bytes per A x: pointing + weights + x and y; TOD excluded)
    axgbs = {}
    for key, sz in (("f32", 4), ("f64", 8)):
        t_ax = (ax[key]["toeplitz_ms"] + ax[key]["scatter_ms"]) * 1e-3
        axgbs[key] = (nt * (4 + 2 * sz) + 2 * n * sz) / t_ax / 1e9
    line = {
        "metric": METRIC,
        "value": ms_step / 1e3, "unit": "s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nt": nt, "n": n, "npix_obs": plan.npix_obs, "k_kept": kk,
                   "fft_block_f64": plan.fft_block_f64, "fft_block_f32": plan.fft_block_f32,
                   "l2": L2_NOTE,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gpu_launches": int(launches),
        "solve": {"iters": st["iters"], "outer": st["outer"], "fp64_products": st["fp64_products"],
                  "rel_resid": st["rel_resid"], "map_rel_err_vs_fp64_2lvl": err_vs_fp64},
        "fp64_bj": {"s": st_bj["ms_total"] / 1e3, "iters": st_bj["iters"], "rel_resid": st_bj["rel_resid"]},
        "fp64_2lvl": {"s": st_2f["ms_total"] / 1e3, "iters": st_2f["iters"]},
        "speedup_vs_fp64_bj": (st_bj["ms_total"] / 1e3) / (ms_step / 1e3),
        "coarse_build_s": t_coarse,
        "coarse_variants": coarse_variants,
        "ax_gbs": {k: round(v, 1) for k, v in axgbs.items()},
        "ax_ms": ax,
        "profile_ms": {k: [round(v[0], 4), v[1]] for k, v in stages.items()},
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(nt * 8), "d2h_bytes_per_step": int(n * 8)},
    }
    if world == 1 and not a.no_cpu_baseline:
        iters, src, _ = oracle_iterations()
        if iters is None:
            iters, src = st_2f["iters"], "FP64 two-level PCG iteration count of this run"
        try:
            vals, info = oracle_time_to_solution(1, iters)
            line["cpu_baseline"] = {"value": vals[0], "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": f"b = P^T N^-1 d plus 2 two-level PCG iterations of the full workload "
                                              f"(FP64 NumPy/SciPy, 1 thread), extrapolated to {iters} iterations "
                                              f"({src}); plan time {info['t_plan']:.1f} s excluded"}
        except Exception as ex:  # the GPU number stands; say why the baseline is missing
            line["cpu_baseline"] = {"value": None, "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {str(ex)[:200]}"}
    print(json.dumps(line))
    plan.close()


def run_sweep():
    """Bandwidth and knee-frequency sweeps (the paper's Sec. 5 studies of lambda_T and
    f_knee, on the synthetic 2^24-sample polarised scan): iterations and times to 1e-6 of
    FP64 block-Jacobi, two-level a priori (Z_S, 32 interval groups) and two-level a
    posteriori (Ritz values below eps_tol = 0.2) PCG, and of the mixed-precision two-level
    solve."""
    import torch
    from paper_1408_3048_gb300 import mm, synth
    base = synth.config(CONFIG)
    sky = synth.sky_map(base.npix_sky, base.ncomp, 1000 + CONFIG)
    cases = [(lam, 1.0) for lam in (1024, 2048, 4096, 8192, 16384)] + [(4096, f) for f in (0.25, 4.0)]
    for lam, fk in cases:
        psds = np.array(base.psds, dtype=np.float64).reshape(-1, 3).copy()
        psds[:, 1] *= fk
        scan = synth.config(CONFIG)
        scan.lam = lam
        scan.psds = psds
        d0 = synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, psds, scan.fsamp, 2200))
        d1 = synth.tod(scan, sky, synth.noise_realisation(scan.offsets, scan.interval_psd, psds, scan.fsamp, 2201))
        plan = mm.Plan(scan.pix, scan.npix_sky, scan.weights, scan.offsets, scan.interval_psd, psds, lam, scan.fsamp)
        dc0, dc1 = torch.from_numpy(d0).cuda(), torch.from_numpy(d1).cuda()
        m = torch.empty(plan.n, dtype=torch.float64, device="cuda")
        out = {"lambda": lam, "fknee_scale": fk}
        if plan.fft_block_f64:
            _, st, _ = plan.solve(dc1, TOL, 20000, mm.MM_PREC_BD, mm.MM_SOLVE_FP64, out=m)
            out["bd_fp64"] = {"iters": st["iters"], "s": st["ms_total"] / 1e3}
        b0 = plan.rhs(dc0) if plan.fft_block_f64 else None
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
        print(json.dumps(out), flush=True)
        plan.close()
        del dc0, dc1, m
        torch.cuda.empty_cache()


def main():
    a = parse()
    if a.sweep:
        run_sweep()
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
