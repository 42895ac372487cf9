"""Host logic of bench.py on the CPU: the DRAM traffic of a kernel is taken from a recorded
ncu capture only while the kernel's sources hash to the recorded value, and the roofline's
algorithmic bytes per launch are those of one A x (pixel index and weights per sample, x
read and y written; time-domain intermediates excluded)."""
import hashlib
import os
import shutil
from types import SimpleNamespace

import numpy as np
import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1408_3048_gb300", "csrc")


def _tree(tmp_path, kernel):
    csrc = tmp_path / "paper_1408_3048_gb300" / "csrc"
    csrc.mkdir(parents=True)
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES[kernel]:
        shutil.copy(os.path.join(CSRC, f), csrc / f)
        h.update((csrc / f).read_bytes())
    (tmp_path / "profiles").mkdir()
    return csrc, h.hexdigest()


def test_recorded_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc, digest = _tree(tmp_path, "toeplitz_f32")
    prof = tmp_path / "profiles" / "toeplitz_f32_case.md"
    assert bench.recorded_traffic("toeplitz_f32") == (None, "no ncu capture recorded")
    prof.write_text("notes\ntraffic: toeplitz_f32 dram_bytes_per_launch=12345 source_sha256=%s\n" % digest)
    assert bench.recorded_traffic("toeplitz_f32") == (12345, os.path.join("profiles", "toeplitz_f32_case.md"))
    # a changed kernel source makes the record stale: no traffic figure is reported
    with open(csrc / "toeplitz_f32.cu", "a") as f:
        f.write("\n// changed\n")
    val, why = bench.recorded_traffic("toeplitz_f32")
    assert val is None and "predates" in why
    assert bench.recorded_traffic("no_such_kernel") == (None, "no source map")


def _plan(ncomp):
    return SimpleNamespace(nt=1 << 20, n=3 * 4096 if ncomp == 3 else 4096, ncomp=ncomp,
                           fft_block_f32=1 << 15, fft_block_f64=1 << 14)


@pytest.mark.parametrize("ncomp", [1, 3])
@pytest.mark.parametrize("kernel", ["toeplitz_f32", "toeplitz_f64", "scatter_f32", "scatter_f64"])
def test_roofline_algorithmic_bytes(kernel, ncomp):
    plan = _plan(ncomp)
    scan = SimpleNamespace(lam=4096, offsets=np.array([0, 1 << 19, 1 << 20]))
    s = 4 if kernel.endswith("f32") else 8
    per_sample = 4 + (2 * s if ncomp == 3 else 0)         # index and weights; no time-domain value
    expect = plan.nt * per_sample + 2 * plan.n * s        # x read, y written
    ms = 0.25
    r = bench.roofline(kernel, ms, plan, scan, 6769.0, "measured")
    hbm = r if r["bound"] == "hbm" else r["hbm"]
    assert hbm["bytes_per_launch"] == expect
    assert hbm["achieved"] == pytest.approx(expect / (ms * 1e-3) / 1e9, abs=0.05)
    assert hbm["frac"] == pytest.approx(hbm["achieved"] / 6769.0, abs=1e-4)
    if kernel.startswith("toeplitz"):
        # the bound is whichever fraction is larger
        alu = r["alu"] if r["bound"] == "hbm" else r
        assert r["frac"] == max(hbm["frac"], alu["frac"])
        B = plan.fft_block_f32 if s == 4 else plan.fft_block_f64
        assert bench.fft_tiles(scan, B) == 2 * -(-(1 << 19) // (B - 2 * 4096))   # one PSD per interval
    else:
        assert r["bound"] == "hbm" and "alu" not in r


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    """Under torchrun the oracle arm runs and prints on rank 0 only; other ranks return at
    once (the oracle is never started there)."""
    monkeypatch.setattr(bench, "oracle_time_to_solution",
                        lambda *a, **k: (_ for _ in ()).throw(AssertionError("oracle started")))
    args = SimpleNamespace(gpus=2, steps=2, warmup=1)
    assert bench.run_reference(args, 1, 2) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line(capsys, monkeypatch):
    """The oracle arm's JSON line: the GPU arm's metric, time-like; `value` the extrapolated
    time-to-solution and ms_per_step the measured sample, each averaged over the steps after
    the warm-up; its own cpu_baseline (cores as used) and e2e."""
    import json
    info = {"samples": [5.0] + [0.5] * 3, "threads": 8, "sample_iters": 2}
    monkeypatch.setattr(bench, "oracle_time_to_solution",
                        lambda steps, iters: ([9.0] + [2.0] * (steps - 1), info))
    bench.run_reference(SimpleNamespace(gpus=1, steps=3, warmup=1), 0, 1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "s"
    assert line["value"] == 2.0 and line["higher_is_better"] is False
    assert line["ms_per_step"] == 500.0 and "extrapolated" in line["value_is"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 8
    assert line["e2e"]["value"] == 2.0 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["workload"] == bench.WORKLOAD


def test_clock_record_parsing(tmp_path):
    """The clocks key: median SM clock over the loaded samples, the maximum clock, and every
    throttle reason seen Active (samples from nvidia-smi --format=csv,noheader,nounits)."""
    path = tmp_path / "clocks.csv"
    rows = ["0, 345, 2070, 120.5, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active",   # idle
            "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbled line"]
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(path)
    cs.proc = SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: None, kill=lambda: None)
    rec = cs.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 4
    assert rec["reasons"] == ["sw_power_cap"]
    assert not path.exists()
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_peak_bandwidth_source(tmp_path, monkeypatch):
    import json
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6769.4}))
    assert bench.peaks() == (6769.4, "measured")


def test_fft_tiles_packs_runs_of_one_psd():
    """Two intervals of one PSD share tiles when the lambda gap between them saves a tile;
    other PSDs stay apart; the count is that of the library's layout on the 2^24-sample
    workload (736 tiles of 2^15 at lambda 4096, 821 without packing)."""
    lam, B = 100, 1000   # 800 valid outputs per tile
    scan = SimpleNamespace(lam=lam, offsets=np.array([0, 900, 1800, 2700]), interval_psd=np.array([0, 0, 1]))
    # run [0, 1]: 2 x 2 single tiles vs ceil((1800 + 100) / 800) = 3 packed; interval 2: 2
    assert bench.fft_tiles(scan, B) == 3 + 2
    scan.interval_psd = np.array([0, 1, 2])
    assert bench.fft_tiles(scan, B) == 6
    from paper_1408_3048_gb300 import synth
    c2 = synth.config(2)
    assert bench.fft_tiles(c2, 1 << 15) == 736
    c2.interval_psd = np.arange(len(c2.offsets) - 1)
    assert bench.fft_tiles(c2, 1 << 15) == 821
