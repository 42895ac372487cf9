"""The multi-GPU form of the bench is replicas only (every rank solves its own noise
realisation; the one collective takes the max of the timings).  Checked with two gloo
ranks on the CPU: distinct realisations per rank, the max over ranks, and that only rank
0 runs the reference arm."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1408_3048_gb300 import synth
    real = bench.replica_realisations(rank)
    scan = synth.config(2, scale=256)
    d = synth.noise_realisation(scan.offsets, scan.interval_psd, scan.psds, scan.fsamp, 2200 + real[1])
    t = bench.max_over_ranks(10.0 * (rank + 1), world, torch.device("cpu"))

    class A:
        steps, warmup, gpus = 1, 0, world
    ran = []
    orig = bench.oracle_iterations
    bench.oracle_iterations = lambda: ran.append(rank) or (None, "")
    try:
        if rank != 0:
            bench.run_reference(A(), rank, world)   # returns without work
    finally:
        bench.oracle_iterations = orig
    q.put((rank, real, float(d[:64].sum()), t, ran))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, real0, s0, t0, ran0), (r1, real1, s1, t1, ran1) = out
    assert real0 != real1 and real0[0] == real1[0] == 0          # own realisation, shared coarse source
    assert s0 != s1                                              # different noise per rank
    assert t0 == t1 == 20.0                                      # max over ranks, on every rank
    assert ran1 == []                                            # rank 1 does no reference work
