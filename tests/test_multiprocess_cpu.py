"""The multi-rank host path on CPU (gloo, world size 2): every rank runs its
own suspension, the job's throughput is all ranks' particles over the slowest
rank's time; the reference arm prints one line from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r processed 1000 (r + 1) particles per step in 100 (r + 1) ms over 2 steps
    value, t = bench.weak_scaling_value(1000 * (rank + 1), 2, 100.0 * (rank + 1), dist, "cpu")
    out.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_value_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, value, t in res:
        assert t == 200.0                                   # the slowest rank
        assert value == pytest.approx((1000 + 2000) * 2 / 0.2)


def test_single_process_value_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.weak_scaling_value(500, 4, 250.0) == (500 * 4 / 0.25, 250.0)


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-rows", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_sampled_error_interval():
    import numpy as np

    import bench
    import oracle
    rng = np.random.default_rng(4)
    ref = rng.standard_normal((64, 3))
    approx = ref + 1e-3 * rng.standard_normal((64, 3))
    lo, hi = bench.rel_err_ci95(ref, approx)
    e = oracle.rel_error(ref, approx)
    assert lo < e < hi and hi - lo < e
    # rows with one common relative error give a zero-width interval
    lo, hi = bench.rel_err_ci95(ref, 1.001 * ref)
    assert abs(lo - 1e-3) < 1e-12 and abs(hi - 1e-3) < 1e-12
