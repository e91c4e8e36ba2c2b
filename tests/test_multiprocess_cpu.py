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
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-rows", "2"]
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


def test_sampled_error_interval_over_forces():
    import numpy as np

    import bench
    import oracle
    rng = np.random.default_rng(5)
    ref = rng.standard_normal((5, 64, 3))
    approx = ref + 1e-3 * rng.standard_normal((5, 64, 3))
    lo, hi = bench.rel_err_ci95_forces(ref, approx)
    e = np.mean([oracle.rel_error(ref[f], approx[f]) for f in range(5)])
    assert lo < e < hi


def _strong_rank(rank, world, port, out):
    """One rank of a strong-scaling prediction on CPU: its share of the blocks
    of one suspension (the W^G / W^H split), its partial velocities from the
    oracle's per-block products, summed over the ranks by all-reduce."""
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import hh_synth
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, leaf, eps = 500, 32, 1e-4
    X, F = hh_synth.rsa_cube(n, 0.1, seed=9), hh_synth.forces(n, 1)
    k = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 7), 32)
    t = oracle.build_tree(X, leaf)
    G, H = oracle.partition(t, leaf, 1.0)
    size = (t.end - t.begin).astype(np.int64)
    wg = np.maximum(size[G[:, 0]], size[G[:, 1]])
    wh = np.zeros(len(size), np.int64)
    np.add.at(wh, H[:, 0], size[H[:, 0]] * size[H[:, 1]])
    gown, nown = bench.shard_owners(wg, world), bench.shard_owners(wh, world)
    Fs = F[t.perm]
    Us = np.zeros((n, 3))
    if rank == 0:
        Us += oracle.self_mobility() * Fs
    for tau, sig in H:                       # near field of the target nodes this rank owns
        if nown[tau] != rank:
            continue
        for m in range(t.begin[tau], t.end[tau]):
            for j in range(t.begin[sig], t.end[sig]):
                if j != m:
                    Us[m] += oracle.pair_block(k, t.Xs[m] - t.Xs[j]) @ Fs[j]
    for b, (tau, sig) in enumerate(G):       # the admissible blocks this rank owns: C (Q F_sigma)
        if gown[b] != rank:
            continue
        t0, c, s0, q = int(t.begin[tau]), int(size[tau]), int(t.begin[sig]), int(size[sig])
        r = oracle.aca_block(k, t.Xs, t0, c, s0, q, eps, 48, 0)
        if r["rank"]:
            tq = np.einsum("pnab,nb->pa", r["Q"], Fs[s0:s0 + q])
            Us[t0:t0 + c] += np.einsum("pmab,pb->ma", r["C"], tq)
    U = torch.zeros((n, 3), dtype=torch.float64)
    U[torch.as_tensor(t.perm, dtype=torch.long)] = torch.as_tensor(Us)
    part = U.clone()
    bench.reduce_partial_u(U, dist)
    out.put((rank, part.numpy(), U.numpy(), int((gown == rank).sum()), int(((nown == rank) & (wh > 0)).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_strong_scaling_split_and_reduction_over_two_gloo_ranks():
    import numpy as np

    import hh_synth
    import oracle
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_strong_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    X, F = hh_synth.rsa_cube(500, 0.1, seed=9), hh_synth.forces(500, 1)
    k = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 7), 32)
    Uo, _ = oracle.hmatvec(X, F, k, leaf=32, eta=1.0, eps=1e-4, max_rank=48)
    for _, part, U, nb, nn in res:
        assert nb > 0 and nn > 0                                  # both ranks hold work
        assert oracle.rel_error(Uo, U) < 1e-12                    # the all-reduce assembles the whole product
    assert not np.allclose(res[0][1], res[1][1])
    assert oracle.rel_error(Uo, res[0][1] + res[1][1]) < 1e-12


def test_shard_owners_contiguous_and_balanced():
    import numpy as np

    import bench
    rng = np.random.default_rng(2)
    w = rng.integers(1, 1000, size=5000)
    for ns in (1, 2, 3, 7):
        own = bench.shard_owners(w, ns)
        assert np.all(np.diff(own) >= 0) and own.min() == 0 and own.max() == ns - 1
        per = np.bincount(own, weights=w, minlength=ns)
        assert np.all(np.abs(per - w.sum() / ns) <= w.max())
    assert np.all(bench.shard_owners(np.zeros(4), 3) == 0)
