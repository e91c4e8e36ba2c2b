"""Benchmark: particle-velocities/s of one H-HIGNN prediction U = M(X) F.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--n 1000000] [--impl ours|reference]

A step is one full prediction through the C-ABI (hh_predict): Morton tree,
admissibility partition, batched ACA fused with the low-rank apply, dense
inadmissible blocks, FP64 accumulation.  Workload: N = 1,000,000 spheres
(a = 1) placed by random sequential addition in a cube at volume fraction
0.1, forces N(0,1), pair MLP 4->32->32->32->6 (SiLU, Xavier weights rounded to
bf16), C_leaf = 64, eta = 1, zeta = 1e-4, max_rank 48.  Precision "bf16"
(default): every pair-kernel MLP evaluation (near field and the rows and
columns the ACA generates) on tcgen05 tensor cores with BF16 operands (each
activation split into a bf16 part and a bf16 remainder) and FP32
accumulation; ACA arithmetic and low-rank apply in FP32; FP64 pivot inverses,
norms and final accumulation.  "fp32" and "fp64" run every kernel in that type.

value    = N * K / (sum of CUDA-event times of the K predictions), inputs
           resident in HBM; L2 (126 MB) is flushed between steps by writing a
           256 MB buffer (outside the event pairs).
e2e      = same metric through the same call with the inputs in pinned host
           memory: H2D copy of X and F, prediction, D2H copy of U, per step.
rel_err  = Eq. 11 (M^(t,2) part only) against the FP64 dense oracle on 512
           sampled target rows, averaged over 5 force vectors (seeds 0..4),
           with a bootstrap 95% interval over the rows (rel_err_ci95);
           fp32 = the plain FP32 H-path on the same forces and rows (its
           time per prediction and error); ms_per_step_min is the fastest
           timed step (rank 0).
roofline = the ACA kernels (the dominant stage).  BF16: the pair-kernel MLP
           is bound by activation throughput: SiLU evaluations (96 per query
           at width 32, one MUFU ex2 and one rcp each) per second of the ACA
           phase against the SiLU rate hh_probe_throughput measures in the
           same run ("alu" bound); "tensor" beside it gives the algorithmic
           MMA flops (2 x MACs of the MLP, 4736 per query) against the
           measured sustained bf16 peak; roofline_near does the same for
           k_near_tc.  FP32 / FP64: FP32-equivalent flops (5145 per query)
           against the measured FP32 FMA rate x 2.
cpu_baseline = the FP64 CPU oracle as it stands: 64 sampled rows of the exact
           dense product on the host cores, scaled to particle-velocities/s.

Under torchrun each rank runs its own independent suspension of N particles
(weak scaling, no collective on the data path); rank 0 prints the line.  With
--scaling strong every rank predicts its shard of one suspension (blocks split
by the W^G / W^H workloads of Section 3.3) and an NCCL all-reduce sums the
partial velocities inside the timed step.

--workload selects a further configuration, one line each (1 GPU):
  batch64      64 suspensions (cubes and Gaussian clouds) in one batched call
  grad200k     N = 200k Gaussian drop: BF16 forward U plus the adjoint of
               the FP32 H-matrix (dL/dF, dL/dX, dL/dtheta; near-field entries
               FP32, admissible blocks FP64, every sum in a fixed order)
  cube10m      N = 10M uniform cube
  shortrange1m the headline with the short-range terms of Eq. 6 switched on
  train        Eq. 5 training steps of the pair MLP
  filament1m   20k straight chains of 50 beads (bond 2.2a, random
               orientation), explicit Euler steps: GPU bead forces (gravity,
               bonds, bending), prediction, position update
  c2sweep      N = 100k, C_leaf 64: MLP 4-64-64-64-6 and RPY x FP64 / FP32 /
               BF16 x eta in {0.7, 1, 1.5} x zeta in {1e-3, 1e-4, 1e-6}, one
               line per cell with its error on 256 exact dense rows
  twodrop      Section 4.3's two sedimenting drops (2 x 523,305 lattice
               particles, F = (0, 0, -1), dt 0.01, zeta 0.1, C_leaf 50):
               explicit Euler steps through hh_simulate, optional dumps
  filsphere    Section 4.3's filament suspension (5120 chains x 21 beads +
               107,520 free particles; k_t 20, k_b 50, dt 0.002, zeta 0.02,
               C_leaf 50), the same way
  latsub       Section 4.1's fixed-domain scenario: random subsets of one
               perturbed 100^3 lattice; per N the error of the BF16
               prediction and of the stored FP32 H-matrix before / after the
               SVD recompression of its factors, with their bytes and apply
               times
  peaks        throughput of the units the pair-kernel MLP leans on (MUFU
               ex2 / rcp / tanh, FP32 and FP64 FMA, the epilogue SiLU), with
               the SM clock sampled meanwhile
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOP_PER_QUERY = {32: 2 * (4 * 32 + 32 * 32 + 32 * 32 + 32 * 6) + 4 * 96 + 25,
                  64: 2 * (4 * 64 + 64 * 64 + 64 * 64 + 64 * 6) + 4 * 192 + 25}
# tensor-core flops of one pair-kernel evaluation: 2 x the MACs of the four
# MLP layers (the bf16 hi/lo operand split and padding are not counted)
MMA_FLOP_PER_QUERY = {32: 2 * (4 * 32 + 32 * 32 + 32 * 32 + 32 * 6), 64: 2 * (4 * 64 + 64 * 64 + 64 * 64 + 64 * 6)}
SILU_PER_QUERY = {32: 3 * 32, 64: 3 * 64}   # activations of the three hidden layers
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
PRECISION_NOTE = {
    "bf16": "pair-kernel MLP (near field and ACA rows/columns) on tcgen05, BF16 hi/lo operands, FP32 accumulate; "
            "ACA + low-rank apply FP32; FP64 pivots, norms and final sum",
    "fp32": "all kernels FP32; FP64 pivots, norms and final sum",
    "fp64": "all kernels FP64",
}
METRIC = "particle-velocities/sec per H-HIGNN prediction at N=1M; rel. L2 err vs FP64 dense"


def metric_for(n):
    """The headline metric's name, with the suspension size when it is not the default 1M."""
    return METRIC if n == 1_000_000 else METRIC.replace("N=1M", f"N={n}")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    # where the raw samples go: --clocks-csv, else a temporary file
    csv_path = None

    def __init__(self, index: int):
        import tempfile
        self.index = index
        self.proc = None
        self.path = ClockSampler.csv_path or os.path.join(tempfile.gettempdir(),
                                                          f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        if os.path.dirname(self.path):
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=10)
            self.f.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if len(r) >= 9]
        mx = [float(r[2]) for r in rows if len(r) >= 9]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# DRAM bytes (read + write) per pair-kernel query of the BF16 ACA, from one
# ncu capture of every ACA launch (k_aca_tc warp and CTA teams, k_round_*) of
# a prediction at N = 100,000 (the ACA capture kept under profiles/):
# 278.9 GB for 809,273,239 queries.  The traffic of a prediction is taken as
# proportional to its queries (the per-block working set does not grow with N).
ACA_TC_DRAM_BYTES_PER_QUERY = 344.6


def aca_traffic(queries):
    return None if ACA_TC_DRAM_BYTES_PER_QUERY is None else ACA_TC_DRAM_BYTES_PER_QUERY * queries


def rel_err_ci95(ref, approx, reps=2000, seed=0):
    """Bootstrap 95% interval of the sampled Eq. 11 error: target rows are
    resampled with replacement and eps = sqrt(sum |dU_i|^2 / sum |U_i|^2)
    recomputed per resample."""
    num = np.sum((np.asarray(approx) - np.asarray(ref)) ** 2, axis=1)
    den = np.sum(np.asarray(ref) ** 2, axis=1)
    pick = np.random.default_rng(seed).integers(0, len(num), size=(reps, len(num)))
    e = np.sqrt(num[pick].sum(1) / den[pick].sum(1))
    return [float(np.percentile(e, 2.5)), float(np.percentile(e, 97.5))]


def rel_err_ci95_forces(ref, approx, reps=2000, seed=0):
    """Bootstrap 95% interval of the Eq. 11 error averaged over force vectors:
    ref, approx [nf, rows, 3]; target rows are resampled with replacement
    (the same rows for every force vector) and the mean over the force
    vectors of eps = sqrt(sum |dU_i|^2 / sum |U_i|^2) recomputed."""
    num = np.sum((np.asarray(approx) - np.asarray(ref)) ** 2, axis=2)   # [nf, rows]
    den = np.sum(np.asarray(ref) ** 2, axis=2)
    pick = np.random.default_rng(seed).integers(0, num.shape[1], size=(reps, num.shape[1]))
    e = np.sqrt(num[:, pick].sum(2) / den[:, pick].sum(2)).mean(0)
    return [float(np.percentile(e, 2.5)), float(np.percentile(e, 97.5))]


def shard_owners(cost, n_shards):
    """The split of one prediction over n_shards GPUs (strong scaling): items
    (admissible blocks by W^G = max(|tau|, |sigma|), target nodes by W^H =
    |tau| sum |sigma|, Section 3.3) in order, cut into contiguous ranges of
    equal cumulative cost; item i with cost w_i, exclusive prefix P_i and
    total T goes to min(n - 1, floor(n (P_i + w_i / 2) / T)).  The library
    applies the same rule on the device (hh_shard_owners)."""
    cost = np.asarray(cost, dtype=np.float64)
    T = cost.sum()
    if T <= 0:
        return np.zeros(len(cost), np.int32)
    excl = np.concatenate([[0.0], np.cumsum(cost)[:-1]])
    return np.minimum(np.floor(n_shards * (excl + 0.5 * cost) / T), n_shards - 1).astype(np.int32)


def reduce_partial_u(U, dist):
    """Strong scaling: every rank holds its shard's partial velocities of the
    same suspension; their sum (all-reduce) is the prediction on every rank."""
    if dist is not None and dist.is_available() and dist.is_initialized():
        dist.all_reduce(U, op=dist.ReduceOp.SUM)
    return U


def weak_scaling_value(n_local, steps, total_ms_local, dist=None, device="cpu"):
    """Whole-job particle-velocities/s: the particles of every rank's own
    suspension over the slowest rank's time (max over ranks); returns
    (value, max total ms).  Without a process group, the local figures."""
    n_total, t_ms = float(n_local), float(total_ms_local)
    if dist is not None and dist.is_available() and dist.is_initialized():
        import torch
        x = torch.tensor([t_ms], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        m = torch.tensor([n_total], dtype=torch.float64, device=device)
        dist.all_reduce(m, op=dist.ReduceOp.SUM)
        t_ms, n_total = float(x.item()), float(m.item())
    return n_total * steps / (t_ms / 1e3), t_ms


def workload(n, seed_geom=1234):
    import hh_synth
    X = hh_synth.rsa_cube(n, 0.1, seed=seed_geom)
    F = hh_synth.forces(n, 0)
    theta = hh_synth.mlp_params(32, 7)
    return X, F, theta


def cpu_baseline(X, F, theta, rows=64, seed=0):
    """The oracle as it stands: exact dense FP64 rows on the host cores."""
    import oracle
    k = oracle.PairKernel("mlp", theta, 32)
    idx = np.sort(np.random.default_rng(seed).choice(len(X), rows, replace=False))
    t0 = time.perf_counter()
    Ud = oracle.dense_matvec(X, F, k, rows=idx, with_self=False)
    dt = time.perf_counter() - t0
    return idx, Ud, rows / dt, oracle.num_threads(), dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    X, F, theta = workload(args.n)
    for _ in range(args.warmup):
        cpu_baseline(X, F, theta, rows=8, seed=99)
    tot_rows, tot_t = 0, 0.0
    for s in range(args.steps):
        _, _, rate, cores, dt = cpu_baseline(X, F, theta, rows=args.cpu_rows, seed=s)
        tot_rows += args.cpu_rows
        tot_t += dt
    v = tot_rows / tot_t
    sample = f"{args.cpu_rows} sampled target rows of the N={args.n} exact dense FP64 product per step"
    line = {"impl": "reference", "metric": metric_for(args.n), "value": v, "unit": "particle-velocities/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"uniform_cube_rsa_N{args.n}_phi0.1_mlp4-32-32-32-6", "n": args.n},
            "cpu_baseline": {"value": v, "unit": "particle-velocities/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "particle-velocities/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world):
    import torch

    import paper_2505_08174_b300 as hh

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    strong = args.scaling == "strong" and world > 1
    # weak: an independent suspension per rank; strong: one suspension, each rank its shard of the work
    X, F, theta = workload(args.n, seed_geom=1234 if strong else 1234 + rank)
    n = len(X)
    ctx = hh.Context(dev)
    ctx.set_mlp(theta, 32)
    prec = args.precision
    p = hh.Params(leaf_size=args.leaf, eta=1.0, eps=args.eps, max_rank=48, precision=prec,
                  mem_budget=args.budget_mb << 20, shard_id=rank if strong else 0, n_shards=world if strong else 1)
    Xd = torch.as_tensor(X).cuda()
    Fd = torch.as_tensor(F).cuda()
    U = torch.empty_like(Xd)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step():
        ctx.predict(Xd, Fd, p, out=U)
        if strong:
            reduce_partial_u(U, dist)   # NCCL all-reduce(sum) of the shards' FP64 partial velocities

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_aca_kern, queries, launches = 0.0, 0, 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for s in range(args.steps):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            step()
            ev[s][1].record(stream)
            st = ctx.stats()
            t_aca_kern += st.get("t_kernel_aca", st["t_aca"])
            queries += st["n_aca_queries"]
            launches += st.get("n_launches", 0)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, total_ms = weak_scaling_value(n, args.steps, float(np.sum(step_ms)), dist, "cuda")
    if strong:   # the whole job predicted one suspension of n particles per step
        value = n * args.steps / (total_ms / 1e3)
    clocks = clk.summary()
    st = ctx.stats()
    if args.profile:   # the timed predictions only (profiling runs): no accuracy, baseline or e2e legs
        if rank == 0:
            print(json.dumps({"profile": True, "n": n, "ms_per_step": total_ms / args.steps, "value": value,
                              "stages_ms": {k: st[k] for k in ("t_tree", "t_part", "t_near", "t_aca", "t_acc")},
                              "n_aca_queries": st["n_aca_queries"], "n_near_pairs": st["n_near_pairs"],
                              "n_aca_rounds": st["n_aca_rounds"], "t_aca_tiles": st["t_aca_tiles"],
                              "t_aca_steps": st["t_aca_steps"], "launches": launches, "clocks": clocks}),
                  flush=True)
        if dist:
            dist.destroy_process_group()
        return

    # end to end: pinned host inputs, H2D + predict + D2H per step
    Xh = torch.as_tensor(X).pin_memory()
    Fh = torch.as_tensor(F).pin_memory()
    Uh = torch.empty_like(Xh).pin_memory()
    e2e_t = []
    for s in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xd.copy_(Xh, non_blocking=True)
        Fd.copy_(Fh, non_blocking=True)
        step()
        Uh.copy_(U, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = n * (1 if strong else world) / float(np.mean(e2e_t))

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # accuracy (Eq. 11 on M^(t,2) F, averaged over 5 force vectors) on ref_rows sampled target rows, and the
    # plain FP32 H-path on the same forces (the "BF16 beats FP32 at equal accuracy" comparison)
    import hh_synth
    import oracle
    a1 = oracle.self_mobility()
    Fs5 = np.stack([hh_synth.forces(n, sd) for sd in range(5)])
    rows = np.sort(np.random.default_rng(0).choice(n, args.ref_rows, replace=False))

    def predictions(prec):
        pp = hh.Params(leaf_size=args.leaf, eta=1.0, eps=args.eps, max_rank=48, precision=prec,
                       mem_budget=args.budget_mb << 20)
        out, ms = [], []
        for sd in range(5):
            Fd.copy_(torch.as_tensor(Fs5[sd]))
            flush.fill_(float(sd))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.predict(Xd, Fd, pp, out=U)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            out.append(U.cpu().numpy()[rows] - a1 * Fs5[sd][rows])
        return np.stack(out), ms
    Ug, _ = predictions(prec)
    U32, ms32 = predictions("fp32") if prec != "fp32" else (Ug, [])
    rates = measure_units(ctx)
    idx, Ud1, cpu_rate, cores, cpu_dt = cpu_baseline(X, F, theta, rows=args.cpu_rows)
    t0 = time.perf_counter()
    Ud = oracle.dense_matvec_multi(X, Fs5, oracle.PairKernel("mlp", theta, 32), rows=rows, with_self=False)
    ref_dt = time.perf_counter() - t0
    errs = [float(oracle.rel_error(Ud[sd], Ug[sd])) for sd in range(5)]
    errs32 = [float(oracle.rel_error(Ud[sd], U32[sd])) for sd in range(5)]
    rel_err = float(np.mean(errs))

    peaks = _peaks()
    aca_ms = t_aca_kern / args.steps
    near_ms = st.get("t_kernel_near", st["t_near"])
    q_step = queries / args.steps
    silu_rate = rates["silu"]
    if prec == "bf16":
        # the binding roofline of the pair-kernel MLP is activation throughput: SiLU evaluations (one ex2 and one
        # rcp on the MUFU unit each, 96 per query at width 32) against the measured rate of the same SiLU
        peak, peak_src = peaks.get("bf16_tflops_sustained"), "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
        if peak is None:
            peak, peak_src = 1400.0, "fallback sustained bf16 1.4 PFLOP/s (of fallback)"
        silu_ach = q_step * SILU_PER_QUERY[32] / (aca_ms / 1e3) / 1e9
        roofline = {"bound": "alu", "kernel": "ACA: k_aca_tc warp + CTA teams, k_round_tiles (largest blocks)",
                    "achieved": silu_ach, "peak": silu_rate / 1e9, "unit": "G SiLU/s", "frac": silu_ach * 1e9 / silu_rate,
                    "traffic": aca_traffic(q_step),
                    "peak_source": "hh_probe_throughput SiLU rate measured in this run (MUFU ex2 + rcp per SiLU)",
                    "tensor": {"achieved": q_step * MMA_FLOP_PER_QUERY[32] / (aca_ms / 1e3) / 1e12, "peak": peak,
                               "unit": "TFLOP/s", "peak_source": peak_src}}
        roofline["tensor"]["frac"] = roofline["tensor"]["achieved"] / peak
        near_silu = st["n_near_pairs"] * SILU_PER_QUERY[32] / (near_ms / 1e3) / 1e9
        near_ach = st["n_near_pairs"] * MMA_FLOP_PER_QUERY[32] / (near_ms / 1e3) / 1e12
        roofline_near = {"bound": "alu", "kernel": "k_near_tc", "achieved": near_silu, "peak": silu_rate / 1e9,
                         "unit": "G SiLU/s", "frac": near_silu * 1e9 / silu_rate,
                         "tensor": {"achieved": near_ach, "peak": peak, "unit": "TFLOP/s", "frac": near_ach / peak}}
    else:
        achieved = q_step * FLOP_PER_QUERY[32] / (aca_ms / 1e3) / 1e12
        fma_peak = rates["ffma"] * 2 / 1e12
        roofline = {"bound": "alu", "kernel": "k_aca_cta + k_aca_warp (block ACA teams)", "achieved": achieved,
                    "peak": fma_peak, "unit": "TFLOP/s", "frac": achieved / fma_peak, "traffic": None,
                    "peak_source": "hh_probe_throughput FP32 FMA rate measured in this run x 2 flop"}
        roofline_near = None
    line = {
        "metric": metric_for(n), "value": value, "unit": "particle-velocities/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if strong else "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16"}[prec], "data": "synthetic",
        "config": {"workload": f"uniform_cube_rsa_N{n}_phi0.1_mlp4-32-32-32-6", "n": n, "leaf_size": args.leaf,
                   "eta": 1.0, "eps": args.eps, "max_rank": 48, "precision": prec,
                   "arithmetic": PRECISION_NOTE[prec],
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": ("one suspension split over the GPUs by W^G / W^H, NCCL all-reduce of U"
                                   if strong else "independent suspension per GPU")},
        "ms_per_step_min": float(np.min(step_ms)),
        "device_mem_gb": {"library_peak": st.get("mem_peak_bytes", -1) / 1e9,
                          "torch_peak": torch.cuda.max_memory_allocated() / 1e9},
        "rel_err": rel_err, "rel_err_rows": len(rows), "rel_err_forces": 5, "rel_err_per_force": errs,
        "rel_err_ci95": rel_err_ci95_forces(Ud, Ug),
        "fp32": {"ms_per_step": float(np.mean(ms32)) if ms32 else None, "rel_err": float(np.mean(errs32)),
                 "rel_err_per_force": errs32, "note": "plain FP32 H-path (SIMT MLP) on the same 5 forces and rows"},
        "units_per_s": rates,
        "stages_ms": {k: st[k] for k in ("t_tree", "t_part", "t_near", "t_aca", "t_acc")},
        "counts": {"n_aca_queries": st["n_aca_queries"], "n_near_pairs": st["n_near_pairs"],
                   "n_blocks_G": st["n_blocks_G"], "n_blocks_H": st["n_blocks_H"], "n_nodes": st["n_nodes"]},
        "roofline": roofline,
        "roofline_near": roofline_near,
        "cpu_baseline": {"value": cpu_rate, "unit": "particle-velocities/s", "cores": cores, "kind": "oracle",
                         "sample": f"{len(idx)} target rows of the N={n} exact dense FP64 product ({cpu_dt:.1f} s)"},
        "rel_err_reference": f"{len(rows)} rows x 5 forces of the exact dense FP64 product ({ref_dt:.1f} s)",
        "e2e": {"value": e2e_value, "unit": "particle-velocities/s", "h2d_bytes_per_step": 2 * 24 * n,
                "d2h_bytes_per_step": 24 * n},
        "gpu_launches": launches,
        "clocks": clocks,
        "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops", "sm_max_mhz")},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---- further workloads (not the headline line) ---------------------------------
def batch64_inputs(seed=99):
    """64 suspensions, N_b log-uniform in [1e3, 2e5]; even b: RSA cube at phi ~ U(0.05, 0.2), odd b:
    Gaussian cloud sigma = 20a (widened to peak phi <= 0.25)."""
    import hh_synth
    rng = np.random.default_rng(seed)
    Ns = np.round(np.exp(rng.uniform(np.log(1e3), np.log(2e5), 64))).astype(int)
    Xs = []
    for b, nb in enumerate(Ns):
        if b % 2 == 0:
            Xs.append(hh_synth.rsa_cube(int(nb), float(rng.uniform(0.05, 0.2)), seed=1000 + b))
        else:
            Xs.append(hh_synth.gaussian_cloud(int(nb), 20.0, seed=1000 + b)[0])
    off = np.concatenate([[0], np.cumsum(Ns)]).astype(np.int64)
    return np.concatenate(Xs), off


def _timed(ctx, call, steps, warmup, dev):
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches = 0
    with ClockSampler(dev) as clk:
        for s in range(steps):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            call()
            ev[s][1].record(stream)
            launches += ctx.stats().get("n_launches", 0)
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return float(np.sum(ms)), clk.summary(), launches


def measure_units(ctx, iters=1 << 17):
    """Measured rates (ops/s) of the arithmetic units of the activation-bound
    MLP (hh_probe_throughput), each timed over ~0.1-1 s."""
    out = {}
    for k, scale in (("mufu_ex2", 1), ("mufu_rcp", 1), ("mufu_tanh", 1), ("silu", 1), ("ffma", 8), ("dfma", 1)):
        out[k] = ctx.probe(k, iters * scale)
    return out


def run_workload(args):
    import torch

    import hh_synth
    import oracle
    import paper_2505_08174_b300 as hh

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    theta = hh_synth.mlp_params(32, 7)
    ctx = hh.Context(dev)
    ctx.set_mlp(theta, 32)
    kern = oracle.PairKernel("mlp", theta, 32)
    a1 = oracle.self_mobility()
    line = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic"}
    if args.workload == "c2sweep":
        # N = 100k uniform cube, C_leaf 64, MLP 4-64-64-64-6 and the closed-form RPY tensor, FP64 / FP32 / BF16
        # (BF16: the MLP only) x eta in {0.7, 1, 1.5} x zeta in {1e-3, 1e-4, 1e-6}; one line per cell
        n = args.n if args.n != 1_000_000 else 100_000
        X = hh_synth.rsa_cube(n, 0.1, seed=1234)
        F = hh_synth.forces(n, 0)
        th64 = hh_synth.mlp_params(64, 7)
        c64 = hh.Context(dev)
        c64.set_mlp(th64, 64)
        Xd, Fd = torch.as_tensor(X).cuda(), torch.as_tensor(F).cuda()
        U = torch.empty_like(Xd)
        rows = np.sort(np.random.default_rng(3).choice(n, 256, replace=False))
        refs = {}
        for kind in ("mlp", "rpy"):
            t0 = time.perf_counter()
            refs[kind] = oracle.dense_matvec(X, F, oracle.PairKernel(kind, th64, 64), rows=rows, with_self=False)
            refs[kind + "_s"] = time.perf_counter() - t0
        for kind in ("mlp", "rpy"):
            for prec in args.c2_precisions.split(","):
                if kind == "rpy" and prec == "bf16":
                    continue
                for eta in (0.7, 1.0, 1.5):
                    for eps in (1e-3, 1e-4, 1e-6):
                        p = hh.Params(leaf_size=64, eta=eta, eps=eps, precision=prec, kernel=kind)
                        c64.predict(Xd, Fd, p, out=U)
                        torch.cuda.synchronize()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        c64.predict(Xd, Fd, p, out=U)
                        e1.record()
                        torch.cuda.synchronize()
                        ms = e0.elapsed_time(e1)
                        st = c64.stats()
                        Ug = U.cpu().numpy()[rows] - a1 * F[rows]
                        cell = dict(line)
                        cell.update({"metric": "particle-velocities/sec, C2 sweep cell", "value": n / (ms / 1e3),
                                     "unit": "particle-velocities/s", "ms_per_step": ms, "steps": 1, "warmup": 1,
                                     "dtype": prec,
                                     "config": {"workload": f"uniform_cube_rsa_N{n}_phi0.1_c2sweep", "n": n,
                                                "kernel": "mlp4-64-64-64-6" if kind == "mlp" else "rpy",
                                                "precision": prec, "eta": eta, "eps": eps, "leaf_size": 64},
                                     "rel_err": float(oracle.rel_error(refs[kind], Ug)), "rel_err_rows": len(rows),
                                     "n_aca_queries": st["n_aca_queries"], "n_near_pairs": st["n_near_pairs"],
                                     "n_blocks_G": st["n_blocks_G"], "stages_ms": {k: st[k] for k in
                                                                                  ("t_near", "t_aca")},
                                     "gpu_launches": st.get("n_launches", 0)})
                        print(json.dumps(cell), flush=True)
        line.update({"metric": "C2 sweep finished", "value": len(rows), "unit": "rows", "ms_per_step": None,
                     "dtype": "mixed", "config": {"workload": "c2sweep_summary",
                                                  "reference_seconds": {k: refs[k + "_s"] for k in ("mlp", "rpy")}},
                     "gpu_launches": 0, "clocks": None})
    elif args.workload == "peaks":
        with ClockSampler(dev) as clk:
            rates = measure_units(ctx)
        line.update({"metric": "arithmetic-unit throughput (MUFU, FMA) on one B300",
                     "value": rates["silu"], "unit": "SiLU/s", "ms_per_step": None, "dtype": "f32",
                     "config": {"workload": "unit_probes_8chains_8x256_threads_per_sm"},
                     "rates_per_s": rates, "gpu_launches": 12, "clocks": clk.summary()})
    elif args.workload == "batch64":
        X, off = batch64_inputs()
        n = len(X)
        F = hh_synth.forces(n, 0)
        p = hh.Params(leaf_size=args.leaf, eps=args.eps, precision=args.precision)
        Xd, Fd = torch.as_tensor(X).cuda(), torch.as_tensor(F).cuda()
        U = torch.empty_like(Xd)
        # autotune the launch shape on the first 16 suspensions (outside the timed region)
        k16 = int(off[16])
        tuned = ctx.autotune(Xd[:k16].contiguous(), p, reps=1, offsets=off[:17])
        total_ms, clocks, launches = _timed(ctx, lambda: ctx.predict(Xd, Fd, p, offsets=off, out=U), args.steps,
                                            args.warmup, dev)
        Uh = U.cpu().numpy()
        rows = np.sort(np.random.default_rng(1).choice(n, 64, replace=False))
        inst = np.searchsorted(off, rows, side="right") - 1
        Ud = np.stack([oracle.dense_matvec(X[off[b]:off[b + 1]], F[off[b]:off[b + 1]], kern,
                                           rows=np.array([r - off[b]]), with_self=False)[0]
                       for r, b in zip(rows, inst)])
        line.update({"metric": "particle-velocities/sec, 64 suspensions in one batched prediction",
                     "value": n * args.steps / (total_ms / 1e3), "unit": "particle-velocities/s",
                     "ms_per_step": total_ms / args.steps, "dtype": args.precision,
                     "config": {"workload": "batch64_logN_1e3_2e5_cubes_and_gaussian_clouds", "n": n,
                                "instances": 64, "leaf_size": args.leaf, "eps": args.eps, "launch": tuned,
                                "l2": "flushed between steps (256 MB write)"},
                     "rel_err": float(oracle.rel_error(Ud, Uh[rows] - a1 * F[rows])),
                     "rel_err_ci95": rel_err_ci95(Ud, Uh[rows] - a1 * F[rows]), "gpu_launches": launches,
                     "clocks": clocks})
    elif args.workload == "grad200k":
        n = args.n if args.n != 1_000_000 else 200000
        X = hh_synth.gaussian_cloud(n, 30.0, seed=7)[0]
        F, W = hh_synth.forces(n, 1), hh_synth.forces(n, 2)
        # forward U by the fused BF16 prediction; the adjoint of the FP32 H-matrix on the same positions:
        # its near-field entries in FP32, its admissible blocks along the pivots of an FP64 pivots-only
        # re-approximation, their factors rebuilt in FP64 group by group within the memory budget
        p = hh.Params(leaf_size=args.leaf, eps=args.eps, precision="bf16")
        pp = hh.Params(leaf_size=args.leaf, eps=args.eps, precision="fp32", pivots_only=True)
        Xd, Fd, Wd = torch.as_tensor(X).cuda(), torch.as_tensor(F).cuda(), torch.as_tensor(W).cuda()
        U = torch.empty_like(Xd)
        gF = torch.empty_like(Xd)
        gX = torch.zeros_like(Xd)
        gT = torch.zeros(len(theta), dtype=torch.float32, device="cuda")

        def step():
            ctx.predict(Xd, Fd, p, out=U)
            t = ctx.build_tree(Xd, pp)
            b = ctx.partition(t, pp)
            h = ctx.aca(t, b, pp)
            ctx.matvec_backward(h, Wd, Fd, gF=gF, gX=gX, gtheta=gT)
        total_ms, clocks, launches = _timed(ctx, step, args.steps, args.warmup, dev)
        line.update({"metric": "particle-gradients/sec: forward U and dL/dF, dL/dX, dL/dtheta of L = sum w.U",
                     "value": n * args.steps / (total_ms / 1e3), "unit": "particles/s",
                     "ms_per_step": total_ms / args.steps, "dtype": "bf16 forward, f32 near / f64 far adjoint",
                     "config": {"workload": f"gaussian_drop_N{n}_sigma30a", "n": n, "leaf_size": args.leaf,
                                "eps": args.eps, "l2": "flushed between steps (256 MB write)"},
                     "gpu_launches": launches, "clocks": clocks})
    elif args.workload == "shortrange1m":
        # the headline prediction with the short-range terms of Eq. 6 switched on (seeded networks)
        n = args.n
        X = hh_synth.rsa_cube(n, 0.1, seed=1234)
        F = hh_synth.forces(n, 0)
        ctx.set_short_range(hh_synth.mlp_params(32, 21), hh_synth.mlp_params(32, 22, n_in=7, n_out=12), 32, 5.0)
        p = hh.Params(leaf_size=args.leaf, eps=args.eps, precision=args.precision, short_range=True)
        Xd, Fd = torch.as_tensor(X).cuda(), torch.as_tensor(F).cuda()
        U = torch.empty_like(Xd)
        total_ms, clocks, launches = _timed(ctx, lambda: ctx.predict(Xd, Fd, p, out=U), args.steps, args.warmup, dev)
        st = ctx.stats()
        line.update({"metric": "particle-velocities/sec per prediction with the short-range terms of Eq. 6",
                     "value": n * args.steps / (total_ms / 1e3), "unit": "particle-velocities/s",
                     "ms_per_step": total_ms / args.steps, "dtype": args.precision,
                     "config": {"workload": f"uniform_cube_rsa_N{n}_phi0.1_short_range_rcut5", "n": n,
                                "leaf_size": args.leaf, "eps": args.eps, "l2": "flushed between steps (256 MB write)"},
                     "stages_ms": {k: st[k] for k in ("t_tree", "t_part", "t_near", "t_short", "t_aca", "t_acc")},
                     "n_short_pairs": st["n_short_pairs"], "gpu_launches": launches, "clocks": clocks})
    elif args.workload == "train":
        # Eq. 5 training of the pair MLP on the GPU: Adam steps on batches of two-particle samples (RPY teacher)
        B = 4096
        r, e = hh_synth.two_particle_samples(B * 64, seed=5)
        rd, ed = torch.as_tensor(r).cuda(), torch.as_tensor(e).cuda()
        th = torch.as_tensor(theta).cuda().contiguous()
        m, v = torch.zeros_like(th), torch.zeros_like(th)
        state = {"k": 0}

        def step():
            i = state["k"] % 64
            ctx.train_step(th, m, v, state["k"] + 1, 32, rd[i * B:(i + 1) * B], ed[i * B:(i + 1) * B], lr=1e-3)
            state["k"] += 1
        total_ms, clocks, launches = _timed(ctx, step, args.steps, args.warmup, dev)
        line.update({"metric": "training samples/sec (Eq. 5 loss, gradient and Adam step on the GPU)",
                     "value": B * args.steps / (total_ms / 1e3), "unit": "samples/s",
                     "ms_per_step": total_ms / args.steps, "dtype": "f32",
                     "config": {"workload": "two_particle_rpy_teacher_batch4096", "batch": B, "width": 32},
                     "gpu_launches": 4 * args.steps,   # per step: per-sample pass, weight sums, loss sum, Adam
                     "clocks": clocks})
    elif args.workload == "cube10m":
        n = 10_000_000
        X = hh_synth.rsa_cube(n, 0.1, seed=1234)
        F = hh_synth.forces(n, 0)
        p = hh.Params(leaf_size=args.leaf, eps=args.eps, precision=args.precision)
        Xd, Fd = torch.as_tensor(X).cuda(), torch.as_tensor(F).cuda()
        U = torch.empty_like(Xd)
        total_ms, clocks, launches = _timed(ctx, lambda: ctx.predict(Xd, Fd, p, out=U), args.steps, args.warmup, dev)
        st = ctx.stats()
        Uh = U.cpu().numpy()
        rows = np.sort(np.random.default_rng(0).choice(n, 16, replace=False))
        Ud = oracle.dense_matvec(X, F, kern, rows=rows, with_self=False)
        line.update({"metric": "particle-velocities/sec per H-HIGNN prediction at N=10M",
                     "value": n * args.steps / (total_ms / 1e3), "unit": "particle-velocities/s",
                     "ms_per_step": total_ms / args.steps, "dtype": args.precision,
                     "config": {"workload": "uniform_cube_rsa_N10000000_phi0.1", "n": n, "leaf_size": args.leaf,
                                "eps": args.eps, "device_mem_peak_gb": torch.cuda.max_memory_allocated() / 1e9,
                                "library_mem_peak_gb": st.get("mem_peak_bytes", -1) / 1e9},
                     "stages_ms": {k: st[k] for k in ("t_tree", "t_part", "t_near", "t_aca", "t_acc")},
                     "rel_err": float(oracle.rel_error(Ud, Uh[rows] - a1 * F[rows])), "rel_err_rows": len(rows),
                     "rel_err_ci95": rel_err_ci95(Ud, Uh[rows] - a1 * F[rows]),
                     "gpu_launches": launches, "clocks": clocks})
    elif args.workload == "filament1m":
        # the filament suspension time-stepped by explicit Euler: each step computes the bead forces
        # (gravity, bonds, bending) on the GPU, predicts U = M(X) F and moves the beads by dt U
        beads, dt = 50, 0.002
        nch = max(1, args.n // beads)
        X, _, side = hh_synth.filaments(nch, beads, seed=1234)
        n = len(X)
        phi = n * (4.0 / 3.0) * np.pi / side ** 3
        p = hh.Params(leaf_size=args.leaf, eps=args.eps, precision=args.precision)
        Xd = torch.as_tensor(X).cuda()
        Fd, U = torch.empty_like(Xd), torch.empty_like(Xd)
        total_ms, clocks, launches = _timed(ctx, lambda: ctx.filament_step(Xd, beads, p, dt, F=Fd, U=U), args.steps,
                                            args.warmup, dev)
        st = ctx.stats()
        # accuracy of one more step's U at the positions it started from
        Xs = Xd.cpu().numpy()
        ctx.filament_step(Xd, beads, p, dt, F=Fd, U=U)
        Fh, Uh = Fd.cpu().numpy(), U.cpu().numpy()
        rows = np.sort(np.random.default_rng(0).choice(n, 64, replace=False))
        Ud = oracle.dense_matvec(Xs, Fh, kern, rows=rows, with_self=False)
        line.update({"metric": "bead-velocities/sec per explicit Euler step of the filament suspension "
                               "(forces + H-HIGNN prediction + update)",
                     "value": n * args.steps / (total_ms / 1e3), "unit": "particle-velocities/s",
                     "ms_per_step": total_ms / args.steps, "dtype": args.precision,
                     "config": {"workload": f"filaments_{nch}x{beads}_bond2.2a_random_orientation_euler_dt{dt}",
                                "n": n, "chains": nch, "beads": beads, "side": side, "phi": phi, "dt": dt,
                                "forces": "gravity + harmonic bonds (k 100) + bending (kappa 10), on the GPU",
                                "leaf_size": args.leaf, "eps": args.eps, "l2": "flushed between steps (256 MB write)"},
                     "stages_ms": {k: st[k] for k in ("t_tree", "t_part", "t_near", "t_aca", "t_acc")},
                     "counts": {"n_aca_queries": st["n_aca_queries"], "n_near_pairs": st["n_near_pairs"]},
                     "rel_err": float(oracle.rel_error(Ud, Uh[rows] - a1 * Fh[rows])), "rel_err_rows": len(rows),
                     "rel_err_ci95": rel_err_ci95(Ud, Uh[rows] - a1 * Fh[rows]),
                     "gpu_launches": launches,
                     "clocks": clocks})
    elif args.workload == "latsub":
        # Section 4.1's fixed-domain scenario: random subsets of one perturbed 100^3 lattice (spacing 3.5),
        # so the concentration grows with N.  Per N: eps_r of the fused BF16 prediction and of the stored
        # FP32 H-matrix before and after the SVD recompression of its factors (eps_rc = zeta), against
        # 64 exact dense rows; the factor bytes and the low-rank apply's device time before and after
        rows_n = 64
        for n in [int(v) for v in args.latsub_n.split(",")]:
            X = hh_synth.lattice_subset(n, n_side=100, subset_seed=n)
            F = hh_synth.forces(n, 1)
            Xd, Fd = torch.as_tensor(X).cuda(), torch.as_tensor(F).cuda()
            rows = np.sort(np.random.default_rng(n).choice(n, min(rows_n, n), replace=False))
            Ud = oracle.dense_matvec(X, F, kern, rows=rows, with_self=False)
            pb = hh.Params(leaf_size=args.leaf, eps=args.eps, precision="bf16")
            Ub = ctx.predict(Xd, Fd, pb).cpu().numpy()
            rec = {"workload": "lattice_subset_fixed_domain_100^3_spacing3.5", "n": n,
                   "phi": n * (4.0 / 3.0) * np.pi / (100 * 3.5) ** 3, "leaf_size": args.leaf, "eps": args.eps,
                   "rel_err_bf16_predict": float(oracle.rel_error(Ud, Ub[rows] - a1 * F[rows]))}
            try:
                p32 = hh.Params(leaf_size=args.leaf, eps=args.eps, precision="fp32")
                t = ctx.build_tree(Xd, p32)
                b = ctx.partition(t, p32)
                h = ctx.aca(t, b, p32)
                nf = h.factor_count()
                def apply_ms():
                    ts = []
                    for _ in range(5):
                        U = ctx.matvec(h, Fd)
                        ts.append(ctx.stats()["t_apply"])
                    return U.cpu().numpy(), float(np.median(ts))
                U0, ms0 = apply_ms()
                t0 = time.perf_counter()
                h.recompress(args.eps)
                t_rc = time.perf_counter() - t0
                sr, so, _ = h.export_recompressed()
                U1, ms1 = apply_ms()
                rec.update({"factor_bytes_aca": 4 * 9 * nf, "factor_bytes_svd": 4 * int(so[-1]),
                            "byte_ratio": int(so[-1]) / max(1, 9 * nf),
                            "apply_ms_aca": ms0, "apply_ms_svd": ms1,
                            "apply_gbs_aca": 4 * 9 * nf / (ms0 * 1e6), "apply_gbs_svd": 4 * int(so[-1]) / (ms1 * 1e6),
                            "recompress_s": t_rc,
                            "rel_err_fp32_stored": float(oracle.rel_error(Ud, U0[rows] - a1 * F[rows])),
                            "rel_err_fp32_recompressed": float(oracle.rel_error(Ud, U1[rows] - a1 * F[rows]))})
                del h, b, t
            except hh.HHError as e:
                rec["stored_factors"] = f"skipped: {e}"
            print(json.dumps(dict(line, metric="relative error and apply bytes, fixed-domain lattice subsets",
                                  value=rec["rel_err_bf16_predict"], unit="eps_r", higher_is_better=False,
                                  config=rec)), flush=True)
        return
    elif args.workload in ("twodrop", "filsphere"):
        # Section 4.3's time-stepped runs: explicit Euler steps through hh_simulate (forces, prediction and
        # update on the GPU; positions copied to the host every --dump-every steps, written as .npy files
        # under --dump-dir)
        if args.workload == "twodrop":
            X = hh_synth.two_drops()
            nch, beads, dt, eps = 0, 1, 0.01, 0.1
            fil = hh.Filament(g=(0.0, 0.0, -1.0))
            cfg = {"workload": "two_lattice_drops_2x523305_radius175_spacing3.5_centres_3R_apart",
                   "forces": "gravity (0, 0, -1)"}
        else:
            X, r_in, r_out = hh_synth.filament_sphere()
            nch, beads, dt, eps = 5120, 21, 0.002, 0.02
            fil = hh.Filament(k_bond=20.0, l0=3.0, kappa=50.0, g=(0.0, 0.0, -1.0))
            cfg = {"workload": "filament_sphere_5120x21_beads_rb3_plus_107520_free",
                   "r_in": r_in, "r_out": r_out,
                   "forces": "gravity + bonds (k_t 20, l0 3) + bending (k_b 50), on the GPU"}
        n = len(X)
        p = hh.Params(leaf_size=50, eps=eps, precision=args.precision)
        Xd = torch.as_tensor(X).cuda()
        if args.warmup > 0:
            ctx.simulate(Xd, p, dt, args.warmup, n_chains=nch, beads=beads, fil=fil)
        X0 = Xd.cpu().numpy()
        torch.cuda.synchronize()
        with ClockSampler(dev) as clk:
            t0 = time.perf_counter()
            dumps, ts = ctx.simulate(Xd, p, dt, args.steps, n_chains=nch, beads=beads, fil=fil,
                                     dump_every=args.dump_every)
            wall = time.perf_counter() - t0
        if dumps is not None and args.dump_dir:
            os.makedirs(args.dump_dir, exist_ok=True)
            for i, d in enumerate(dumps):
                np.save(os.path.join(args.dump_dir, f"{args.workload}_step{args.warmup + i * args.dump_every:05d}.npy"), d)
        # accuracy of the step's velocities at the positions the timed run started from
        Fh = np.empty_like(X0)
        Fh[:nch * beads] = oracle.filament_forces(X0[:nch * beads], beads, fil.k_bond, fil.l0, fil.kappa,
                                                  tuple(fil.g)) if nch else Fh[:0]
        Fh[nch * beads:] = np.asarray(fil.g)
        Uh = ctx.predict(torch.as_tensor(X0).cuda(), torch.as_tensor(Fh).cuda(), p).cpu().numpy()
        rows = np.sort(np.random.default_rng(0).choice(n, 32, replace=False))
        Ud = oracle.dense_matvec(X0, Fh, kern, rows=rows, with_self=False)
        line.update({"metric": "particle-velocities/sec per explicit Euler step (forces + H-HIGNN prediction + "
                               "position update)",
                     "value": n * args.steps / (float(np.sum(ts)) / 1e3), "unit": "particle-velocities/s",
                     "ms_per_step": float(np.mean(ts)), "ms_per_step_each": [float(v) for v in ts],
                     "wall_s_with_dumps": wall, "dtype": args.precision,
                     "config": dict(cfg, n=n, dt=dt, leaf_size=50, eps=eps, steps_before=args.warmup,
                                    dump_every=args.dump_every),
                     "rel_err": float(oracle.rel_error(Ud, Uh[rows] - a1 * Fh[rows])), "rel_err_rows": len(rows),
                     "gpu_launches": None, "clocks": clk.summary()})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-rows", type=int, default=512,
                    help="sampled target rows of the exact dense product for the accuracy (x 5 force vectors)")
    ap.add_argument("--cpu-rows", type=int, default=64,
                    help="sampled target rows the timed CPU baseline computes")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="under torchrun: weak = a suspension per GPU; strong = one suspension split over the GPUs")
    ap.add_argument("--budget-mb", type=int, default=0,
                    help="memory budget of the BF16 ACA's active blocks in MB (0 = the library default)")
    ap.add_argument("--profile", action="store_true",
                    help="run the warm-up and timed predictions only and print their stage times (for ncu runs)")
    ap.add_argument("--c2-precisions", default="fp64,fp32,bf16",
                    help="c2sweep: the precisions swept (comma-separated)")
    ap.add_argument("--latsub-n", default="8000,27000,64000,125000,216000",
                    help="latsub: the subset sizes of the 100^3 lattice")
    ap.add_argument("--dump-every", type=int, default=0,
                    help="twodrop / filsphere: copy the positions to the host every this many steps")
    ap.add_argument("--dump-dir", default=None, help="twodrop / filsphere: write the position dumps here (.npy)")
    ap.add_argument("--clocks-csv", default=None,
                    help="keep the raw nvidia-smi clock samples of the timed region in this file")
    ap.add_argument("--workload", default="cube1m",
                    choices=["cube1m", "batch64", "grad200k", "cube10m", "shortrange1m", "train", "filament1m", "peaks",
                             "c2sweep", "twodrop", "filsphere", "latsub"],
                    help="cube1m is the headline; the others measure further configurations")
    args = ap.parse_args()
    if args.clocks_csv:
        ClockSampler.csv_path = args.clocks_csv
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload != "cube1m":
        if rank == 0:
            run_workload(args)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
