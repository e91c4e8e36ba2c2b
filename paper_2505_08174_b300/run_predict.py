"""Run H-HIGNN predictions U = M(X) F on a synthetic suspension and print
stage times: a command-line driver for profiling one configuration.

    python -m paper_2505_08174_b300.run_predict --n 100000 --steps 2 \
        --precision bf16 --leaf 64 --width 32

Workload: N spheres (a = 1) placed by random sequential addition in a cube
at volume fraction 0.1, forces N(0,1), pair MLP 4->W->W->W->6 with seeded
Xavier weights.  Every prediction runs through hh_predict on the GPU.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--precision", default="bf16")
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--eta", type=float, default=1.0)
    ap.add_argument("--max-rank", type=int, default=48)
    ap.add_argument("--phi", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=1234)
    a = ap.parse_args(argv)

    import torch

    import hh_synth
    from . import Context, Params

    X = hh_synth.rsa_cube(a.n, a.phi, seed=a.seed)
    F = hh_synth.forces(a.n, 0)
    theta = hh_synth.mlp_params(a.width, 7)
    ctx = Context()
    ctx.set_mlp(theta, a.width)
    p = Params(leaf_size=a.leaf, eta=a.eta, eps=a.eps, max_rank=a.max_rank, precision=a.precision)
    Xd, Fd = torch.as_tensor(X).cuda(), torch.as_tensor(F).cuda()
    U = torch.empty_like(Xd)
    for s in range(a.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.predict(Xd, Fd, p, out=U)
        torch.cuda.synchronize()
        st = ctx.stats()
        st["wall_ms"] = 1e3 * (time.perf_counter() - t0)
        print(json.dumps({"step": s, **st}), flush=True)


if __name__ == "__main__":
    main()
