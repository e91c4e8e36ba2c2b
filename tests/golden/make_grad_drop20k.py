"""Writes grad_drop20k.txt: the dense gradient of L = sum_i w_i . U_i, U the
dense mobility product (alpha_1 F + M F with the seeded pair MLP), for the
N = 20,000 Gaussian drop of the differentiation workload (sigma = 30 a, every
input seeded below), computed by the FP64 oracle over all N (N - 1) pairs:
dL/dtheta in full and dL/dX, dL/dF on 128 seeded rows.  Takes several
minutes on a few cores.

    python tests/golden/make_grad_drop20k.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import hh_synth  # noqa: E402
import oracle  # noqa: E402

N, SIGMA, GEOM_SEED, F_SEED, W_SEED, ROW_SEED, N_ROWS = 20000, 30.0, 7, 1, 2, 20, 128


def inputs():
    X, sigma = hh_synth.gaussian_cloud(N, SIGMA, seed=GEOM_SEED)
    F, W = hh_synth.forces(N, F_SEED), hh_synth.forces(N, W_SEED)
    rows = np.sort(np.random.default_rng(ROW_SEED).choice(N, N_ROWS, replace=False))
    return X, F, W, rows, sigma


def main():
    X, F, W, rows, sigma = inputs()
    k = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 7), 32)
    gF, gX, gT = oracle.dense_grad(X, F, W, k)
    out = os.path.join(HERE, "grad_drop20k.txt")
    with open(out, "w") as f:
        f.write(f"# dense FP64 gradient (oracle.dense_grad), N={N} Gaussian drop sigma_eff={sigma!r}, "
                f"geometry seed {GEOM_SEED}, F seed {F_SEED}, w seed {W_SEED}, MLP w=32 seed 7; "
                f"written by make_grad_drop20k.py\n")
        f.write(f"theta {len(gT)}\n")
        f.writelines(f"{float(v)!r}\n" for v in gT)
        f.write(f"rows {len(rows)}\n")
        for i in rows:
            f.write(f"{int(i)} " + " ".join(repr(float(v)) for v in gX[i]) + " "
                    + " ".join(repr(float(v)) for v in gF[i]) + "\n")


if __name__ == "__main__":
    main()
