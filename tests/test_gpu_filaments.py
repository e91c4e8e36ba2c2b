"""Parity on the filament suspension: straight bead chains (bond 2.2a) under
gravity, and a perturbed variant whose bond and bending forces are non-zero.
Chains make elongated clusters and dense near-field pairs along each chain,
a geometry unlike the uniform cube.  Tolerances as in the cube tests."""
import numpy as np
import pytest

import hh_synth
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402

THETA = hh_synth.mlp_params(32, 7)
BF16_FLOOR = 2e-4


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def ctx():
    c = hh.Context()
    c.set_mlp(THETA, 32)
    return c


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("perturbed", [False, True])
def test_filaments_against_oracle(ctx, prec, perturbed):
    X, _, _ = hh_synth.filaments(80, 50, seed=21)
    if perturbed:
        X = hh_synth.perturb(X, 0.05, seed=22)
    F = oracle.filament_forces(X, 50)
    k = oracle.PairKernel("mlp", THETA, 32)
    p = hh.Params(precision=prec, leaf_size=32)
    U = ctx.predict(cuda(X), cuda(F), p).cpu().numpy()
    Uo, _ = oracle.hmatvec(X, F, k, leaf=32, eta=1.0, eps=1e-4, max_rank=48)
    tol = {"fp64": 1e-6, "fp32": 2e-5, "bf16": 1e-4}[prec]
    assert oracle.rel_error(Uo, U) < tol
    a1 = oracle.self_mobility()
    rows = np.arange(0, len(X), 7)
    Ud = oracle.dense_matvec(X, F, k, rows=rows, with_self=False)
    assert oracle.rel_error(Ud, U[rows] - a1 * F[rows]) <= {"fp64": 1e-4, "fp32": 1e-4, "bf16": BF16_FLOOR}[prec]


def test_filaments_bf16_leaf64_sampled_rows(ctx):
    # the bench's launch configuration (BF16, C_leaf 64) on 600 chains x 50 beads
    X, _, _ = hh_synth.filaments(600, 50, seed=23)
    F = oracle.filament_forces(X, 50)
    p = hh.Params(precision="bf16", leaf_size=64)
    U = ctx.predict(cuda(X), cuda(F), p).cpu().numpy()
    U2 = ctx.predict(cuda(X), cuda(F), p).cpu().numpy()
    assert np.array_equal(U, U2)
    rows = np.arange(0, len(X), 211)
    k = oracle.PairKernel("mlp", THETA, 32)
    Ud = oracle.dense_matvec(X, F, k, rows=rows, with_self=False)
    a1 = oracle.self_mobility()
    assert oracle.rel_error(Ud, U[rows] - a1 * F[rows]) <= BF16_FLOOR
