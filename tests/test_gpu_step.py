"""The filament suspension's bead forces and explicit Euler step on the GPU
(hh_filament_forces, hh_filament_step) against the FP64 oracle.

The forces are FP64 on both sides but summed in a different order (the
kernel gathers per bead, the oracle accumulates per bond and joint): 1e-12
of the largest force.  The step's U follows the prediction tolerances of
the parity tests; X_new = X + dt U to rounding."""
import numpy as np
import pytest

import hh_synth
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402

THETA = hh_synth.mlp_params(32, 7)


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def ctx():
    c = hh.Context()
    c.set_mlp(THETA, 32)
    return c


def chains(n_chains, beads, seed, scale=0.3):
    X, _, _ = hh_synth.filaments(n_chains, beads, seed=seed)
    return hh_synth.perturb(X, scale, seed=seed + 1)


@pytest.mark.parametrize("n_chains,beads", [(1, 1), (4, 1), (3, 2), (5, 3), (7, 4), (40, 50), (300, 21)])
def test_forces_against_oracle(ctx, n_chains, beads):
    X = chains(n_chains, beads, seed=31 + beads)
    fil = hh.Filament(k_bond=100.0, l0=2.2, kappa=10.0, g=(0.3, -0.2, -1.0))
    F = ctx.filament_forces(cuda(X), beads, fil).cpu().numpy()
    Fo = oracle.filament_forces(X, beads, 100.0, 2.2, 10.0, (0.3, -0.2, -1.0))
    assert np.max(np.abs(F - Fo)) <= 1e-12 * max(1.0, np.abs(Fo).max())


def test_straight_chains_and_empty(ctx):
    X, _, _ = hh_synth.filaments(25, 50, seed=41)
    F = ctx.filament_forces(cuda(X), 50).cpu().numpy()
    assert np.allclose(F, [0.0, 0.0, -1.0], rtol=0, atol=1e-9)
    E = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    assert ctx.filament_forces(E, 50).shape == (0, 3)


def test_zero_length_bond_is_a_numeric_error(ctx):
    X = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0], [3.2, 2.0, 3.0]])
    with pytest.raises(hh.HHError):
        ctx.filament_forces(cuda(X), 3)
    with pytest.raises(ValueError):
        ctx.filament_forces(cuda(X), 2)                     # not whole chains


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("fp32", 2e-5), ("bf16", 1e-4)])
def test_euler_step_against_oracle(ctx, prec, tol):
    beads, dt = 20, 0.002
    X = chains(40, beads, seed=51, scale=0.05)
    k = oracle.PairKernel("mlp", THETA, 32)
    X1o, Fo, Uo = oracle.euler_step(X, beads, k, dt, leaf=32, eps=1e-4)
    Xd = cuda(X)
    F, U = ctx.filament_step(Xd, beads, hh.Params(precision=prec, leaf_size=32), dt)
    F, U, X1 = F.cpu().numpy(), U.cpu().numpy(), Xd.cpu().numpy()
    assert np.max(np.abs(F - Fo)) <= 1e-12 * np.abs(Fo).max()
    assert oracle.rel_error(Uo, U) < tol
    assert np.max(np.abs(X1 - (X + dt * U))) <= 4e-16 * np.abs(X).max()
    assert np.max(np.abs(X1 - X1o)) <= 2 * dt * tol * np.abs(Uo).max() * np.sqrt(len(X))


def test_step_is_forces_then_predict_then_update(ctx):
    beads, dt = 21, 0.002
    X = chains(120, beads, seed=61, scale=0.05)
    p = hh.Params(precision="bf16", leaf_size=64)
    Xd = cuda(X)
    F1 = ctx.filament_forces(Xd, beads)
    U1 = ctx.predict(Xd, F1, p)
    n_pred = ctx.stats()["n_launches"]
    F, U = ctx.filament_step(Xd, beads, p, dt)
    assert torch.equal(F, F1) and torch.equal(U, U1)          # same kernels, deterministic
    assert ctx.stats()["n_launches"] == n_pred + 2            # + the force and update kernels
    assert np.max(np.abs(Xd.cpu().numpy() - (X + dt * U1.cpu().numpy()))) <= 4e-16 * np.abs(X).max()
    # a second step starts from the moved positions
    F2, _ = ctx.filament_step(Xd, beads, p, dt)
    assert not torch.equal(F2, F)


def _mixture(seed):
    # a small version of the paper's filament suspension: chains inside, free
    # particles in the shell around them
    X, _, _ = hh_synth.filament_sphere(8, 6, 3.0, 300, seed=seed)
    return X


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("bf16", 1e-4)])
def test_simulate_against_oracle(ctx, prec, tol):
    # hh_simulate: chains (bonds, bending, gravity) then free particles (gravity
    # only); three steps with a dump after each, against the oracle's steps.
    # Positions drift apart by at most dt * (the per-step velocity error),
    # accumulated over the steps
    X = _mixture(71)
    fil = hh.Filament(k_bond=20.0, l0=3.0, kappa=50.0)
    dt, steps = 0.05, 3
    k = oracle.PairKernel("mlp", THETA, 32)
    ref = oracle.simulate(X, 8, 6, k, dt, steps, dump_every=1, leaf=32, eps=1e-4, k=20.0, l0=3.0, kappa=50.0)
    Xd = cuda(X)
    dumps, ts = ctx.simulate(Xd, hh.Params(precision=prec, leaf_size=32), dt, steps, n_chains=8, beads=6, fil=fil,
                             dump_every=1)
    assert dumps.shape == (steps + 1, len(X), 3) and len(ts) == steps and np.all(ts > 0)
    assert np.array_equal(dumps[0], X)
    assert np.array_equal(dumps[-1], Xd.cpu().numpy())
    for s in range(1, steps + 1):
        Uo = (ref[s] - ref[s - 1]) / dt
        assert np.max(np.abs(dumps[s] - ref[s])) <= s * dt * tol * np.abs(Uo).max() * np.sqrt(len(X)), s


def test_simulate_is_repeated_steps(ctx):
    # chains only: the same kernels as hh_filament_step, step after step
    beads, dt = 21, 0.002
    X = chains(60, beads, seed=81, scale=0.05)
    p = hh.Params(precision="bf16", leaf_size=64)
    Xa, Xb = cuda(X), cuda(X)
    for _ in range(3):
        ctx.filament_step(Xa, beads, p, dt)
    dumps, _ = ctx.simulate(Xb, p, dt, 3, n_chains=60, beads=beads, dump_every=3)
    assert torch.equal(Xa, Xb) and np.array_equal(dumps[1], Xb.cpu().numpy())
    # a drop (free particles only) under gravity with the RPY kernel: every
    # pair term pulls along the force (both RPY coefficients are positive for
    # r >= 2a), so every particle sinks, and faster than alone
    D0 = hh_synth.lattice_sphere(20.0, 3.5)
    D = cuda(D0)
    ctx.simulate(D, hh.Params(precision="fp64", kernel="rpy", leaf_size=64), 0.5, 2)
    dz = D.cpu().numpy()[:, 2] - D0[:, 2]
    assert np.all(dz < 2 * 0.5 * -oracle.self_mobility())


def test_simulate_stops_at_an_error(ctx):
    X = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0], [3.2, 2.0, 3.0], [9.0, 9.0, 9.0]])
    Xd = cuda(X)
    with pytest.raises(hh.HHError) as e:
        ctx.simulate(Xd, hh.Params(precision="fp64"), 0.01, 2, n_chains=1, beads=3, dump_every=1)
    assert e.value.status == hh.HH_ERR_NUMERIC
    assert np.array_equal(Xd.cpu().numpy(), X)
