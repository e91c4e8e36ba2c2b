"""The filament suspension: chain placement (hh_synth) and the oracle's bead
forces (gravity, harmonic bonds, bending) that the explicit Euler step feeds
to the mobility product.

The oracle's energy is pinned to closed forms of hand-built configurations;
its forces to central differences of that energy, to the two-bead spring,
and to the invariants of internal forces (zero net force and torque), so a
dropped term, a wrong sign or a wrong index fails one of them."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import hh_synth
import oracle

G = np.array([0.0, 0.0, -1.0])


def test_chains_are_straight_spaced_and_apart():
    nch, nb = 60, 12
    X, cid, side = hh_synth.filaments(nch, nb, seed=3)
    assert X.shape == (nch * nb, 3) and np.array_equal(cid, np.repeat(np.arange(nch), nb))
    C = X.reshape(nch, nb, 3)
    r = np.diff(C, axis=1)
    assert np.allclose(np.linalg.norm(r, axis=2), 2.2, rtol=0, atol=1e-12)
    t = r / np.linalg.norm(r, axis=2)[..., None]
    assert np.allclose(t, t[:, :1], atol=1e-12)                       # straight
    assert X.min() >= 0.0 and X.max() <= side
    pr = cKDTree(X).query_pairs(2.1, output_type="ndarray")
    assert not np.any(cid[pr[:, 0]] != cid[pr[:, 1]])                 # different chains >= 2.1 apart
    X2, _, side2 = hh_synth.filaments(nch, nb, seed=3)
    assert side2 == side and np.array_equal(X, X2)                    # seeded


def test_box_grows_when_rods_jam():
    # 40 rods of 20 beads (length 41.8) at phi = 0.1 ask for a cube of side
    # 32: they cannot all fit, so the cube grows in 5% steps
    X, cid, side = hh_synth.filaments(40, 20, seed=5)
    s0 = hh_synth.cube_side(40 * 20, 0.1)
    k = np.log(side / s0) / np.log(1.05)
    assert side > s0 and abs(k - round(k)) < 1e-9
    assert X.min() >= 0.0 and X.max() <= side
    pr = cKDTree(X).query_pairs(2.1, output_type="ndarray")
    assert not np.any(cid[pr[:, 0]] != cid[pr[:, 1]])


def test_energy_closed_forms():
    # two beads stretched to 3.2: bond energy (100/2)(1.0)^2 = 50; gravity -g.x
    X = np.array([[0.0, 0.0, 5.0], [3.2, 0.0, 5.0]])
    assert oracle.filament_energy(X, 2) == pytest.approx(50.0 + 10.0, abs=1e-12)
    assert oracle.filament_energy(X, 2, g=(0, 0, 0)) == pytest.approx(50.0, abs=1e-12)
    # three beads at rest length, right angle: bending 10 (1 - cos 90) = 10
    X = np.array([[0.0, 0.0, 0.0], [2.2, 0.0, 0.0], [2.2, 2.2, 0.0]])
    assert oracle.filament_energy(X, 3, g=(0, 0, 0)) == pytest.approx(10.0, abs=1e-12)
    # folded back on itself: 10 (1 - cos 180) = 20
    X = np.array([[0.0, 0.0, 0.0], [2.2, 0.0, 0.0], [0.0, 0.0, 0.0]])
    assert oracle.filament_energy(X, 3, g=(0, 0, 0)) == pytest.approx(20.0, abs=1e-12)
    # a straight chain at rest length has only the gravity energy
    X = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 3.2], [0.0, 0.0, 5.4]])
    assert oracle.filament_energy(X, 3) == pytest.approx(9.6, abs=1e-12)


def test_two_bead_force_is_the_spring():
    X = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])                  # |r| = 5
    F = oracle.filament_forces(X, 2, g=(0, 0, 0))
    u = np.array([0.6, 0.8, 0.0])
    assert np.allclose(F[1], -100.0 * (5.0 - 2.2) * u, atol=1e-12)    # pulled back
    assert np.allclose(F[0], +100.0 * (5.0 - 2.2) * u, atol=1e-12)


def test_straight_chains_feel_only_gravity():
    X, _, _ = hh_synth.filaments(30, 50, seed=9)
    F = oracle.filament_forces(X, 50)
    assert np.allclose(F, G[None, :], rtol=0, atol=1e-9)


@pytest.mark.parametrize("beads", [2, 3, 7])
def test_forces_are_minus_the_energy_gradient(beads):
    X, _, _ = hh_synth.filaments(3, beads, seed=11)
    X = hh_synth.perturb(X, 0.3, seed=12)
    F = oracle.filament_forces(X, beads)
    h = 1e-6
    Fd = np.empty_like(X)
    for i in range(X.shape[0]):
        for c in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, c] += h
            Xm[i, c] -= h
            Fd[i, c] = -(oracle.filament_energy(Xp, beads) - oracle.filament_energy(Xm, beads)) / (2 * h)
    assert np.max(np.abs(F - Fd)) <= 1e-6 * np.max(np.abs(F))


def test_internal_forces_have_no_net_force_or_torque():
    X, _, _ = hh_synth.filaments(20, 9, seed=13)
    X = hh_synth.perturb(X, 0.2, seed=14)
    Fi = oracle.filament_forces(X, 9) - G[None, :]
    scale = np.abs(Fi).max() * len(X)
    for c in range(20):
        s = slice(9 * c, 9 * c + 9)
        assert np.abs(Fi[s].sum(axis=0)).max() <= 1e-12 * scale
        assert np.abs(np.cross(X[s], Fi[s]).sum(axis=0)).max() <= 1e-10 * scale * np.abs(X).max()
    assert np.abs(Fi).max() > 1.0                                      # the perturbation is felt


def test_euler_step_composes_its_parts():
    X, _, _ = hh_synth.filaments(6, 8, seed=15)
    X = hh_synth.perturb(X, 0.1, seed=16)
    k = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 7), 32)
    X1, F, U = oracle.euler_step(X, 8, k, 0.01)
    assert np.array_equal(F, oracle.filament_forces(X, 8))
    Ud = oracle.dense_matvec(X, F, k)                       # nothing admissible at 48 beads: exact
    assert oracle.rel_error(Ud, U) < 1e-13
    assert np.allclose(X1, X + 0.01 * U, rtol=0, atol=1e-15)


def test_two_spheres_sediment_together_rpy_closed_form():
    # Stokes flow: two identical spheres under the same force keep their
    # relative position (the RPY pair tensor is even in r), and fall with
    # U = F / (6 pi mu a) + K_RPY(r) F; for r along the force,
    # K_RPY(r) F = F (1 + 2a^2/(3r^2) + 1 - 2a^2/r^2) / (8 pi mu r)
    k = oracle.PairKernel("rpy")
    r, dt = 5.0, 0.7
    X0 = np.array([[0.3, -0.2, 1.0], [0.3, -0.2, 1.0 + r]])
    dumps = oracle.simulate(X0, 0, 1, k, dt, 4, dump_every=1, leaf=8)
    assert len(dumps) == 5
    for Xk in dumps:
        assert np.allclose(Xk[1] - Xk[0], [0, 0, r], rtol=0, atol=1e-13)
    uz = -(1.0 / (6 * np.pi) + (2.0 + 2.0 / (3 * r * r) - 2.0 / (r * r)) / (8 * np.pi * r))
    assert np.allclose(dumps[1] - dumps[0], [[0, 0, dt * uz]] * 2, rtol=1e-13, atol=0)
    assert np.allclose(dumps[4] - dumps[0], [[0, 0, 4 * dt * uz]] * 2, rtol=1e-12, atol=0)


def test_simulate_dt_zero_and_dump_slots():
    k = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 7), 32)
    X, _, _ = hh_synth.filaments(3, 4, seed=8)
    X = np.concatenate([hh_synth.perturb(X, 0.1, 9), hh_synth.rsa_cube(20, 0.1, seed=10) + 40.0])
    d0 = oracle.simulate(X, 3, 4, k, 0.0, 3, dump_every=1)
    assert all(np.array_equal(d, X) for d in d0)
    d = oracle.simulate(X, 3, 4, k, 0.01, 5, dump_every=2)
    assert len(d) == 3 and not np.array_equal(d[1], X)
    Xe, _, _ = oracle.euler_step(X[:12], 4, k, 0.01)                 # chains alone: the one-step composition
    de = oracle.simulate(X[:12], 3, 4, k, 0.01, 1)
    assert np.array_equal(de[1], Xe)
