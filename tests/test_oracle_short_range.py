"""Pins of the oracle's short-range terms (Eq. 6: M^(s,2), M^(t,3), M^(s,3);
Eq. 2 sums with the Eq. 4 normalisations) and of its generic MLP.

The short-range oracle loops over neighbour lists and 3-cliques; the pins
below use other formulations: constant-output networks reduce both sums to
distance-matrix algebra (numpy / scipy), a hand-derived three-particle
configuration fixes the clique set and the strict cutoff, and invariances
hold for any network."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

import hh_synth
import oracle


def sym3(o):
    return np.array([[o[0], o[3], o[4]], [o[3], o[1], o[5]], [o[4], o[5], o[2]]])


def constant_net(n_in, w, n_out, out):
    """Packed MLP whose weights are all zero and whose output bias is `out`."""
    theta = np.zeros(hh_synth.mlp_param_count(w, 3, n_in, n_out))
    theta[-n_out:] = out
    return theta


def test_mlp_gen_equals_pair_mlp():
    rng = np.random.default_rng(1)
    for w in (32, 64):
        th = hh_synth.mlp_params(w, 3 + w)
        for _ in range(20):
            f = rng.normal(size=4)
            assert np.array_equal(oracle.mlp_gen(th, 4, w, 6, f), oracle.mlp_forward(th, w, f))


def test_mlp_gen_output_bias_and_sizes():
    out = np.arange(12) * 0.25 - 1.0
    th = constant_net(7, 32, 12, out)
    assert np.array_equal(oracle.mlp_gen(th, 7, 32, 12, np.ones(7)), out)


def _distance_formulation(X, F, Ss2, Ss3, St3, rcut, a):
    D = cdist(X, X)
    A = (D < rcut) & ~np.eye(len(X), dtype=bool)
    Dm = np.where(A, D, 1.0)
    c2 = np.where(A, (a / Dm) ** 4 / Dm, 0.0).sum(axis=1)            # sum_j (a/d)^4 / d
    B = np.where(A, 1.0 / Dm, 0.0)                                    # B_ik = 1/d_ik on neighbours
    # sum_k B_ik sum_{j != i} B_kj = (B @ B)_ii-free row sums
    T1 = B @ B.sum(axis=1) - np.diag(B @ B)
    # sum_k B_ik sum_{j != i} B_kj F_j
    T2 = B @ (B @ F) - (np.diag(B @ B))[:, None] * F
    return c2[:, None] * (F @ Ss2.T) + T1[:, None] * (F @ Ss3.T) + T2 @ St3.T


@pytest.mark.parametrize("seed", [0, 1])
def test_constant_networks_against_distance_matrices(seed):
    X = hh_synth.rsa_cube(300, 0.2, seed=seed)
    F = hh_synth.forces(300, seed)
    o2 = np.array([0.7, -0.2, 1.1, 0.3, -0.4, 0.05])
    o3 = np.array([0.2, 0.9, -0.5, 0.1, 0.6, -0.3, -1.0, 0.4, 0.8, 0.25, -0.15, 0.5])
    ts, t3 = constant_net(4, 32, 6, o2), constant_net(7, 32, 12, o3)
    U = oracle.short_range(X, F, ts, 32, t3, 32, rcut=5.0, a=1.0)
    Ue = _distance_formulation(X, F, sym3(o2), sym3(o3[:6]), sym3(o3[6:]), 5.0, 1.0)
    assert np.abs(Ue).max() > 0
    assert np.allclose(U, Ue, rtol=1e-12, atol=1e-14 * np.abs(Ue).max())
    # each term alone
    U2 = oracle.short_range(X, F, ts, 32, None, 32, rcut=5.0)
    U3 = oracle.short_range(X, F, None, 32, t3, 32, rcut=5.0)
    assert np.allclose(U2 + U3, U, rtol=1e-13, atol=1e-15)


def test_three_particles_by_hand():
    # d01 = 3, d02 = 4, d12 = 5: with R_cut = 5 (strict) N(0) = {1, 2}, N(1) = N(2) = {0}.
    # Cliques (j, k, i): none for i = 0; (2, 0, 1) and (1, 0, 2) with d_jk d_ki = 4*3 and 3*4.
    X = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0], [0.0, 4.0, 0.0]])
    F = np.array([[1.0, 2.0, 3.0], [-1.0, 0.5, 0.0], [0.0, 0.0, 2.0]])
    o3 = np.array([1.0, 2.0, 3.0, 0.5, -0.5, 0.25, -1.0, 1.5, 0.5, 0.0, 1.0, -2.0])
    t3 = constant_net(7, 32, 12, o3)
    U = oracle.short_range(X, F, None, 32, t3, 32, rcut=5.0)
    Ss, St = sym3(o3[:6]), sym3(o3[6:])
    assert np.array_equal(U[0], np.zeros(3))
    assert np.allclose(U[1], (Ss @ F[1] + St @ F[2]) / 12.0, rtol=1e-15, atol=0)
    assert np.allclose(U[2], (Ss @ F[2] + St @ F[1]) / 12.0, rtol=1e-15, atol=0)
    # alpha2s: particle 0 has two neighbours, 1 and 2 one each
    o2 = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])                     # S = I
    U2 = oracle.short_range(X, F, constant_net(4, 32, 6, o2), 32, None, 32, rcut=5.0)
    assert np.allclose(U2[0], (1 / 3 ** 5 + 1 / 4 ** 5) * F[0], rtol=1e-15)
    assert np.allclose(U2[1], F[1] / 3 ** 5, rtol=1e-15)
    assert np.allclose(U2[2], F[2] / 4 ** 5, rtol=1e-15)
    # raising the cutoff past 5 brings the pair (1, 2) and its cliques in
    U3 = oracle.short_range(X, F, None, 32, t3, 32, rcut=5.0 + 1e-9)
    assert not np.allclose(U3[0], 0.0)


def test_invariances_with_seeded_networks():
    X = hh_synth.rsa_cube(200, 0.2, seed=3)
    F = hh_synth.forces(200, 4)
    ts = hh_synth.mlp_params(32, 11)
    t3 = hh_synth.mlp_params(32, 12, n_in=7, n_out=12)
    U = oracle.short_range(X, F, ts, 32, t3, 32, rcut=5.0)
    assert np.abs(U).max() > 0
    Ut = oracle.short_range(X + np.array([17.25, -3.5, 8.0]), F, ts, 32, t3, 32, rcut=5.0)
    assert np.allclose(U, Ut, rtol=1e-9, atol=1e-12 * np.abs(U).max())
    perm = np.random.default_rng(5).permutation(200)
    Up = oracle.short_range(X[perm], F[perm], ts, 32, t3, 32, rcut=5.0)
    assert np.allclose(Up, U[perm], rtol=1e-12, atol=1e-15)
    # forces enter linearly
    U2 = oracle.short_range(X, 2.0 * F, ts, 32, t3, 32, rcut=5.0)
    assert np.allclose(U2, 2.0 * U, rtol=1e-14, atol=1e-16)
