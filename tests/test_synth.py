"""The seeded input generators: each one against the property it promises.

These inputs feed both the CUDA path and the oracle, so a generator that
silently breaks its contract (overlapping spheres, weights that are not
bf16-exact, a shifted random stream) would weaken every parity test without
failing any of them."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import hh_synth


def test_splitmix64_published_outputs():
    # SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), state seeded with 0: the
    # first outputs of the public reference generator
    z = hh_synth.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # counter based: any window of the stream recomputes the same values
    assert np.array_equal(hh_synth.splitmix64(7, 10)[4:], hh_synth.splitmix64(7, 6, start=4))
    u = hh_synth.uniform01(3, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-8, 8, 20000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, -7.5e-39]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(hh_synth.round_bf16(x), ref)


@pytest.mark.parametrize("width", [32, 64])
def test_mlp_params_xavier_and_bf16_exact(width):
    th = hh_synth.mlp_params(width, 11)
    assert th.size == hh_synth.mlp_param_count(width) == 2 * width * width + 13 * width + 6
    assert np.array_equal(hh_synth.round_bf16(th).astype(np.float64), th)      # bf16-representable
    dims = [4, width, width, width, 6]
    o = 0
    for i in range(4):
        nin, nout = dims[i], dims[i + 1]
        W = th[o:o + nin * nout]
        b = th[o + nin * nout:o + nin * nout + nout]
        lim = math.sqrt(6.0 / (nin + nout))
        assert np.abs(W).max() <= lim * (1 + 2 ** -8) and np.abs(W).max() > 0.5 * lim
        assert np.all(b == 0.0)
        o += nin * nout + nout
    assert o == th.size
    assert not np.array_equal(th, hh_synth.mlp_params(width, 12))


def test_rsa_cube_no_overlap_inside_and_seeded():
    n, phi = 4000, 0.1
    X = hh_synth.rsa_cube(n, phi, seed=5)
    L = hh_synth.cube_side(n, phi)
    assert abs(n * 4.0 / 3.0 * math.pi / L ** 3 - phi) < 1e-12
    assert X.shape == (n, 3) and X.min() >= 0.0 and X.max() <= L
    assert len(cKDTree(X).query_pairs(2.0 - 1e-12)) == 0                       # centres >= 2a apart
    assert np.array_equal(X, hh_synth.rsa_cube(n, phi, seed=5))
    assert not np.array_equal(X, hh_synth.rsa_cube(n, phi, seed=6))


def test_gaussian_cloud_width_rule():
    n = 20000
    smin = hh_synth.sigma_min(n)
    assert abs(n * 4.0 / 3.0 * math.pi / ((2 * math.pi) ** 1.5 * smin ** 3) - 0.25) < 1e-12   # peak phi
    X, s = hh_synth.gaussian_cloud(n, 20.0, seed=3)
    assert s == max(20.0, smin)
    assert len(cKDTree(X).query_pairs(2.0 - 1e-12)) == 0
    # overlap rejection turns candidates away from the dense core (peak phi
    # 0.25), so the accepted cloud is somewhat wider than the drawn sigma
    w = np.std(X - X.mean(0)) / s
    assert 1.0 <= w <= 1.15
    X2, s2 = hh_synth.gaussian_cloud(2000, 30.0, seed=3)                        # feasible: sigma kept
    assert s2 == 30.0
    assert abs(np.std(X2 - X2.mean(0)) / s2 - 1.0) < 0.03                       # dilute: the drawn width


def test_two_particle_samples_ranges():
    r, e = hh_synth.two_particle_samples(5000, 9, dmin=2.0, dmax=1000.0)
    d = np.linalg.norm(r, axis=1)
    assert d.min() >= 2.0 and d.max() <= 1000.0
    assert abs(np.mean(np.log(d)) - 0.5 * (np.log(2.0) + np.log(1000.0))) < 0.1    # log-uniform
    assert np.all(np.sort(e, axis=1)[:, :2] == 0.0) and np.all(e.sum(1) == 1.0)    # unit axis forces


def test_forces_and_perturb():
    F = hh_synth.forces(100000, 2)
    assert F.shape == (100000, 3) and abs(F.mean()) < 0.01 and abs(F.std() - 1.0) < 0.01
    X = np.zeros((1000, 3))
    P = hh_synth.perturb(X, 0.05, seed=1)
    assert abs(P.std() - 0.05) < 0.005 and np.array_equal(P, hh_synth.perturb(X, 0.05, seed=1))


def test_lattice_drop_has_the_papers_particle_count():
    # Section 4.3: each drop is the primitive cubic lattice inside a sphere of
    # radius 175 at ~10% volume fraction, 523,305 particles (two drops:
    # 1,046,610).  Spacing 3.5 gives exactly that count: the integer points
    # of a ball of radius 50 lattice units.
    P = hh_synth.lattice_sphere(175.0, 3.5)
    assert len(P) == 523305
    m = np.arange(-50, 51)
    assert int(np.sum((m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2) <= 2500)) == 523305
    assert abs((4.0 / 3.0) * math.pi / 3.5 ** 3 - 0.1) < 0.003          # the volume fraction of the lattice
    d, _ = cKDTree(P).query(P, k=2)
    assert d[:, 1].min() > 2.0                                          # jitter 0.2 keeps spheres apart
    assert np.linalg.norm(P, axis=1).max() <= 175.0 + 0.2 * math.sqrt(3)
    assert np.array_equal(P, hh_synth.lattice_sphere(175.0, 3.5))       # seeded
    D = hh_synth.two_drops()
    assert len(D) == 1046610
    assert np.allclose(D[:523305].mean(0), [0, 0, 525.0], atol=0.05) and np.allclose(D[523305:].mean(0), 0, atol=0.05)


def test_lattice_subset_fixed_domain():
    P = hh_synth.lattice_cube(10, 3.5)
    assert len(P) == 1000 and np.all(P > -0.21) and np.all(P < 9 * 3.5 + 0.21)
    S = hh_synth.lattice_subset(300, n_side=10, subset_seed=3)
    assert len(S) == 300 and len(np.unique(S, axis=0)) == 300
    assert len({tuple(r) for r in S} & {tuple(r) for r in P}) == 300  # rows of the lattice, in lattice order
    assert not np.array_equal(S, hh_synth.lattice_subset(300, n_side=10, subset_seed=4))


def test_filament_sphere_layout():
    # the paper's filament suspension, scaled down: chains straight with bead
    # spacing r_b inside R_in, free particles in the shell, gaps >= 2.1
    n_fil, beads, n_free = 60, 21, 1260
    X, r_in, r_out = hh_synth.filament_sphere(n_fil, beads, 3.0, n_free, seed=5)
    assert X.shape == (n_fil * beads + n_free, 3)
    assert r_out == pytest.approx(4 * 10 ** (1 / 3) * 20 * 3.0) and r_in == pytest.approx(0.5 ** (1 / 3) * r_out)
    C = X[:n_fil * beads].reshape(n_fil, beads, 3)
    seg = np.diff(C, axis=1)
    assert np.allclose(np.linalg.norm(seg, axis=2), 3.0)
    t = seg / 3.0
    assert np.allclose(np.einsum("cbi,cbi->cb", t[:, 1:], t[:, :-1]), 1.0)       # straight
    assert np.linalg.norm(C, axis=2).max() <= r_in + 1e-9
    rf = np.linalg.norm(X[n_fil * beads:], axis=1)
    assert rf.min() >= r_in - 1e-9 and rf.max() <= r_out + 1e-9
    d, i = cKDTree(X).query(X, k=2)
    assert d[:, 1].min() >= 2.1 - 1e-9
