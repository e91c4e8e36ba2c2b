"""Pins of the FP64 oracle against things other than itself: closed forms,
hand-derived cases, invariants, brute force and library routines (numpy SVD,
scipy distances).  CPU only."""
import os

import numpy as np
import pytest

import hh_synth
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rpy_golden():
    rows, self_v = [], None
    for line in open(os.path.join(GOLD, "rpy_values.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        if parts[0] == "self":
            self_v = float(parts[1])
        else:
            rows.append(tuple(float(x) for x in parts))
    return rows, self_v


# --------------------------------------------------------------------------
# pair kernel
# --------------------------------------------------------------------------
def test_rpy_closed_form_values():
    rows, self_v = _rpy_golden()
    k = oracle.PairKernel("rpy")
    for r, perp, par in rows:
        K = oracle.pair_block(k, [0.0, 0.0, r])       # r along z
        assert K[0, 0] == pytest.approx(perp, rel=2e-6)
        assert K[1, 1] == pytest.approx(perp, rel=2e-6)
        assert K[2, 2] == pytest.approx(par, rel=2e-6)
        assert abs(K[0, 1]) + abs(K[0, 2]) + abs(K[1, 2]) < 1e-15
    assert oracle.self_mobility(1.0, 1.0) == pytest.approx(self_v, rel=2e-6)


def test_rpy_continuity_and_symmetry():
    k = oracle.PairKernel("rpy")
    u = np.array([0.3, -0.5, 0.8]); u /= np.linalg.norm(u)
    below = oracle.pair_block(k, u * (2.0 - 1e-9))
    above = oracle.pair_block(k, u * (2.0 + 1e-9))
    assert np.max(np.abs(below - above)) < 1e-9
    K = oracle.pair_block(k, u * 3.7)
    assert np.allclose(K, K.T, rtol=1e-15, atol=0)
    assert np.allclose(K, oracle.pair_block(k, -u * 3.7), atol=1e-18)


def _affine_mlp(width, A, b, alpha=0.5, beta=0.7, gamma=0.9):
    """Parameters of 4 -> w -> w -> w -> 6 that compute o = A f + b exactly in
    exact arithmetic: SiLU(x) - SiLU(-x) = x, so a (+x, -x) unit pair passes x
    through a SiLU layer."""
    w = width
    W1 = np.zeros((w, 4)); W2 = np.zeros((w, w)); W3 = np.zeros((w, w)); W4 = np.zeros((6, w))
    for kk in range(4):
        W1[2 * kk, kk] = alpha
        W1[2 * kk + 1, kk] = -alpha
        for (W, s_in, s_out) in ((W2, alpha, beta), (W3, beta, gamma)):
            W[2 * kk, 2 * kk] = s_out / s_in
            W[2 * kk, 2 * kk + 1] = -s_out / s_in
            W[2 * kk + 1, 2 * kk] = -s_out / s_in
            W[2 * kk + 1, 2 * kk + 1] = s_out / s_in
        W4[:, 2 * kk] = A[:, kk] / gamma
        W4[:, 2 * kk + 1] = -A[:, kk] / gamma
    z = np.zeros(w)
    return np.concatenate([W1.ravel(), z, W2.ravel(), z, W3.ravel(), z, W4.ravel(), b])


def _sym(o):
    return np.array([[o[0], o[3], o[4]], [o[3], o[1], o[5]], [o[4], o[5], o[2]]])


@pytest.mark.parametrize("width", [32, 64])
def test_mlp_affine_network_closed_form(width):
    rng = np.random.default_rng(3)
    A = rng.normal(size=(6, 4)); b = rng.normal(size=6)
    th = _affine_mlp(width, A, b)
    assert len(th) == hh_synth.mlp_param_count(width)
    k = oracle.PairKernel("mlp", th, width, a=1.3)
    for _ in range(20):
        r = rng.normal(size=3) * rng.uniform(1, 50)
        d = np.linalg.norm(r)
        f = np.array([r[0] / d, r[1] / d, r[2] / d, 1.3 / d])
        want = _sym(A @ f + b) / d
        got = oracle.pair_block(k, r)
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_mlp_silu_unit():
    """A single SiLU unit in layer 3: o0 = SiLU(c f0) (paired pass-through in
    layers 1-2).  Pins the activation itself."""
    w = 32
    A = np.zeros((6, 4)); b = np.zeros(6)
    th = _affine_mlp(w, A, b, alpha=1.0, beta=1.0, gamma=1.0)
    # layer 3 unit 0 := 2.5 * (h2_0 - h2_1) = 2.5 f0, unit 1 := 0; output o0 = h3_0
    off3 = 4 * w + w + w * w + w
    W3 = np.zeros((w, w)); W3[0, 0] = 2.5; W3[0, 1] = -2.5
    th[off3:off3 + w * w] = W3.ravel()
    off4 = off3 + w * w + w
    W4 = np.zeros((6, w)); W4[0, 0] = 1.0
    th[off4:off4 + 6 * w] = W4.ravel()
    for f0 in (-0.9, -0.2, 0.3, 0.8):
        o = oracle.mlp_forward(th, w, [f0, 0.1, -0.2, 0.05])
        x = 2.5 * f0
        assert o[0] == pytest.approx(x / (1.0 + np.exp(-x)), rel=1e-14)
        assert np.all(o[1:] == 0.0)


def test_mlp_block_symmetric_and_translation_invariant():
    th = hh_synth.mlp_params(32, 11)
    k = oracle.PairKernel("mlp", th, 32)
    rng = np.random.default_rng(0)
    X = hh_synth.rsa_cube(60, 0.1)
    F = rng.normal(size=(60, 3))
    U1 = oracle.dense_matvec(X, F, k)
    U2 = oracle.dense_matvec(X + np.array([13.25, -7.5, 101.0]), F, k)
    assert np.max(np.abs(U1 - U2)) < 1e-12 * np.max(np.abs(U1))
    K = oracle.pair_block(k, [1.0, 2.0, -3.0])
    assert np.array_equal(K, K.T)


# --------------------------------------------------------------------------
# dense product
# --------------------------------------------------------------------------
def test_dense_constant_network_against_scipy_distances():
    from scipy.spatial.distance import cdist

    w = 32
    b = np.array([1.0, 2.0, 0.5, 0.25, -0.5, 0.75])
    th = np.concatenate([np.zeros(hh_synth.mlp_param_count(w) - 6), b])
    k = oracle.PairKernel("mlp", th, w)
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 20, size=(50, 3))
    F = rng.normal(size=(50, 3))
    D = cdist(X, X)
    np.fill_diagonal(D, np.inf)
    want = (1.0 / D) @ F @ _sym(b).T + F / (6 * np.pi)
    got = oracle.dense_matvec(X, F, k)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_dense_two_particles_rpy():
    rows, self_v = _rpy_golden()
    k = oracle.PairKernel("rpy")
    X = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 5.0]])
    F = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 3.0]])
    U = oracle.dense_matvec(X, F, k)
    perp, par = rows[1][1], rows[1][2]
    assert U[0, 0] == pytest.approx(self_v, rel=2e-6)
    assert U[0, 1] == pytest.approx(2.0 * perp, rel=2e-6)
    assert U[0, 2] == pytest.approx(3.0 * par, rel=2e-6)


def test_dense_matrix_consistency_and_rpy_symmetry():
    X = hh_synth.rsa_cube(40, 0.1)
    F = hh_synth.forces(40, 2)
    kr = oracle.PairKernel("rpy")
    M = oracle.dense_matrix(X, kr)
    assert np.max(np.abs(M - M.T)) <= 1e-15 * np.max(np.abs(M))
    assert np.allclose(M @ F.ravel(), oracle.dense_matvec(X, F, kr).ravel(), rtol=1e-13, atol=1e-15)
    km = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 5), 32)
    Mm = oracle.dense_matrix(X, km)
    assert np.allclose(Mm @ F.ravel(), oracle.dense_matvec(X, F, km).ravel(), rtol=1e-12, atol=1e-14)
    rows = np.array([3, 17, 39])
    assert np.allclose(oracle.dense_matvec(X, F, km, rows=rows), oracle.dense_matvec(X, F, km)[rows], rtol=0, atol=0)


# --------------------------------------------------------------------------
# Morton order and tree
# --------------------------------------------------------------------------
def test_morton_hand_derived():
    X = np.array([[0, 0, 0], [1, 1, 1], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.5, 0, 0]], dtype=float)
    c = oracle.morton_codes(X)
    ones = (8 ** 21 - 1) // 7          # 0b001001...001 (21 groups)
    assert int(c[0]) == 0
    assert int(c[1]) == 7 * ones == 2 ** 63 - 1
    assert int(c[2]) == 4 * ones
    assert int(c[3]) == 2 * ones
    assert int(c[4]) == ones
    assert int(c[5]) == 2 ** 62          # x = 1/2 -> q_x = 2^20: only the top x bit
    perm, sc = oracle.morton_sort(c)
    assert list(perm) == [0, 4, 3, 5, 2, 1] and np.all(np.diff(sc.astype(np.float64)) >= 0)


def test_morton_sort_stable_on_ties():
    X = np.array([[0.1, 0.1, 0.1]] * 3 + [[5.0, 5.0, 5.0]] + [[0.1, 0.1, 0.1]])
    perm, _ = oracle.morton_sort(oracle.morton_codes(X))
    assert list(perm) == [0, 1, 2, 4, 3]


def test_tree_1d_grid_is_dyadic():
    """16 points evenly spaced on a line: Morton bisection halves every range
    (the 1-D cluster tree of Fig. 4)."""
    X = np.zeros((16, 3)); X[:, 0] = (np.arange(16) + 0.5) / 16
    t = oracle.build_tree(X, leaf=2)
    want = [(0, 16)]
    for lvl in range(4):
        want += [(i * (16 >> (lvl + 1)), (i + 1) * (16 >> (lvl + 1))) for i in range(2 ** (lvl + 1))]
    assert list(zip(t.begin.tolist(), t.end.tolist())) == want


def test_tree_invariants():
    X = hh_synth.rsa_cube(3000, 0.1, seed=9)
    leaf = 16
    t = oracle.build_tree(X, leaf)
    assert t.begin[0] == 0 and t.end[0] == 3000
    for i in range(t.n_nodes):
        sz = t.size(i)
        assert sz >= 1
        pts = t.Xs[t.begin[i]:t.end[i]]
        assert np.array_equal(t.lo[i], pts.min(0)) and np.array_equal(t.hi[i], pts.max(0))
        c0, c1 = t.child[i]
        if c0 < 0:
            assert sz < leaf
        else:
            assert sz >= leaf and c1 == c0 + 1 and c0 > i
            assert t.begin[c0] == t.begin[i] and t.end[c0] == t.begin[c1] and t.end[c1] == t.end[i]
            assert t.parent[c0] == i and t.parent[c1] == i
    leaves = [i for i in range(t.n_nodes) if t.child[i, 0] < 0]
    assert sum(t.size(i) for i in leaves) == 3000
    assert np.array_equal(np.sort(t.perm), np.arange(3000))


# --------------------------------------------------------------------------
# partition
# --------------------------------------------------------------------------
def test_partition_1d_hand_derived():
    """8 unit-spaced points on a line, C_leaf = 2, eta = 1.  By hand: every
    single-point diagonal pair is inadmissible, everything else is admissible
    at the coarsest level Algorithm 1 reaches (including the touching pair
    ([2,4), [4,6)) where diam = dist = 1)."""
    X = np.zeros((8, 3)); X[:, 0] = np.arange(8.0)
    t = oracle.build_tree(X, leaf=2)
    G, H = oracle.partition(t, leaf=2, eta=1.0)
    rng = lambda i: (int(t.begin[i]), int(t.end[i]))
    gH = sorted((rng(a), rng(b)) for a, b in H)
    gG = sorted((rng(a), rng(b)) for a, b in G)
    assert gH == sorted(((i, i + 1), (i, i + 1)) for i in range(8))
    want = []
    for base in (0, 4):
        for a, b in ((0, 1), (1, 0), (2, 3), (3, 2)):
            want.append(((base + a, base + a + 1), (base + b, base + b + 1)))
        want += [((base, base + 2), (base + 2, base + 4)), ((base + 2, base + 4), (base, base + 2))]
    for a in ((0, 2), (2, 4)):
        for b in ((4, 6), (6, 8)):
            want += [(a, b), (b, a)]
    assert gG == sorted(want)


@pytest.mark.parametrize("eta", [0.7, 1.0, 1.5])
def test_partition_exact_cover_symmetry_bruteforce(eta):
    n, leaf = 180, 8
    X = hh_synth.rsa_cube(n, 0.1, seed=4)
    t = oracle.build_tree(X, leaf)
    G, H = oracle.partition(t, leaf, eta)
    cover = np.zeros((n, n), np.int32)
    for (a, b) in np.concatenate([G, H]):
        cover[t.begin[a]:t.end[a], t.begin[b]:t.end[b]] += 1
    assert np.all(cover == 1)
    Gs = set(map(tuple, G.tolist())); Hs = set(map(tuple, H.tolist()))
    assert all((b, a) in Gs for a, b in Gs) and all((b, a) in Hs for a, b in Hs)
    # brute force Eq. 7 on every listed block, in the same squared form
    for a, b in Gs:
        da = np.sum((t.hi[a] - t.lo[a]) ** 2); db = np.sum((t.hi[b] - t.lo[b]) ** 2)
        gap = np.maximum(0, np.maximum(t.lo[b] - t.hi[a], t.lo[a] - t.hi[b]))
        assert np.sum(gap ** 2) > 0 and max(da, db) <= eta * eta * np.sum(gap ** 2)
    for a, b in Hs:
        assert t.size(a) < leaf and t.size(b) < leaf and not oracle.admissible(t, a, b, eta)
    assert list(G.tolist()) == sorted(G.tolist()) and list(H.tolist()) == sorted(H.tolist())


# --------------------------------------------------------------------------
# ACA
# --------------------------------------------------------------------------
def _dense_block(G):
    c, q = G.shape[:2]
    return G.transpose(0, 2, 1, 3).reshape(3 * c, 3 * q)


def _cq(res):
    l = res["rank"]
    C, Q = res["C"], res["Q"]
    return np.einsum("pmab,pnbc->mnac", C, Q) if l else 0.0


@pytest.mark.parametrize("r", [1, 3, 5])
def test_aca_exact_low_rank(r):
    rng = np.random.default_rng(r)
    c, q = 23, 17
    A = rng.normal(size=(r, c, 3, 3)); B = rng.normal(size=(r, q, 3, 3))
    G = np.einsum("kmab,knbc->mnac", A, B)
    res = oracle.aca_dense(G, eps=1e-10, max_rank=17)
    assert res["rank"] <= r + 1
    err = np.linalg.norm(_dense_block(G - _cq(res))) / np.linalg.norm(_dense_block(G))
    assert err < 1e-11


def _geo_block(n=1024, seed=5, width=32):
    X = hh_synth.rsa_cube(n, 0.1, seed=seed)
    t = oracle.build_tree(X, 32)
    G, _ = oracle.partition(t, 32, 1.0)
    sizes = [(t.size(a) * t.size(b), a, b) for a, b in G]
    _, a, b = max(sizes)
    k = oracle.PairKernel("mlp", hh_synth.mlp_params(width, 7), width)
    c, q = t.size(a), t.size(b)
    Gm = np.zeros((c, q, 3, 3))
    for m in range(c):
        for nn in range(q):
            Gm[m, nn] = oracle.pair_block(k, t.Xs[t.begin[a] + m] - t.Xs[t.begin[b] + nn])
    return k, t, a, b, Gm


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-6])
def test_aca_vs_svd_and_lambda(eps):
    k, t, a, b, Gm = _geo_block()
    c, q = Gm.shape[:2]
    res = oracle.aca_block(k, t.Xs, int(t.begin[a]), c, int(t.begin[b]), q, eps, 48)
    l = res["rank"]
    CQ = _cq(res)
    D = _dense_block(Gm)
    err = np.linalg.norm(_dense_block(Gm - CQ))
    # Algorithm 2's lambda^2 recurrence equals |CQ|_F^2 formed explicitly
    assert res["lambda2"] == pytest.approx(np.linalg.norm(_dense_block(CQ)) ** 2, rel=1e-10)
    # ACA error within a small multiple of zeta (Eq. 10 estimate)
    assert err <= 10 * eps * np.linalg.norm(D)
    # Eckart-Young: no rank-3l matrix beats the truncated SVD
    s = np.linalg.svd(D, compute_uv=False)
    assert np.sqrt(np.sum(s[3 * l:] ** 2)) <= err * (1 + 1e-9)
    # the ACA block agrees with the geometric entries on its pivot rows/columns
    for p in range(l):
        i = res["I"][p]
        assert np.allclose(CQ[i], Gm[i], rtol=0, atol=1e-10 * np.abs(Gm).max())


def test_aca_rank_grows_as_eps_falls():
    k, t, a, b, Gm = _geo_block()
    c, q = Gm.shape[:2]
    ranks = [oracle.aca_block(k, t.Xs, int(t.begin[a]), c, int(t.begin[b]), q, e, 48)["rank"]
             for e in (1e-2, 1e-4, 1e-6)]
    assert ranks[0] < ranks[1] < ranks[2]


# --------------------------------------------------------------------------
# ACA pivot guard (Algorithm 2 with the determinant fallback) and the
# randomised j_1 of Algorithm 2 (rule 1)
# --------------------------------------------------------------------------
def _fallback_block(P00, col1):
    """3 x 2 block whose first column (j_1 = 0) is given element by element."""
    rng = np.random.default_rng(11)
    G = np.zeros((3, 2, 3, 3))
    for m in range(3):
        G[m, 0] = P00[m]
        G[m, 1] = col1[m] if col1 is not None else rng.normal(size=(3, 3))
    return G


def test_aca_fallback_takes_largest_det():
    # column 0: row 0 has the largest Frobenius norm (10) but is singular;
    # row 1 is second by norm (|.|_F ~ 3.00, det 0.03); row 2 has the largest
    # |det| (3.375).  The guard must take row 2 -- not the smallest |det|
    # (row 0) and not the next row by norm (row 1).
    P = [np.diag([10.0, 0.0, 0.0]), np.diag([3.0, 0.1, 0.1]), 1.5 * np.eye(3)]
    G = _fallback_block(P, None)
    res = oracle.aca_dense(G, eps=1e-4, max_rank=8)
    assert res["I"][0] == 2 and res["J"][0] == 0
    assert np.allclose(res["C"][0, 2], np.eye(3), atol=1e-15)      # c_0 scaled by its pivot's inverse
    # two column steps reach k = min(c, q): the 9 x 6 scalar matrix is reproduced
    D = _dense_block(G)
    assert np.linalg.norm(_dense_block(G - _cq(res))) <= 10 * 1e-4 * np.linalg.norm(D)


def test_aca_fallback_on_ill_conditioned_pivot():
    # row 0 is the Frobenius-best and non-singular (det 1e-8) but its
    # reciprocal condition number 1/(|P|_F |P^-1|_F) ~ 7e-12 is below 1e-10:
    # the guard replaces it by the eligible row of largest |det| (row 2, det 3.375)
    P = [np.diag([10.0, 10.0, 1e-10]), np.diag([3.0, 0.1, 0.1]), 1.5 * np.eye(3)]
    res = oracle.aca_dense(_fallback_block(P, None), eps=1e-4, max_rank=8)
    assert res["I"][0] == 2
    # just above the threshold (rc ~ 7e-10) the Frobenius-best row is kept
    P[0] = np.diag([10.0, 10.0, 1e-8])
    res = oracle.aca_dense(_fallback_block(P, None), eps=1e-4, max_rank=8)
    assert res["I"][0] == 0


def test_aca_fallback_without_usable_pivot_stops():
    # every element of the first column is singular: no eligible row has
    # |det| > 0, so the block ends with the pairs found so far (none)
    P = [np.diag([10.0, 0.0, 0.0]), np.diag([0.0, 3.0, 0.0]), np.diag([0.0, 0.0, 1.0])]
    res = oracle.aca_dense(_fallback_block(P, None), eps=1e-4, max_rank=8)
    assert res["rank"] == 0


def test_aca_fallback_skips_used_rows():
    # Step 0 takes row 0 (the only non-zero row of column 0); its scaled
    # element C_0(0) = P P^-1 is the identity up to rounding.  At step 1 the
    # column residual of the used row 0 is that rounding noise (tiny but of
    # full rank), while the unused rows 1..3 are exactly singular: the guard
    # finds no eligible pivot and stops at rank 1.  A guard that forgot the
    # used-row test would take row 0 a second time.
    rng = np.random.default_rng(3)
    G = np.zeros((4, 3, 3, 3))
    G[0, 0] = 10.0 * rng.normal(size=(3, 3))
    G[0, 1] = 5.0 * rng.normal(size=(3, 3))
    G[0, 2] = 0.1 * rng.normal(size=(3, 3))
    for m, a in zip((1, 2, 3), (3.0, 2.0, 1.0)):
        G[m, 1] = np.diag([a, 0.0, 0.0])
    res = oracle.aca_dense(G, eps=1e-6, max_rank=8)
    assert res["rank"] == 1 and res["I"][0] == 0 and res["J"][0] == 0


_SPLITMIX64_SEED0 = (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC)


def test_j1_rule1_is_splitmix64():
    # Rule 1 draws j_1 = splitmix64(seed ^ (tau << 32) ^ sigma) mod q.  The
    # published SplitMix64 stream started from state 0 gives outputs
    # mix(n * gamma), n = 1, 2, ...; with tau = sigma = 0 and seed = (n-1) gamma
    # the oracle must return output n mod q.  Four moduli whose product
    # exceeds 2^64 pin every bit of each output.
    gamma, mask = 0x9E3779B97F4A7C15, (1 << 64) - 1
    for n, out in enumerate(_SPLITMIX64_SEED0):
        seed = (n * gamma) & mask
        for q in (2 ** 31 - 1, 1000003, 65536, 97):
            assert oracle.j1(1, seed, 0, 0, q) == out % q
    # tau enters shifted by 32 bits and sigma unshifted, both xor-ed into the seed
    t, s = 5, 7
    seed = gamma ^ (t << 32) ^ s
    assert oracle.j1(1, seed, t, s, 1000003) == _SPLITMIX64_SEED0[1] % 1000003
    assert oracle.j1(1, seed, s, t, 1000003) != _SPLITMIX64_SEED0[1] % 1000003
    # rule 0 and one-column blocks give the first source
    assert oracle.j1(0, seed, t, s, 1000003) == 0
    assert oracle.j1(1, seed, t, s, 1) == 0


# --------------------------------------------------------------------------
# H-matrix product
# --------------------------------------------------------------------------
def test_hmatvec_exact_when_nothing_far():
    X = hh_synth.rsa_cube(300, 0.1, seed=2)
    F = hh_synth.forces(300, 0)
    k = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 7), 32)
    Ud = oracle.dense_matvec(X, F, k)
    Uh, st = oracle.hmatvec(X, F, k, leaf=16, eta=1e-9, eps=1e-4)
    assert oracle.rel_error(Ud, Uh) < 1e-12


def test_hmatvec_error_bounded_by_zeta():
    X = hh_synth.rsa_cube(1024, 0.1)
    F = hh_synth.forces(1024, 0)
    for kind in ("mlp", "rpy"):
        k = oracle.PairKernel(kind, hh_synth.mlp_params(32, 7), 32)
        Ud = oracle.dense_matvec(X, F, k, with_self=False)
        errs = []
        for eps in (1e-3, 1e-4, 1e-6):
            Uh, st = oracle.hmatvec(X, F, k, leaf=32, eta=1.0, eps=eps, with_self=False)
            errs.append(oracle.rel_error(Ud, Uh))
            assert errs[-1] <= eps
            assert st["nG"] > 0 and st["rank_capped"] == 0
        assert errs[0] > errs[1] > errs[2]


# --------------------------------------------------------------------------
# gradients and training
# --------------------------------------------------------------------------
def test_dense_grad_finite_differences():
    n = 30
    X = hh_synth.rsa_cube(n, 0.1, seed=12)
    F = hh_synth.forces(n, 1)
    W = hh_synth.forces(n, 2)
    th = hh_synth.mlp_params(32, 4).astype(np.float64)
    k = oracle.PairKernel("mlp", th, 32)
    gF, gX, gT = oracle.dense_grad(X, F, W, k)
    L = lambda X_, F_, t_: float(np.sum(W * oracle.dense_matvec(X_, F_, oracle.PairKernel("mlp", t_, 32))))
    h = 1e-6
    for (i, a) in ((0, 0), (7, 2), (29, 1)):
        Xp = X.copy(); Xp[i, a] += h; Xm = X.copy(); Xm[i, a] -= h
        assert gX[i, a] == pytest.approx((L(Xp, F, th) - L(Xm, F, th)) / (2 * h), rel=1e-6, abs=1e-9)
        Fp = F.copy(); Fp[i, a] += h; Fm = F.copy(); Fm[i, a] -= h
        assert gF[i, a] == pytest.approx((L(X, Fp, th) - L(X, Fm, th)) / (2 * h), rel=1e-6, abs=1e-9)
    for p in (0, 130, 600, 2000, 2469):
        tp = th.copy(); tp[p] += h; tm = th.copy(); tm[p] -= h
        assert gT[p] == pytest.approx((L(X, F, tp) - L(X, F, tm)) / (2 * h), rel=1e-5, abs=1e-8)
    # gF is M^T W
    M = oracle.dense_matrix(X, k)
    assert np.allclose(gF.ravel(), M.T @ W.ravel(), rtol=1e-12, atol=1e-14)


def test_train_loss_grad_and_adam():
    rng = np.random.default_rng(8)
    B = 16
    r = rng.normal(size=(B, 3)) * 5
    e = np.eye(3)[rng.integers(0, 3, B)]
    U = rng.normal(size=(B, 3)) * 0.01
    th = hh_synth.mlp_params(32, 3).astype(np.float64)
    L, g = oracle.train_loss_grad(th, 32, r, e, U)
    h = 1e-6
    for p in (5, 400, 2465):
        tp = th.copy(); tp[p] += h; tm = th.copy(); tm[p] -= h
        fd = (oracle.train_loss_grad(tp, 32, r, e, U, grad=False) - oracle.train_loss_grad(tm, 32, r, e, U, grad=False)) / (2 * h)
        assert g[p] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # Adam, first step from zero moments: theta -= lr * g / (|g| + eps)
    t2 = th.copy(); m = np.zeros_like(th); v = np.zeros_like(th)
    oracle.adam_step(t2, g, m, v, 1, lr=1e-3)
    assert np.allclose(t2, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_dense_matvec_multi_equals_single():
    # several force vectors share each pair block's evaluation but keep the
    # single-vector summation order, so every product is bit-identical
    X = hh_synth.rsa_cube(400, 0.1, seed=31)
    k = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 7), 32)
    Fs = np.stack([hh_synth.forces(400, s) for s in range(5)])
    rows = np.array([0, 7, 123, 399])
    Um = oracle.dense_matvec_multi(X, Fs, k, rows=rows, with_self=False)
    for f in range(5):
        assert np.array_equal(Um[f], oracle.dense_matvec(X, Fs[f], k, rows=rows, with_self=False))
    assert np.array_equal(oracle.dense_matvec_multi(X, Fs[:1], k)[0], oracle.dense_matvec(X, Fs[0], k))


# --------------------------------------------------------------------------
# SVD recompression of a block's factors
# --------------------------------------------------------------------------
def _factors_of(M, c, q):
    """3x3 factors C [l, c, 3, 3], Q [l, q, 3, 3] whose block_matrix is M
    (3c x 3q), with l = 3c / 3 = c steps of an exact split M = I M."""
    l = c
    Cs = np.eye(3 * c)
    C = Cs.reshape(c, 3, l, 3).transpose(2, 0, 1, 3)
    Q = M.reshape(l, 3, q, 3).transpose(0, 2, 1, 3)
    return C, Q


def test_recompress_prescribed_singular_values():
    # M = P diag(s) R^T with orthonormal P, R: the kept rank is the one the
    # tail rule gives and the error equals the discarded tail (Eckart-Young)
    rng = np.random.default_rng(3)
    c, q = 6, 5
    P, _ = np.linalg.qr(rng.standard_normal((3 * c, 15)))
    R, _ = np.linalg.qr(rng.standard_normal((3 * q, 15)))
    s = 10.0 ** -np.arange(15, dtype=float) * 3.0
    M = (P * s) @ R.T
    C, Q = _factors_of(M, c, q)
    assert np.allclose(oracle.block_matrix(C, Q), M, rtol=0, atol=1e-14)
    # tail(r) / ||M|| = 10^-r exactly for this geometric spectrum
    for eps, r_want in ((2e-3, 3), (5e-6, 6), (0.0, 15)):
        U, V, r, sv = oracle.recompress(C, Q, eps)
        tail = np.sqrt(np.sum(s[r_want:] ** 2))
        assert r == r_want and U.shape == (3 * c, r) and V.shape == (r, 3 * q)
        assert np.allclose(sv[:15], s, rtol=1e-10)
        assert abs(np.linalg.norm(M - U @ V) - tail) <= 1e-12 * np.linalg.norm(M) + 1e-9 * tail
        assert tail <= eps * np.linalg.norm(M) + 1e-15


def test_recompress_aca_blocks():
    # on ACA blocks of the MLP kernel: rank <= 3 l, error within eps_rc, and
    # the scalar rank is below the 3 l the 3x3 steps give
    X = hh_synth.rsa_cube(1500, 0.1, seed=12)
    k = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 7), 32)
    t = oracle.build_tree(X, 32)
    G, _ = oracle.partition(t, 32, 1.0)
    fewer = 0
    for tau, sig in G[:: max(1, len(G) // 40)]:
        t0, c, s0, q = int(t.begin[tau]), int(t.size(tau)), int(t.begin[sig]), int(t.size(sig))
        a = oracle.aca_block(k, t.Xs, t0, c, s0, q, 1e-6, 48, 0)
        l = a["rank"]
        M = oracle.block_matrix(a["C"], a["Q"])
        U, V, r, _ = oracle.recompress(a["C"], a["Q"], 1e-4)
        assert r <= 3 * l
        assert np.linalg.norm(M - U @ V) <= 1e-4 * np.linalg.norm(M) * (1 + 1e-12)
        fewer += r < 3 * l
    assert fewer > 0
