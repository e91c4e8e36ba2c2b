"""Parity of the CUDA path (through the C-ABI) against the FP64 CPU oracle.

Integer/index results (Morton codes, permutation, tree, block lists) must be
bit-identical.  Velocities: FP64 mode against the oracle's H-matrix product to
1e-2 * zeta relative: the arithmetic agrees to rounding, but a pivot whose two
candidates tie to rounding may flip, which swaps one valid rank-l block for
another that differs at the zeta level in that block only (observed 5e-10 for
the MLP kernel and 4e-7 for RPY at zeta = 1e-4).  FP32 mode to 2e-5 relative of the oracle's H-matrix product
(FP32 rounding of ~10^3-term sums, observed ~1e-6) and to eps_r <= zeta
against the exact dense product (Eq. 11, the paper's own bound).
"""
import numpy as np
import pytest

import hh_synth
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402

THETA32 = hh_synth.mlp_params(32, 7)
THETA64 = hh_synth.mlp_params(64, 7)


@pytest.fixture(scope="module")
def ctx():
    c = hh.Context()
    c.set_mlp(THETA32, 32)
    return c


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def kern(kind="mlp", width=32):
    return oracle.PairKernel(kind, THETA32 if width == 32 else THETA64, width)


# --------------------------------------------------------------------------
# tree and partition: bit-exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,leaf", [(1, 32), (2, 2), (31, 32), (32, 32), (33, 32), (1024, 32), (5000, 16),
                                    (3000, 64)])
def test_tree_bit_exact(ctx, n, leaf):
    X = hh_synth.rsa_cube(n, 0.1, seed=n) if n > 1 else np.array([[1.0, 2.0, 3.0]])
    t = ctx.build_tree(cuda(X), hh.Params(leaf_size=leaf))
    g = t.export()
    o = oracle.build_tree(X, leaf)
    assert np.array_equal(g["perm"], o.perm)
    assert np.array_equal(g["codes"], o.codes)
    assert np.array_equal(g["begin"], o.begin) and np.array_equal(g["end"], o.end)
    assert np.array_equal(g["child"], o.child)
    assert np.array_equal(g["lo"], o.lo) and np.array_equal(g["hi"], o.hi)


def test_tree_duplicate_codes_and_degenerate_extent(ctx):
    # 40 points on 2 sites (equal codes force the begin + size/2 split) and a flat plane
    X = np.zeros((40, 3)); X[20:, 0] = 1.0
    Y = np.random.default_rng(0).uniform(0, 10, size=(200, 3)); Y[:, 2] = 5.0
    for A in (X, Y):
        g = ctx.build_tree(cuda(A), hh.Params(leaf_size=8)).export()
        o = oracle.build_tree(A, 8)
        assert np.array_equal(g["perm"], o.perm) and np.array_equal(g["begin"], o.begin)
        assert np.array_equal(g["child"], o.child) and np.array_equal(g["lo"], o.lo)


@pytest.mark.parametrize("eta", [0.7, 1.0, 1.5])
def test_partition_bit_exact(ctx, eta):
    X = hh_synth.rsa_cube(4096, 0.1, seed=3)
    p = hh.Params(leaf_size=32, eta=eta)
    t = ctx.build_tree(cuda(X), p)
    G, H = ctx.partition(t, p).export()
    ot = oracle.build_tree(X, 32)
    oG, oH = oracle.partition(ot, 32, eta)
    assert np.array_equal(G, oG) and np.array_equal(H, oH)


def test_batch_tree_matches_instances(ctx):
    sizes = [700, 1, 1500, 64]
    Xs = [hh_synth.rsa_cube(s, 0.1, seed=10 + i) if s > 1 else np.array([[0.5, 0.5, 0.5]])
          for i, s in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    g = ctx.build_tree(cuda(np.concatenate(Xs)), hh.Params(leaf_size=32), offsets=off).export()
    for b, X in enumerate(Xs):
        o = oracle.build_tree(X, 32)
        assert np.array_equal(g["perm"][off[b]:off[b + 1]] - off[b], o.perm)
        assert np.array_equal(g["codes"][off[b]:off[b + 1]], o.codes)
        # node ranges of this instance (the forest interleaves instances level by level)
        mine = (g["begin"] >= off[b]) & (g["end"] <= off[b + 1])
        rng_g = sorted(zip((g["begin"][mine] - off[b]).tolist(), (g["end"][mine] - off[b]).tolist()))
        assert rng_g == sorted(zip(o.begin.tolist(), o.end.tolist()))


# --------------------------------------------------------------------------
# ACA pivots and ranks (FP64 mode)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("j1_rule", [0, 1])
def test_aca_fp64_ranks_and_pivots(ctx, j1_rule):
    X = hh_synth.rsa_cube(2048, 0.1, seed=5)
    F = hh_synth.forces(2048, 0)
    p = hh.Params(precision="fp64", eps=1e-4, max_rank=48, j1_rule=j1_rule, seed=77)
    t = ctx.build_tree(cuda(X), p)
    b = ctx.partition(t, p)
    h = ctx.aca(t, b, p)
    ranks, pI, pJ = h.export()
    _, st = oracle.hmatvec(X, F, kern(), leaf=32, eta=1.0, eps=1e-4, max_rank=48, j1_rule=j1_rule, seed=77,
                           want_ranks=True)
    same = (ranks == st["ranks"]) & np.all(pI == st["pivI"], axis=1) & np.all(pJ == st["pivJ"], axis=1)
    # rounding-level differences in the MLP may flip a near-tie; allow at most 0.5% of blocks
    assert same.mean() >= 0.995, f"{(~same).sum()} of {len(same)} blocks differ"
    assert ranks.sum() == pytest.approx(st["ranks"].sum(), rel=2e-3)
    if j1_rule == 1:   # the drawn first columns are used (not all zero)
        assert np.count_nonzero(pJ[:, 0]) > len(pJ) // 2
    # where the pivots agree, the factors themselves agree to rounding: C and
    # Q element by element against the oracle's Algorithm 2 on the same block
    ot = oracle.build_tree(X, 32)
    PG, _ = b.export()
    fofs, fac = h.export_factors()
    idx = np.flatnonzero(same & (ranks > 0))
    rng = np.random.default_rng(j1_rule)
    worst_line, worst_prod = 0.0, 0.0
    for bb in rng.choice(idx, size=min(150, len(idx)), replace=False):
        ta, sa = PG[bb]
        t0, c = int(ot.begin[ta]), int(ot.end[ta] - ot.begin[ta])
        s0, q = int(ot.begin[sa]), int(ot.end[sa] - ot.begin[sa])
        l = int(ranks[bb])
        j1 = oracle.j1(j1_rule, 77, int(ta), int(sa), q)
        ro = oracle.aca_block(kern(), ot.Xs, t0, c, s0, q, 1e-4, 48, j1)
        assert ro["rank"] == l
        base = int(fofs[bb]) * 9
        Cg = fac[base: base + l * 9 * c].reshape(l, 3, 3, c).transpose(0, 3, 1, 2)
        Qg = fac[base + l * 9 * c: base + l * 9 * (c + q)].reshape(l, 3, 3, q).transpose(0, 3, 1, 2)
        Go = np.einsum("pmab,pnbc->mnac", ro["C"], ro["Q"])
        Gg = np.einsum("pmab,pnbc->mnac", Cg, Qg)
        worst_prod = max(worst_prod, np.linalg.norm(Gg - Go) / np.linalg.norm(Go))
        # each rank term c_p q_p^T perturbed by the factor differences, against
        # the block's scale.  Looser than the product: a pivot element of
        # modest condition number turns rounding-level differences into term
        # differences that the later terms of the recursion absorb (observed
        # 1.2e-7 with the products still equal to 1e-11)
        scale = np.abs(Go).max()
        for pp in range(l):
            dC, dQ = np.abs(Cg[pp] - ro["C"][pp]).max(), np.abs(Qg[pp] - ro["Q"][pp]).max()
            term = dC * np.abs(ro["Q"][pp]).max() + np.abs(ro["C"][pp]).max() * dQ
            worst_line = max(worst_line, term / scale)
    print(f"j1 rule {j1_rule}: worst block product {worst_prod:.2e}, worst factor term {worst_line:.2e}")
    assert worst_prod < 1e-11, worst_prod
    assert worst_line < 1e-6, worst_line


# --------------------------------------------------------------------------
# velocities
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["mlp", "rpy"])
def test_predict_fp64_matches_oracle_hmatvec(ctx, kind):
    n = 2048
    X = hh_synth.rsa_cube(n, 0.1, seed=6)
    F = hh_synth.forces(n, 1)
    U = ctx.predict(cuda(X), cuda(F), hh.Params(precision="fp64", kernel=kind)).cpu().numpy()
    Uo, _ = oracle.hmatvec(X, F, kern(kind), leaf=32, eta=1.0, eps=1e-4, max_rank=48)
    assert oracle.rel_error(Uo, U) < 1e-6


FP32_FLOOR = 1e-5   # eps_r floor of FP32 arithmetic (observed 0.5-5e-6 at N = 1024)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-6])
def test_predict_against_dense(ctx, eps, prec):
    n = 1024
    X = hh_synth.rsa_cube(n, 0.1)
    ks = kern()
    errs = []
    a1 = oracle.self_mobility()
    for s in range(5):   # Eq. 11 averaged over 5 force vectors
        F = hh_synth.forces(n, s)
        U = ctx.predict(cuda(X), cuda(F), hh.Params(precision=prec, eps=eps)).cpu().numpy()
        Ud = oracle.dense_matvec(X, F, ks, with_self=True)
        errs.append(oracle.rel_error(Ud - a1 * F, U - a1 * F))
        if s == 0 and prec == "fp32":
            # the FP32 path does not invert singular values of a pivot element
            # below the noise floor of its FP32 residuals (2^-17 of the first
            # pivot's norm), where the FP64 oracle inverts them: a few terms
            # differ at that level (observed 2.9e-5 at zeta = 1e-3)
            Uo, _ = oracle.hmatvec(X, F, ks, leaf=32, eta=1.0, eps=eps, max_rank=48)
            assert oracle.rel_error(Uo, U) < 5e-5
    assert np.mean(errs) <= (eps if prec == "fp64" else max(eps, FP32_FLOOR))


def test_predict_ragged_and_tiny(ctx):
    a1 = oracle.self_mobility()
    for n in (1, 2, 3, 37, 257):
        X = hh_synth.rsa_cube(n, 0.1, seed=n) if n > 1 else np.array([[3.0, 1.0, 2.0]])
        F = hh_synth.forces(n, n)
        U = ctx.predict(cuda(X), cuda(F), hh.Params(precision="fp64")).cpu().numpy()
        Ud = oracle.dense_matvec(X, F, kern())
        assert oracle.rel_error(Ud, U) < 1e-12 if n < 64 else oracle.rel_error(Ud, U) < 1e-4
        if n == 1:
            assert np.allclose(U, a1 * F, rtol=1e-15)


def test_predict_width64(ctx):
    c = hh.Context()
    c.set_mlp(THETA64, 64)
    n = 1500
    X = hh_synth.rsa_cube(n, 0.1, seed=8)
    F = hh_synth.forces(n, 2)
    Uo, _ = oracle.hmatvec(X, F, kern("mlp", 64), leaf=64, eta=1.0, eps=1e-4, max_rank=48)
    for prec, tol in (("fp64", 1e-6), ("fp32", 2e-5)):
        U = c.predict(cuda(X), cuda(F), hh.Params(precision=prec, leaf_size=64)).cpu().numpy()
        assert oracle.rel_error(Uo, U) < tol


def test_staged_matvec_equals_predict_and_transpose_is_adjoint(ctx):
    n = 2048
    X = hh_synth.rsa_cube(n, 0.1, seed=9)
    F = hh_synth.forces(n, 3)
    W = hh_synth.forces(n, 4)
    p = hh.Params(precision="fp64")
    Xd = cuda(X)
    t = ctx.build_tree(Xd, p)
    b = ctx.partition(t, p)
    h = ctx.aca(t, b, p)
    U1 = ctx.matvec(h, cuda(F)).cpu().numpy()
    U2 = ctx.predict(Xd, cuda(F), p).cpu().numpy()
    assert oracle.rel_error(U2, U1) < 1e-13
    UT = ctx.matvec(h, cuda(W), transpose=True).cpu().numpy()
    lhs = np.sum(W * U1)
    rhs = np.sum(UT * F)
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(W * W) * np.sum(U1 * U1))


def test_shards_sum_to_whole(ctx):
    n = 3000
    X = hh_synth.rsa_cube(n, 0.1, seed=11)
    F = hh_synth.forces(n, 5)
    Xd, Fd = cuda(X), cuda(F)
    full = ctx.predict(Xd, Fd, hh.Params(precision="fp64")).cpu().numpy()
    parts = [ctx.predict(Xd, Fd, hh.Params(precision="fp64", shard_id=s, n_shards=3)).cpu().numpy()
             for s in range(3)]
    assert oracle.rel_error(full, sum(parts)) < 1e-14


def test_shard_split_is_cost_balanced():
    import bench
    # N = 100k, C_leaf 64: the split the shards use equals the definition, is
    # contiguous, and each shard's W^G / W^H is within one item of the mean
    c = hh.Context()
    c.set_mlp(THETA32, 32)
    n = 100000
    X = hh_synth.rsa_cube(n, 0.1, seed=17)
    p = hh.Params(precision="bf16", leaf_size=64)
    t = c.build_tree(cuda(X), p)
    b = c.partition(t, p)
    G, H = b.export()
    te = t.export()
    size = (te["end"] - te["begin"]).astype(np.int64)
    wg = np.maximum(size[G[:, 0]], size[G[:, 1]])
    wh = np.zeros(len(size), np.int64)
    np.add.at(wh, H[:, 0], size[H[:, 0]] * size[H[:, 1]])
    for ns in (2, 3, 8):
        bo, no = b.shard_owners(ns)
        assert np.array_equal(bo, bench.shard_owners(wg, ns)) and np.array_equal(no, bench.shard_owners(wh, ns))
        assert np.all(np.diff(bo) >= 0) and np.all(np.diff(no) >= 0)
        for own, w in ((bo, wg), (no, wh)):
            per = np.bincount(own, weights=w, minlength=ns)
            assert np.all(np.abs(per - w.sum() / ns) <= w.max()), per
    # the BF16 prediction splits into shards that sum to the whole (to FP32 rounding of the sum)
    F = hh_synth.forces(n, 2)
    full = c.predict(cuda(X), cuda(F), p).cpu().numpy()
    parts = [c.predict(cuda(X), cuda(F), hh.Params(precision="bf16", leaf_size=64, shard_id=s, n_shards=4))
             .cpu().numpy() for s in range(4)]
    assert oracle.rel_error(full, sum(parts)) < 1e-12


def test_batch_predict_equals_separate(ctx):
    sizes = [900, 1300, 2]
    Xs = [hh_synth.rsa_cube(s, 0.1, seed=20 + i) for i, s in enumerate(sizes)]
    Fs = [hh_synth.forces(s, 30 + i) for i, s in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    p = hh.Params(precision="fp64")
    Ub = ctx.predict(cuda(np.concatenate(Xs)), cuda(np.concatenate(Fs)), p, offsets=off).cpu().numpy()
    for i in range(len(sizes)):
        Ui = ctx.predict(cuda(Xs[i]), cuda(Fs[i]), p).cpu().numpy()
        assert np.array_equal(Ub[off[i]:off[i + 1]], Ui)


def test_deterministic(ctx):
    n = 4000
    X, F = cuda(hh_synth.rsa_cube(n, 0.1, seed=12)), cuda(hh_synth.forces(n, 6))
    p = hh.Params(precision="fp32")
    a = ctx.predict(X, F, p).cpu().numpy()
    b = ctx.predict(X, F, p).cpu().numpy()
    assert np.array_equal(a, b)


def test_larger_sampled_rows(ctx):
    n = 30000
    X = hh_synth.rsa_cube(n, 0.1, seed=13)
    F = hh_synth.forces(n, 7)
    U = ctx.predict(cuda(X), cuda(F), hh.Params(precision="fp32", eps=1e-4)).cpu().numpy()
    rows = np.arange(0, n, 97)
    Ud = oracle.dense_matvec(X, F, kern(), rows=rows, with_self=False)
    a1 = oracle.self_mobility()
    assert oracle.rel_error(Ud, U[rows] - a1 * F[rows]) <= 1e-4
    st = ctx.stats()
    assert st["n_blocks_G"] > 0 and st["n_aca_queries"] > 0 and st["n_near_pairs"] > 0


def test_bad_arguments(ctx):
    X = cuda(hh_synth.rsa_cube(100, 0.1))
    with pytest.raises(hh.HHError) as e:
        ctx.predict(X, X, hh.Params(max_rank=65))
    assert e.value.status == hh.HH_ERR_ARG
    with pytest.raises(hh.HHError):
        ctx.predict(X, X, hh.Params(leaf_size=1))
    bad = X.clone()
    bad[5, 1] = float("nan")
    with pytest.raises(hh.HHError) as e:
        ctx.predict(bad, X, hh.Params())
    assert e.value.status == hh.HH_ERR_NUMERIC


# --------------------------------------------------------------------------
# pair kernel element-wise, every precision (BF16 = tcgen05 tensor cores)
# --------------------------------------------------------------------------
# BF16 bound: features and activations are split into a bf16 part and a bf16
# remainder (~16 significant bits, relative 2^-17 = 7.6e-6 each), weights are
# exactly bf16, accumulation FP32: a few 1e-5 of the block scale per entry.
PAIR_TOL = {"fp64": 1e-12, "fp32": 2e-6, "bf16": 1e-4}


@pytest.mark.parametrize("width", [32, 64])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_eval_pairs_against_oracle(prec, width):
    c = hh.Context()
    th = THETA32 if width == 32 else THETA64
    c.set_mlp(th, width)
    rng = np.random.default_rng(17)
    n = 3001                      # ragged: 23 full 128-pair tiles + 57
    u = rng.normal(size=(n, 3)); u /= np.linalg.norm(u, axis=1)[:, None]
    r = u * np.exp(rng.uniform(np.log(2.0), np.log(800.0), size=n))[:, None]
    K = c.eval_pairs(cuda(r), hh.Params(precision=prec)).cpu().numpy()
    k = kern("mlp", width)
    Ko = np.stack([oracle.pair_block(k, ri) for ri in r])
    scale = np.abs(Ko).reshape(n, 9).max(axis=1)
    err = (np.abs(K - Ko).reshape(n, 9).max(axis=1) / scale).max()
    assert err < PAIR_TOL[prec], f"{prec} w={width}: max relative entry error {err:.3e}"


BF16_FLOOR = 1e-4   # eps_r floor of the BF16 tensor-core near field (see PAIR_TOL)


def test_predict_bf16_against_oracle(ctx):
    n = 2048
    X = hh_synth.rsa_cube(n, 0.1, seed=6)
    F = hh_synth.forces(n, 1)
    U = ctx.predict(cuda(X), cuda(F), hh.Params(precision="bf16")).cpu().numpy()
    Uo, _ = oracle.hmatvec(X, F, kern(), leaf=32, eta=1.0, eps=1e-4, max_rank=48)
    assert oracle.rel_error(Uo, U) < 1e-4
    a1 = oracle.self_mobility()
    Ud = oracle.dense_matvec(X, F, kern(), with_self=False)
    assert oracle.rel_error(Ud, U - a1 * F) < max(1e-4, BF16_FLOOR)


def test_predict_bf16_width64_and_transpose(ctx):
    c = hh.Context()
    c.set_mlp(THETA64, 64)
    n = 1500
    X = hh_synth.rsa_cube(n, 0.1, seed=8)
    F = hh_synth.forces(n, 2)
    W = hh_synth.forces(n, 9)
    p = hh.Params(precision="bf16", leaf_size=64)
    U = c.predict(cuda(X), cuda(F), p).cpu().numpy()
    Uo, _ = oracle.hmatvec(X, F, kern("mlp", 64), leaf=64, eta=1.0, eps=1e-4, max_rank=48)
    assert oracle.rel_error(Uo, U) < 1e-4
    t = c.build_tree(cuda(X), p)
    h = c.aca(t, c.partition(t, p), p)
    U1 = c.matvec(h, cuda(F)).cpu().numpy()
    UT = c.matvec(h, cuda(W), transpose=True).cpu().numpy()
    assert oracle.rel_error(U, U1) < 1e-6
    # <W, M F> = <M^T W, F> holds to the BF16 pair-kernel noise of the two near-field sweeps
    assert abs(np.sum(W * U1) - np.sum(UT * F)) <= 1e-4 * np.sqrt(np.sum(W * W) * np.sum(U1 * U1))


def test_predict_bf16_large_blocks_sampled_rows(ctx):
    # N = 30k at C_leaf = 64 has admissible blocks with more than 512 rows or
    # columns (the tensor-core ACA's CTA teams) besides the warp-team blocks
    n = 30000
    X = hh_synth.rsa_cube(n, 0.1, seed=14)
    F = hh_synth.forces(n, 8)
    p = hh.Params(precision="bf16", leaf_size=64)
    t = ctx.build_tree(cuda(X), p)
    G, _ = ctx.partition(t, p).export()
    te = t.export()
    side = te["end"] - te["begin"]
    assert max(side[G[:, 0]].max(), side[G[:, 1]].max()) > 512
    U = ctx.predict(cuda(X), cuda(F), p).cpu().numpy()
    U2 = ctx.predict(cuda(X), cuda(F), p).cpu().numpy()
    assert np.array_equal(U, U2)                         # independent of team scheduling
    rows = np.arange(0, n, 97)
    Ud = oracle.dense_matvec(X, F, kern(), rows=rows, with_self=False)
    a1 = oracle.self_mobility()
    assert oracle.rel_error(Ud, U[rows] - a1 * F[rows]) <= 2e-4
    U32 = ctx.predict(cuda(X), cuda(F), hh.Params(precision="fp32", leaf_size=64)).cpu().numpy()
    assert oracle.rel_error(U32, U) <= 2e-4


def test_predict_bf16_batch_equals_separate(ctx):
    sizes = [1700, 2500, 3]
    Xs = [hh_synth.rsa_cube(s, 0.1, seed=40 + i) for i, s in enumerate(sizes)]
    Fs = [hh_synth.forces(s, 50 + i) for i, s in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    p = hh.Params(precision="bf16")
    Ub = ctx.predict(cuda(np.concatenate(Xs)), cuda(np.concatenate(Fs)), p, offsets=off).cpu().numpy()
    for i in range(len(sizes)):
        Ui = ctx.predict(cuda(Xs[i]), cuda(Fs[i]), p).cpu().numpy()
        assert np.array_equal(Ub[off[i]:off[i + 1]], Ui)


def test_bf16_rounds_independent_of_budget_and_j1_rule_1(ctx):
    # The BF16 ACA runs as rounds over a set of active blocks whose size the
    # memory budget sets; which blocks share a round must not change a bit of
    # the result.  N = 30k has blocks from a few dozen up to thousands of rows.
    n = 30000
    X = cuda(hh_synth.rsa_cube(n, 0.1, seed=14))
    F = cuda(hh_synth.forces(n, 8))
    c = hh.Context()
    c.set_mlp(THETA32, 32)
    c.set_launch(rounds_min_cq=513)                      # every block with c or q > 512 through the rounds
    U = c.predict(X, F, hh.Params(precision="bf16", leaf_size=64)).cpu().numpy()
    rounds = c.stats()["n_aca_rounds"]
    assert rounds > 0
    Ub = c.predict(X, F, hh.Params(precision="bf16", leaf_size=64, mem_budget=16 << 20)).cpu().numpy()
    assert c.stats()["n_aca_rounds"] > rounds            # fewer slots, more rounds
    assert np.array_equal(U, Ub)
    # the same blocks on CTA teams (the default threshold) agree within the BF16 tolerance
    U0 = ctx.predict(X, F, hh.Params(precision="bf16", leaf_size=64)).cpu().numpy()
    assert oracle.rel_error(U0, U) < 1e-4
    # the randomised first column (rule 1) against the oracle's product with the same rule
    n = 4096
    Xh, Fh = hh_synth.rsa_cube(n, 0.1, seed=21), hh_synth.forces(n, 3)
    p = hh.Params(precision="bf16", j1_rule=1, seed=5)
    U1 = ctx.predict(cuda(Xh), cuda(Fh), p).cpu().numpy()
    Uo, _ = oracle.hmatvec(Xh, Fh, kern(), leaf=32, eta=1.0, eps=1e-4, max_rank=48, j1_rule=1, seed=5)
    assert oracle.rel_error(Uo, U1) < 1e-4


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_low_precision_rank_loops_stop_at_their_noise_floor(ctx, eps):
    # FP32 residuals: pivot elements whose singular values sit at the rounding
    # noise of the residual entries are not inverted (damped inverse), so a
    # block's rank loop does not fit amplified noise and run to max_rank.
    # Without it, at N = 30k RPY the FP32 error was 5x the FP64 one at
    # zeta = 1e-4 and flat near 2.6e-4 at zeta = 1e-6
    n = 30000
    X = hh_synth.rsa_cube(n, 0.1, seed=21)
    F = hh_synth.forces(n, 1)
    rows = np.sort(np.random.default_rng(2).choice(n, 256, replace=False))
    Ud = oracle.dense_matvec(X, F, kern("rpy"), rows=rows, with_self=False)
    a1 = oracle.self_mobility()
    err = {}
    for prec in ("fp64", "fp32"):
        p = hh.Params(precision=prec, eps=eps, leaf_size=64, kernel="rpy")
        U = ctx.predict(cuda(X), cuda(F), p).cpu().numpy()
        err[prec] = oracle.rel_error(Ud, U[rows] - a1 * F[rows])
        if prec == "fp32":
            t = ctx.build_tree(cuda(X), p)
            b = ctx.partition(t, p)
            h = ctx.aca(t, b, hh.Params(precision=prec, eps=eps, leaf_size=64, kernel="rpy", pivots_only=True))
            ranks, _, _ = h.export()
            assert np.mean(ranks == 48) < 0.01, np.mean(ranks == 48)
    assert err["fp32"] <= 2.0 * err["fp64"] + 2e-5, err
