"""Properties of the cluster tree (Definition 1) and the block partition
(Eq. 7, Algorithm 1) that hold at any size, checked with plain numpy on the
exported structures.  Used where the oracle cannot rebuild the structures
element by element (N = 1M), and pinned on the CPU against the oracle's own
tree and partition (and corrupted copies of them).

tree: mapping or object with perm [N], begin/end [nn], child [nn, 2] (-1 for
a leaf), lo/hi [nn, 3]; G, H: [nb, 2] (target node, source node)."""
import numpy as np


def _get(tree, k):
    return np.asarray(tree[k] if isinstance(tree, dict) else getattr(tree, k))


def check_tree(X, tree, leaf):
    perm, begin, end = _get(tree, "perm"), _get(tree, "begin"), _get(tree, "end")
    child, lo, hi = _get(tree, "child"), _get(tree, "lo"), _get(tree, "hi")
    n, nn = len(X), len(begin)
    # the permutation is a bijection of [0, n)
    assert len(perm) == n and np.array_equal(np.sort(perm), np.arange(n))
    assert begin[0] == 0 and end[0] == n
    is_leaf = child[:, 0] < 0
    assert np.array_equal(is_leaf, child[:, 1] < 0)
    # children tile their parent's range and come after it (breadth-first)
    inner = np.nonzero(~is_leaf)[0]
    c0, c1 = child[inner, 0], child[inner, 1]
    assert np.all(c0 > inner) and np.all(c1 > inner)
    assert np.array_equal(begin[c0], begin[inner]) and np.array_equal(end[c0], begin[c1])
    assert np.array_equal(end[c1], end[inner])
    assert np.all(begin[c0] < end[c0]) and np.all(begin[c1] < end[c1])
    # every node but the root has exactly one parent
    par = np.full(nn, -1)
    par[c0] = inner
    par[c1] = inner
    assert par[0] == -1 and np.all(par[1:] >= 0)
    assert len(np.unique(np.concatenate([c0, c1]))) == 2 * len(inner)
    # leaf iff |tau| < C_leaf
    size = end - begin
    assert np.all(size[is_leaf] < leaf) and np.all(size[inner] >= leaf)
    # boxes are the exact extents of the node's (sorted) positions
    Xs = np.asarray(X)[perm]
    lv = np.nonzero(is_leaf)[0]
    lv = lv[np.argsort(begin[lv])]
    assert np.array_equal(begin[lv], np.r_[0, end[lv][:-1]]) and end[lv][-1] == n   # leaves tile [0, n)
    blo = np.empty_like(lo)
    bhi = np.empty_like(hi)
    blo[lv] = np.minimum.reduceat(Xs, begin[lv], axis=0)
    bhi[lv] = np.maximum.reduceat(Xs, begin[lv], axis=0)
    for t in inner[::-1]:
        blo[t] = np.minimum(blo[child[t, 0]], blo[child[t, 1]])
        bhi[t] = np.maximum(bhi[child[t, 0]], bhi[child[t, 1]])
    assert np.array_equal(blo, lo) and np.array_equal(bhi, hi)
    return par, is_leaf


def _admissible(lo, hi, t, s, eta):
    """Eq. 7 on boxes of centres: dist^2 > 0 and max(diam^2) <= eta^2 dist^2,
    returned as (lhs, rhs, dist2) so callers can allow rounding slack."""
    dt = np.sum((hi[t] - lo[t]) ** 2, axis=1)
    ds = np.sum((hi[s] - lo[s]) ** 2, axis=1)
    gap = np.maximum(0.0, np.maximum(lo[s] - hi[t], lo[t] - hi[s]))
    d2 = np.sum(gap ** 2, axis=1)
    return np.maximum(dt, ds), (eta * eta) * d2, d2


def check_partition(X, tree, G, H, leaf, eta, samples=200000, seed=0):
    par, is_leaf = check_tree(X, tree, leaf)
    begin, end = _get(tree, "begin"), _get(tree, "end")
    lo, hi = _get(tree, "lo"), _get(tree, "hi")
    n = len(X)
    G = np.asarray(G, dtype=np.int64).reshape(-1, 2)
    H = np.asarray(H, dtype=np.int64).reshape(-1, 2)
    # admissible blocks satisfy Eq. 7; near blocks fail it and have a leaf side
    slack = 1e-12
    lhs, rhs, d2 = _admissible(lo, hi, G[:, 0], G[:, 1], eta)
    assert np.all(d2 > 0) and np.all(lhs <= rhs * (1 + slack))
    lhs, rhs, d2 = _admissible(lo, hi, H[:, 0], H[:, 1], eta)
    assert np.all((d2 <= 0) | (lhs >= rhs * (1 - slack)))
    assert np.all(is_leaf[H[:, 0]] | is_leaf[H[:, 1]])
    # exact cover of [0, n)^2: the areas add up to n^2 ...
    B = np.concatenate([G, H])
    area = (end[B[:, 0]] - begin[B[:, 0]]).astype(np.int64) * (end[B[:, 1]] - begin[B[:, 1]])
    assert int(area.sum()) == n * n
    # ... the source ranges of one target node never overlap ...
    o = np.lexsort((begin[B[:, 1]], B[:, 0]))
    B = B[o]
    same = B[1:, 0] == B[:-1, 0]
    assert np.all(end[B[:-1, 1]][same] <= begin[B[1:, 1]][same])
    # ... and sampled (i, j) lie in exactly one block
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, samples)
    j = rng.integers(0, n, samples)
    lv = np.nonzero(is_leaf)[0]
    lv = lv[np.argsort(begin[lv])]
    node = lv[np.searchsorted(begin[lv], i, side="right") - 1]
    key = B[:, 0] * (n + 1) + begin[B[:, 1]]          # blocks sorted by (target node, source begin)
    se = end[B[:, 1]]
    hits = np.zeros(samples, dtype=np.int64)
    while True:
        live = np.nonzero(node >= 0)[0]
        if len(live) == 0:
            break
        a = node[live]
        k = np.searchsorted(key, a * (n + 1) + j[live], side="right") - 1
        kk = np.maximum(k, 0)
        hit = (k >= 0) & (B[kk, 0] == a) & (j[live] < se[kk])
        hits[live[hit]] += 1
        node[live] = par[a]
    assert np.all(hits == 1)
