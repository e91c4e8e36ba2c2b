"""The size-independent tree and partition checks (tests/hmat_invariants.py)
pinned on the oracle: they accept the oracle's structures and reject
corrupted copies (a dropped block, a block moved between the lists, a
duplicated block, a shrunken box, two particles swapped)."""
import numpy as np
import pytest

import hh_synth
import oracle
from hmat_invariants import check_partition, check_tree


@pytest.mark.parametrize("n,leaf,eta", [(5000, 32, 1.0), (3000, 64, 0.7), (2000, 16, 1.5), (1, 32, 1.0),
                                        (33, 32, 1.0)])
def test_oracle_structures_pass(n, leaf, eta):
    X = hh_synth.rsa_cube(n, 0.1, seed=n) if n > 1 else np.array([[1.0, 2.0, 3.0]])
    t = oracle.build_tree(X, leaf)
    G, H = oracle.partition(t, leaf, eta)
    check_partition(X, t, G, H, leaf, eta, samples=50000)


def test_degenerate_inputs_pass():
    X = np.zeros((40, 3)); X[20:, 0] = 1.0                      # two sites: equal codes
    t = oracle.build_tree(X, 8)
    G, H = oracle.partition(t, 8, 1.0)
    check_partition(X, t, G, H, 8, 1.0, samples=20000)


def _case():
    X = hh_synth.rsa_cube(3000, 0.1, seed=5)
    t = oracle.build_tree(X, 32)
    G, H = oracle.partition(t, 32, 1.0)
    tree = {k: np.array(getattr(t, k)) for k in ("perm", "begin", "end", "child", "lo", "hi")}
    return X, tree, G, H


def test_corruptions_are_caught():
    X, tree, G, H = _case()
    check_partition(X, tree, G, H, 32, 1.0)
    with pytest.raises(AssertionError):                          # a dropped admissible block
        check_partition(X, tree, G[1:], H, 32, 1.0)
    with pytest.raises(AssertionError):                          # an admissible block listed as near
        check_partition(X, tree, G[1:], np.concatenate([H, G[:1]]), 32, 1.0)
    big = np.argmax([(tree["end"][a] - tree["begin"][a]) * (tree["end"][b] - tree["begin"][b]) for a, b in G])
    same = [k for k, (a, b) in enumerate(G) if k != big and
            (tree["end"][a] - tree["begin"][a]) * (tree["end"][b] - tree["begin"][b]) ==
            (tree["end"][G[big][0]] - tree["begin"][G[big][0]]) * (tree["end"][G[big][1]] - tree["begin"][G[big][1]])]
    if same:                                                     # area kept, one region twice, one missing
        G2 = G.copy()
        G2[same[0]] = G[big]
        with pytest.raises(AssertionError):
            check_partition(X, tree, G2, H, 32, 1.0)
    t2 = {k: v.copy() for k, v in tree.items()}
    t2["lo"][5, 1] += 1e-9                                       # a box that no longer fits its points
    with pytest.raises(AssertionError):
        check_tree(X, t2, 32)
    t3 = {k: v.copy() for k, v in tree.items()}
    t3["perm"][[0, -1]] = t3["perm"][[-1, 0]]                    # two particles in the wrong leaves
    with pytest.raises(AssertionError):
        check_tree(X, t3, 32)
    with pytest.raises(AssertionError):                          # a leaf size the rule forbids
        check_tree(X, tree, 8)
