"""Tree and partition at the benchmark's full size (N = 1M uniform cube,
C_leaf 64, eta 1) and on a 100k-bead filament suspension: bit-exact against
the oracle (which builds both in seconds) and checked against the
size-independent invariants of tests/hmat_invariants.py."""
import numpy as np
import pytest

import hh_synth
import oracle
from hmat_invariants import check_partition

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = hh.Context()
    c.set_mlp(hh_synth.mlp_params(32, 7), 32)
    return c


def _compare(ctx, X, leaf, eta):
    p = hh.Params(leaf_size=leaf, eta=eta)
    t = ctx.build_tree(torch.as_tensor(X).cuda(), p)
    g = t.export()
    G, H = ctx.partition(t, p).export()
    o = oracle.build_tree(X, leaf)
    oG, oH = oracle.partition(o, leaf, eta)
    assert np.array_equal(g["perm"], o.perm) and np.array_equal(g["codes"], o.codes)
    assert np.array_equal(g["begin"], o.begin) and np.array_equal(g["end"], o.end)
    assert np.array_equal(g["child"], o.child)
    assert np.array_equal(g["lo"], o.lo) and np.array_equal(g["hi"], o.hi)
    assert np.array_equal(G, oG) and np.array_equal(H, oH)
    check_partition(X, g, G, H, leaf, eta)


def test_full_size_cube(ctx):
    _compare(ctx, hh_synth.rsa_cube(1_000_000, 0.1, seed=1234), 64, 1.0)


def test_filament_suspension(ctx):
    X, _, _ = hh_synth.filaments(2000, 50, seed=1234)
    _compare(ctx, X, 64, 1.0)
