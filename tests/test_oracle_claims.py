"""Properties the paper states for the method (Sections 3.3, 4.1 and 4.2),
checked on the oracle's H-matrix product:

* the ACA ranks of admissible blocks stay nearly constant as N grows, set by
  the tolerance zeta rather than by the configuration;
* the relative error eps_r (Eq. 11) is controlled by zeta and moves by less
  than a decade when the leaf size C_leaf changes.
"""
import numpy as np

import hh_synth
import oracle

K = oracle.PairKernel("mlp", hh_synth.mlp_params(32, 7), 32)


def test_ranks_nearly_constant_in_n():
    means, spreads = [], []
    for n in (1000, 2000, 4000):
        X = hh_synth.rsa_cube(n, 0.1, seed=3)
        _, st = oracle.hmatvec(X, hh_synth.forces(n, 0), K, leaf=32, eps=1e-4, want_ranks=True)
        r = st["ranks"]
        assert len(r) > 0
        means.append(r.mean())
        spreads.append(np.percentile(r, 90) - np.percentile(r, 10))
    assert max(means) / min(means) < 1.15
    assert max(spreads) <= 6
    # and the rank follows zeta: a looser tolerance gives lower ranks
    X = hh_synth.rsa_cube(2000, 0.1, seed=3)
    _, lo = oracle.hmatvec(X, hh_synth.forces(2000, 0), K, leaf=32, eps=1e-2, want_ranks=True)
    assert lo["ranks"].mean() < 0.7 * means[1]


def test_error_insensitive_to_leaf_size():
    n = 2048
    X = hh_synth.rsa_cube(n, 0.1, seed=4)
    F = hh_synth.forces(n, 1)
    Ud = oracle.dense_matvec(X, F, K)
    errs = []
    for leaf in (16, 32, 64):
        U, _ = oracle.hmatvec(X, F, K, leaf=leaf, eps=1e-4)
        errs.append(oracle.rel_error(Ud, U))
    assert max(errs) <= 1e-4
    assert max(errs) / min(errs) < 10.0
