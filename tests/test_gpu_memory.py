"""The library's own device-memory high-water mark (hh_stats_t.mem_peak_bytes):
positive after a prediction, below the device's memory, and growing with N."""
import pytest

import hh_synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402


def test_peak_memory_is_reported():
    import gc
    gc.collect()                      # structures of earlier tests are freed before the marks are taken
    torch.cuda.synchronize()
    c = hh.Context()
    c.set_mlp(hh_synth.mlp_params(32, 7), 32)
    total = torch.cuda.get_device_properties(0).total_memory
    peaks = []
    for n in (2000, 40000):
        X = torch.as_tensor(hh_synth.rsa_cube(n, 0.1, seed=n)).cuda()
        c.predict(X, X.clone(), hh.Params(precision="bf16", leaf_size=64))
        m = c.stats()["mem_peak_bytes"]
        assert 0 < m < total
        peaks.append(m)
    assert peaks[1] > peaks[0]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_memory_budget_bounds_the_peak_and_changes_no_bit(prec):
    # hh_params.mem_budget: the admissible blocks run in groups whose partial
    # outputs fit half of it, the team workspaces and the round engine take
    # the other shares.  A small budget bounds the library's peak (beyond
    # the O(N) arrays: positions, forces, tree, partition, sums) and gives
    # the same velocities bit for bit.
    import gc

    import numpy as np
    gc.collect()
    torch.cuda.synchronize()
    c = hh.Context()
    c.set_mlp(hh_synth.mlp_params(32, 7), 32)
    n = 100000
    X = torch.as_tensor(hh_synth.rsa_cube(n, 0.1, seed=23)).cuda()
    F = torch.as_tensor(hh_synth.forces(n, 4)).cuda()
    U = c.predict(X, F, hh.Params(precision=prec, leaf_size=64)).cpu().numpy()
    assert c.stats()["n_aca_groups"] == 1
    budget = 96 << 20
    Ub = c.predict(X, F, hh.Params(precision=prec, leaf_size=64, mem_budget=budget)).cpu().numpy()
    st = c.stats()
    assert st["n_aca_groups"] > 1
    assert np.array_equal(U, Ub)
    o_n = 64 * 200 * n            # the O(N) arrays: well under 200 doubles' worth per particle
    assert st["mem_peak_bytes"] <= budget + o_n, (st["mem_peak_bytes"], budget + o_n)
