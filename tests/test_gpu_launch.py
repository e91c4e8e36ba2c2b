"""Launch shapes (hh_set_launch / hh_get_launch) and the autotuner
(hh_autotune): the shape changes which team runs a block and how many CTAs
share an SM, never what a block computes."""
import numpy as np
import pytest

import hh_synth
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402

THETA = hh_synth.mlp_params(32, 7)


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(torch.float64).cuda()


@pytest.fixture()
def ctx():
    c = hh.Context()
    c.set_mlp(THETA, 32)
    return c


def test_set_get_and_validation(ctx):
    assert ctx.get_launch() == dict(small_max=0, aca_small_cps=0, aca_large_cps=0, near_cps=0, rounds_min_cq=0)
    ctx.set_launch(small_max=128, aca_small_cps=2, aca_large_cps=1, near_cps=8, rounds_min_cq=2048)
    assert ctx.get_launch() == dict(small_max=128, aca_small_cps=2, aca_large_cps=1, near_cps=8, rounds_min_cq=2048)
    for bad in (dict(small_max=16), dict(small_max=1024), dict(aca_small_cps=9), dict(near_cps=-1),
                dict(rounds_min_cq=100)):
        with pytest.raises(hh.HHError):
            ctx.set_launch(**bad)
    assert ctx.get_launch()["small_max"] == 128     # unchanged by the rejected calls


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_ctas_per_sm_do_not_change_results(ctx, prec):
    n = 20000
    X, F = cuda(hh_synth.rsa_cube(n, 0.1, seed=3)), cuda(hh_synth.forces(n, 4))
    p = hh.Params(precision=prec, leaf_size=64)
    ref = ctx.predict(X, F, p).cpu().numpy()
    for cfg in (dict(aca_small_cps=1, aca_large_cps=1, near_cps=2), dict(aca_small_cps=3, aca_large_cps=4, near_cps=8)):
        ctx.set_launch(**cfg)
        assert np.array_equal(ctx.predict(X, F, p).cpu().numpy(), ref), cfg


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_team_threshold_changes_only_rounding(ctx, prec):
    # a block moved between warp and CTA teams sums its Gram matrices in
    # another order; ranks may move by one near the threshold, so the
    # products agree to well inside the ACA tolerance
    n = 20000
    X, F = cuda(hh_synth.rsa_cube(n, 0.1, seed=5)), cuda(hh_synth.forces(n, 6))
    p = hh.Params(precision=prec, leaf_size=64)
    ref = ctx.predict(X, F, p).cpu().numpy()
    for sm in (64, 256):
        ctx.set_launch(small_max=sm)
        U = ctx.predict(X, F, p).cpu().numpy()
        assert oracle.rel_error(ref, U) < 2e-5, sm


def test_autotune_picks_a_candidate_and_keeps_it(ctx):
    n = 30000
    X = cuda(hh_synth.rsa_cube(n, 0.1, seed=7))
    p = hh.Params(precision="bf16", leaf_size=64)
    best = ctx.autotune(X, p, reps=1)
    assert best == ctx.get_launch()
    assert best["small_max"] in (0, 128, 256, 512)
    assert best["aca_small_cps"] in (0, 1, 2, 3, 4)
    assert best["aca_large_cps"] in (0, 1, 2, 4)
    assert best["near_cps"] in (0, 2, 4, 8)
    F = cuda(hh_synth.forces(n, 8))
    U = ctx.predict(X, F, p).cpu().numpy()
    c2 = hh.Context()
    c2.set_mlp(THETA, 32)
    assert oracle.rel_error(c2.predict(X, F, p).cpu().numpy(), U) < 2e-5


def test_unit_probes_are_physical(ctx):
    # hh_probe_throughput: each unit's rate is positive and below what 148 SMs
    # could issue at 2.1 GHz (128 FP32 lanes per SM per clock; MUFU and FP64
    # far fewer), and the SiLU (two MUFU operations) is slower than one MUFU op
    r = {k: ctx.probe(k, 1 << 12) for k in ctx.PROBES}
    lanes_ops = 148 * 128 * 2.1e9
    for k, v in r.items():
        assert 0 < v < lanes_ops, (k, v)
    assert r["silu"] < r["mufu_ex2"]
    assert r["dfma"] < r["ffma"]
    with pytest.raises(hh.HHError):
        ctx.probe("ffma", 0)
