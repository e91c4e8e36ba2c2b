"""Failure paths on the GPU, none of which faults, traps or hangs it: the rank
cap of Algorithm 2 (a warning with a usable product), a device allocation
made to fail at successive points of a prediction (HH_ERR_OOM, nothing
leaked, the context still usable), and tensor-core MMA waits that run out
(HH_ERR_TIMEOUT from a bounded wait on a barrier nothing arrives at, the
accumulator memory still released after the MMA's own completion)."""
import numpy as np
import pytest

import hh_synth
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402


def _pool_used():
    """Bytes in use in the device's default memory pool, which only the
    library's stream-ordered temporaries draw on in these tests."""
    from cuda.bindings import runtime as rt
    err, pool = rt.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    assert err == rt.cudaError_t.cudaSuccess
    err, v = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)
    assert err == rt.cudaError_t.cudaSuccess
    return int(v)


def _setup(n, seed):
    c = hh.Context()
    c.set_mlp(hh_synth.mlp_params(32, 7), 32)
    X = torch.as_tensor(hh_synth.rsa_cube(n, 0.1, seed=seed)).cuda()
    F = torch.as_tensor(hh_synth.forces(n, seed)).cuda()
    return c, X, F


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_rank_cap_warns_and_keeps_a_usable_product(prec):
    # max_rank = 2 with eps = 1e-12: blocks stop at the cap (the stopping test
    # of Algorithm 2 is never met), the call returns HH_WARN_RANK_CAP, and the
    # product is the rank-2 truncation: finite, within a bounded distance of
    # the converged one (the oracle's rank-2 truncation of this suspension at
    # N = 3000 is 12% away from its converged product)
    c, X, F = _setup(3000, 3)
    U = c.predict(X, F, hh.Params(precision=prec, leaf_size=64, eps=1e-12, max_rank=2)).cpu().numpy()
    assert c.last_status == hh.HH_WARN_RANK_CAP
    assert np.isfinite(U).all()
    U0 = c.predict(X, F, hh.Params(precision=prec, leaf_size=64)).cpu().numpy()
    assert c.last_status == hh.HH_OK
    e = oracle.rel_error(U0, U)
    assert 1e-3 < e < 0.5, e


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_failed_allocation_leaks_nothing(prec):
    # the k-th device allocation of a prediction fails: the call returns
    # HH_ERR_OOM, every temporary it took is freed (the pool's used bytes are
    # back to their level before the call), and the next call on the same
    # context gives the same velocities bit for bit
    c, X, F = _setup(30000, 5)
    p = hh.Params(precision=prec, leaf_size=64)
    U0 = c.predict(X, F, p).clone()
    torch.cuda.synchronize()
    base = _pool_used()
    hits, k = 0, 1
    while True:
        hh.debug_fail_alloc(k)
        try:
            c.predict(X, F, p)
            failed = False
        except hh.HHError as e:
            assert e.status == hh.HH_ERR_OOM, e
            failed = True
        hh.debug_fail_alloc(0)
        torch.cuda.synchronize()
        assert _pool_used() == base, (k, _pool_used(), base)
        if not failed:
            break
        hits += 1
        U = c.predict(X, F, p)
        assert torch.equal(U, U0), k
        k = k + 1 if k < 8 else k + k // 3    # every early allocation, then a spread over the rest
    assert hits >= 8, hits


def test_failed_allocation_in_the_stages():
    # the same at the separate stages: tree, partition, H-matrix assembly
    c, X, F = _setup(20000, 6)
    p = hh.Params(precision="fp32", leaf_size=64)
    torch.cuda.synchronize()
    base = _pool_used()
    for stage in ("tree", "partition", "aca"):
        t = c.build_tree(X, p) if stage != "tree" else None
        b = c.partition(t, p) if stage == "aca" else None
        for k in (1, 2, 3):
            hh.debug_fail_alloc(k)
            with pytest.raises(hh.HHError) as ei:
                if stage == "tree":
                    c.build_tree(X, p)
                elif stage == "partition":
                    c.partition(t, p)
                else:
                    c.aca(t, b, p)
            assert ei.value.status == hh.HH_ERR_OOM
            hh.debug_fail_alloc(0)
            torch.cuda.synchronize()
            assert _pool_used() == base, (stage, k)
        del b, t
    c.predict(X, F, p)                     # the context still works
    assert c.last_status in (hh.HH_OK, hh.HH_WARN_RANK_CAP)


def test_stalled_mma_waits_time_out_and_the_context_recovers():
    # every tensor-core MMA wait watches a barrier nothing arrives at for 64
    # polls: the BF16 prediction (warp teams, CTA teams, the round engine and
    # the near field) returns HH_ERR_TIMEOUT instead of hanging; with normal
    # waits restored the same context gives the same velocities as before
    c, X, F = _setup(30000, 8)
    p = hh.Params(precision="bf16", leaf_size=64)
    c.set_launch(rounds_min_cq=513)        # the round engine takes the largest blocks at this size
    U0 = c.predict(X, F, p).clone()
    c.debug_stall_mma_waits(64)
    with pytest.raises(hh.HHError) as ei:
        c.predict(X, F, p)
    assert ei.value.status == hh.HH_ERR_TIMEOUT
    c.debug_stall_mma_waits(0)
    U = c.predict(X, F, p)
    assert c.last_status in (hh.HH_OK, hh.HH_WARN_RANK_CAP)
    assert torch.equal(U, U0)
