"""GPU test of hh_aca_block_apply_noalloc, the entry point for callers that
may not allocate device memory at the time they call (for example an
application whose device memory all belongs to its own pool, or a real-time
step that must not risk the synchronisation or failure of a cudaMalloc).

It must return what the existing entry point hh_predict computes for the same
block, and what the FP64 oracle's block ACA gives.  Geometry: two clusters A
(targets) and B (sources) far apart along x, with C_leaf just above both
sizes, so the tree is root -> {A, B} and the only admissible blocks are (A, B)
and (B, A).  With zero force on A, hh_predict's velocity of A is exactly the
low-rank product of block (A, B) with F_B, taken in the tree's (Morton) order
-- which is the order the test passes to the allocation-free call.  Two calls
in a row with different forces check that nothing from the previous call
leaks through the shared device array, and the second call is watched for
device allocations.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import hh_synth
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402

THETA = hh_synth.mlp_params(32, 7)


def _noalloc(ctx, Xt, Xs, F, params, y=None, rank=None):
    c, q = Xt.shape[0], Xs.shape[0]
    y = torch.zeros((c, 3), dtype=torch.float64, device="cuda") if y is None else y
    rank = torch.zeros(1, dtype=torch.int32, device="cuda") if rank is None else rank
    st = hh.lib().hh_aca_block_apply_noalloc(ctx._h, hh._dptr(Xt), c, hh._dptr(Xs), q, hh._dptr(F),
                                             ctypes.byref(params), hh._stream(), hh._dptr(y), hh._dptr(rank))
    return st, y, rank


def _pool_used():
    """(used bytes now, high-water mark) of the device's default memory pool,
    which the library's stream-ordered temporaries come from."""
    from cuda.bindings import runtime as cudart
    err, pool = cudart.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    assert err == cudart.cudaError_t.cudaSuccess
    out = []
    for a in (cudart.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent, cudart.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh):
        err, v = cudart.cudaMemPoolGetAttribute(pool, a)
        assert err == cudart.cudaError_t.cudaSuccess
        out.append(int(v))
    return tuple(out)


def _two_clusters(c, q):
    rng = np.random.default_rng(5)
    A = rng.uniform(0.0, 14.0, size=(c, 3))
    B = rng.uniform(0.0, 14.0, size=(q, 3)) + np.array([400.0, 3.0, -2.0])
    return np.concatenate([A, B])


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("fp64", 1e-6)])
def test_noalloc_block_matches_predict_and_oracle(prec, tol):
    c, q = 100, 77
    X = _two_clusters(c, q)
    ctx = hh.Context()
    ctx.set_mlp(THETA, 32)
    p = hh.Params(precision=prec, leaf_size=max(c, q) + 1, eps=1e-4, max_rank=48)
    Xd = torch.as_tensor(X).cuda()

    tree = ctx.build_tree(Xd, p)
    G, H = ctx.partition(tree, p).export()
    t = tree.export()
    assert [tuple(g) for g in G] == [(1, 2), (2, 1)] and [tuple(h) for h in H] == [(1, 1), (2, 2)]
    perm = t["perm"]
    assert np.all(perm[:c] < c) and np.all(perm[c:] >= c)
    Xsorted = X[perm]
    Xt = torch.as_tensor(Xsorted[:c]).cuda()
    Xs = torch.as_tensor(Xsorted[c:]).cuda()
    # the oracle's Algorithm 2 on the same block (targets first, then sources)
    ref = oracle.aca_block(oracle.PairKernel("mlp", THETA, 32), Xsorted, 0, c, c, q, 1e-4, 48, 0)

    for call, seed in enumerate((3, 4)):   # two calls in a row
        F = hh_synth.forces(c + q, seed)
        F[:c] = 0.0
        U = ctx.predict(Xd, torch.as_tensor(F).cuda(), p).cpu().numpy()
        want = U[perm[:c]]
        Fs = torch.as_tensor(F[perm[c:]]).cuda()
        y = torch.zeros((c, 3), dtype=torch.float64, device="cuda")
        rank = torch.zeros(1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        used0 = _pool_used()
        st, y, rank = _noalloc(ctx, Xt, Xs, Fs, p, y, rank)
        torch.cuda.synchronize()
        if call == 1:   # the second call allocates nothing (device free memory, default pool)
            assert torch.cuda.mem_get_info()[0] == free0
            assert _pool_used() == used0
        assert st == hh.HH_OK, hh.lib().hh_last_error(ctx._h)
        got = y.cpu().numpy()
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err < tol, f"{prec}: relative difference {err:.3e} vs hh_predict"
        yo = np.einsum("pmab,pb->ma", ref["C"], np.einsum("pnbc,nc->pb", ref["Q"], F[perm[c:]]))
        err_o = np.linalg.norm(got - yo) / np.linalg.norm(yo)
        assert err_o < tol, f"{prec}: relative difference {err_o:.3e} vs the oracle"
        assert 1 <= int(rank.item()) <= 48
        if prec == "fp64":
            assert int(rank.item()) == ref["rank"]


def test_noalloc_rejects_oversize_block_and_bf16():
    ctx = hh.Context()
    ctx.set_mlp(THETA, 32)
    X = torch.zeros((129, 3), dtype=torch.float64, device="cuda")
    st, _, _ = _noalloc(ctx, X, X[:10], X[:10], hh.Params())
    assert st == hh.HH_ERR_ARG
    assert b"at most 128" in hh.lib().hh_last_error(ctx._h)
    # the tensor-core precision is not offered here (it would silently run FP32)
    X = torch.as_tensor(_two_clusters(20, 20)).cuda()
    st, _, _ = _noalloc(ctx, X[:20], X[20:], X[20:], hh.Params(precision="bf16"))
    assert st == hh.HH_ERR_ARG
    assert b"HH_FP32 or HH_FP64" in hh.lib().hh_last_error(ctx._h)
