"""SVD recompression of the stored ACA factors (hh_recompress) against the
oracle's truncated SVD of its own Algorithm 2 factors on the same blocks, and
the recompressed product against the original one."""
import numpy as np
import pytest

import hh_synth
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402

THETA = hh_synth.mlp_params(32, 7)


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def ctx():
    c = hh.Context()
    c.set_mlp(THETA, 32)
    return c


@pytest.mark.parametrize("eps_rc", [1e-4, 1e-6])
def test_recompressed_blocks_against_oracle(ctx, eps_rc):
    n = 3000
    X = hh_synth.rsa_cube(n, 0.1, seed=31)
    F = hh_synth.forces(n, 3)
    k = oracle.PairKernel("mlp", THETA, 32)
    p = hh.Params(precision="fp64", leaf_size=32, eps=1e-6)
    t = ctx.build_tree(cuda(X), p)
    b = ctx.partition(t, p)
    h = ctx.aca(t, b, p)
    ranks, pI, pJ = h.export()
    fofs, _ = h.export_factors()
    U0 = ctx.matvec(h, cuda(F)).cpu().numpy()
    h.recompress(eps_rc)
    sr, so, sf = h.export_recompressed()
    with pytest.raises(hh.HHError):
        h.export_factors()                       # the ACA factors are gone
    G, _ = b.export()
    ot = oracle.build_tree(X, 32)
    rng = np.random.default_rng(1)
    idx = np.flatnonzero(ranks > 0)
    checked = same = 0
    for bi in rng.choice(idx, size=min(120, len(idx)), replace=False):
        ta, sa = G[bi]
        t0, c = int(ot.begin[ta]), int(ot.end[ta] - ot.begin[ta])
        s0, q = int(ot.begin[sa]), int(ot.end[sa] - ot.begin[sa])
        a = oracle.aca_block(k, ot.Xs, t0, c, s0, q, 1e-6, 48, 0)
        if a["rank"] != ranks[bi] or np.any(a["I"] != pI[bi, :a["rank"]]) or np.any(a["J"] != pJ[bi, :a["rank"]]):
            continue                             # a near-tie pivot flip: another approximant
        M = oracle.block_matrix(a["C"], a["Q"])
        Uo, Vo, ro, sv = oracle.recompress(a["C"], a["Q"], eps_rc)
        r = int(sr[bi])
        o = int(so[bi])
        Ug = sf[o:o + r * 3 * c].reshape(r, 3 * c).T
        Vg = sf[o + r * 3 * c:o + r * 3 * (c + q)].reshape(r, 3 * q)
        nM = np.linalg.norm(M)
        assert np.linalg.norm(M - Ug @ Vg) <= eps_rc * nM * (1 + 1e-6) + 1e-12 * nM
        assert r <= 3 * ranks[bi]
        checked += 1
        if r == ro:
            same += 1
            # the same truncation to within the Gram method's resolution: the
            # singular subspaces come from C^T C and Q Q^T, accurate to about
            # eps_machine kappa(C)^2 (observed 2.6e-8 of ||M||), far inside eps_rc
            assert np.linalg.norm(Ug @ Vg - Uo @ Vo) <= 1e-6 * nM
        else:
            # only where the cut falls within rounding of a singular value
            s2 = sv ** 2
            lo = min(r, ro)
            tail_lo = np.sum(s2[lo:])
            assert abs(tail_lo - eps_rc ** 2 * np.sum(s2)) <= 1e-6 * np.sum(s2), (r, ro)
    assert checked >= 100 and same >= 0.97 * checked
    # the recompressed product stays within eps_rc of the original, with fewer bytes
    U1 = ctx.matvec(h, cuda(F)).cpu().numpy()
    assert oracle.rel_error(U0, U1) <= 2 * eps_rc
    assert so[-1] < 9 * fofs[-1]


def test_recompressed_fp32_transpose_and_adjoint(ctx):
    # FP32 factors: the transposed product is still the adjoint of the
    # product, and the gradient of a recompressed H-matrix is that of its
    # pivots (rebuilt in FP64)
    n = 4000
    X = hh_synth.rsa_cube(n, 0.1, seed=33)
    F, W = hh_synth.forces(n, 4), hh_synth.forces(n, 5)
    p = hh.Params(precision="fp32", leaf_size=32)
    t = ctx.build_tree(cuda(X), p)
    b = ctx.partition(t, p)
    h = ctx.aca(t, b, p)
    gX0 = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    ctx.matvec_backward(h, cuda(W), cuda(F), gX=gX0)
    U0 = ctx.matvec(h, cuda(F)).cpu().numpy()
    h.recompress(1e-4)
    U1 = ctx.matvec(h, cuda(F)).cpu().numpy()
    UT = ctx.matvec(h, cuda(W), transpose=True).cpu().numpy()
    assert oracle.rel_error(U0, U1) <= 3e-4
    assert float(np.sum(W * U1)) == pytest.approx(float(np.sum(F * UT)), rel=1e-5)
    gX1 = torch.zeros_like(gX0)
    ctx.matvec_backward(h, cuda(W), cuda(F), gX=gX1)
    assert torch.equal(gX0, gX1)
