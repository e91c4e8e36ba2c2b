"""Adjoint of the H-matrix product (hh_matvec_backward) against finite
differences and the FP64 oracle's dense gradient.

L = sum_i w_i . U_i, U = alpha_1 F + M_H F.  The gradient is taken with tree,
partition and pivots frozen; a finite difference is only meaningful when the
perturbation leaves them unchanged, so every central difference checks that
the Morton order, the block lists and all ACA pivots are identical at x +- h
(h = 1e-5 for positions: smaller steps let the rounding noise of the rank
loop, about 1e-13 relative in L, dominate the difference quotient).
"""
import numpy as np
import pytest

import hh_synth
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402

THETA = hh_synth.mlp_params(32, 7)


def cuda(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()


@pytest.fixture(scope="module")
def ctx():
    c = hh.Context()
    c.set_mlp(THETA, 32)
    return c


def build(ctx, X, p):
    t = ctx.build_tree(cuda(X), p)
    b = ctx.partition(t, p)
    h = ctx.aca(t, b, p)
    return t, b, h


def structure(t, b, h):
    te = t.export()
    G, H = b.export()
    ranks, pI, pJ = h.export()
    return b"".join(a.tobytes() for a in (te["perm"], te["begin"], te["end"], te["child"], G, H, ranks, pI, pJ))


def loss(ctx, X, F, W, p):
    t, b, h = build(ctx, X, p)
    U = ctx.matvec(h, cuda(F)).cpu().numpy()
    return float(np.sum(W * U)), structure(t, b, h)


def grads(ctx, X, F, W, p):
    t, b, h = build(ctx, X, p)
    gF = torch.zeros((len(X), 3), dtype=torch.float64, device="cuda")
    gX = torch.zeros_like(gF)
    gT = torch.zeros(len(THETA), dtype=torch.float32, device="cuda")
    ctx.matvec_backward(h, cuda(W), cuda(F), gF=gF, gX=gX, gtheta=gT)
    return gF.cpu().numpy(), gX.cpu().numpy(), gT.cpu().numpy().astype(np.float64), (t, b, h)


def test_gF_is_transposed_product(ctx):
    n = 2000
    X = hh_synth.rsa_cube(n, 0.1, seed=41)
    F, W = hh_synth.forces(n, 1), hh_synth.forces(n, 2)
    p = hh.Params(precision="fp64")
    gF, _, _, (t, b, h) = grads(ctx, X, F, W, p)
    UT = ctx.matvec(h, cuda(W), transpose=True).cpu().numpy()
    assert np.array_equal(gF, UT)


def test_gX_central_differences(ctx):
    n = 2000
    X = hh_synth.rsa_cube(n, 0.1, seed=42)
    F, W = hh_synth.forces(n, 3), hh_synth.forces(n, 4)
    p = hh.Params(precision="fp64")
    _, gX, _, _ = grads(ctx, X, F, W, p)
    _, ref = loss(ctx, X, F, W, p)
    h = 1e-5
    checked = 0
    for (i, a) in [(0, 0), (17, 1), (345, 2), (999, 0), (1500, 1), (1999, 2), (700, 1), (1234, 0)]:
        Xp = X.copy(); Xp[i, a] += h
        Xm = X.copy(); Xm[i, a] -= h
        Lp, sp = loss(ctx, Xp, F, W, p)
        Lm, sm = loss(ctx, Xm, F, W, p)
        if sp != ref or sm != ref:
            continue          # the perturbation crossed a cell boundary or flipped a pivot
        fd = (Lp - Lm) / (2 * h)
        assert gX[i, a] == pytest.approx(fd, rel=1e-5, abs=1e-8 * np.abs(gX).max())
        checked += 1
    assert checked >= 5


def test_gtheta_central_differences(ctx):
    # small problem with small leaves: few admissible blocks, so a parameter
    # step rarely flips an ACA pivot, and still several ranks > 1
    n = 400
    X = hh_synth.rsa_cube(n, 0.1, seed=43)
    F, W = hh_synth.forces(n, 5), hh_synth.forces(n, 6)
    p = hh.Params(precision="fp64", leaf_size=16)
    _, _, gT, (t, b, h0) = grads(ctx, X, F, W, p)
    ref = structure(t, b, h0)
    h = 1e-4
    checked = 0
    for k in (3, 140, 600, 1300, 2300, 2469):
        out = []
        for sgn in (1, -1):
            th = THETA.astype(np.float64).copy()
            th[k] += sgn * h
            c = hh.Context()
            c.set_mlp(th.astype(np.float32), 32)   # exactly representable steps: see below
            out.append(loss(c, X, F, W, p))
        if out[0][1] != ref or out[1][1] != ref:
            continue
        # the perturbed parameter is rounded to float32 by the C-ABI; use the actual step
        th_p = np.float32(THETA[k] + h); th_m = np.float32(THETA[k] - h)
        fd = (out[0][0] - out[1][0]) / (float(th_p) - float(th_m))
        assert gT[k] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.abs(gT).max())
        checked += 1
    assert checked >= 4


def test_gradient_close_to_dense_oracle(ctx):
    # the gradient of the approximant converges to the dense gradient with
    # the ACA tolerance (about 10 zeta measured in FP64).  For an FP32 or
    # BF16 H-matrix, dL/dX and dL/dtheta are those of its FP64 counterpart
    # (re-approximated inside the call); dL/dF is its own transpose product
    n = 2000
    X = hh_synth.rsa_cube(n, 0.1, seed=44)
    F, W = hh_synth.forces(n, 7), hh_synth.forces(n, 8)
    k = oracle.PairKernel("mlp", THETA, 32)
    gFo, gXo, gTo = oracle.dense_grad(X, F, W, k)
    for prec, eps, tol in (("fp64", 1e-6, 1e-4), ("fp64", 1e-4, 3e-3), ("fp32", 1e-4, 3e-3), ("bf16", 1e-4, 3e-3)):
        gF, gX, gT, _ = grads(ctx, X, F, W, hh.Params(precision=prec, eps=eps))
        tf = 1e-3 if prec == "bf16" else tol    # BF16 near field: 1e-4-level entries
        assert np.linalg.norm(gF - gFo) <= tf * np.linalg.norm(gFo), prec
        assert np.linalg.norm(gX - gXo) <= tol * np.linalg.norm(gXo), prec
        assert np.linalg.norm(gT - gTo) <= tol * np.linalg.norm(gTo), prec


def test_near_only_is_exact_dense_gradient(ctx):
    # with eta -> 0 nothing is admissible: the adjoint is the dense gradient
    n = 700
    X = hh_synth.rsa_cube(n, 0.1, seed=45)
    F, W = hh_synth.forces(n, 9), hh_synth.forces(n, 10)
    gFo, gXo, gTo = oracle.dense_grad(X, F, W, oracle.PairKernel("mlp", THETA, 32))
    # FP64 H-matrix: FP64 entries (float32 theta output); FP32: the near
    # field's entries run in FP32, as its product did
    for prec, tx, tt in (("fp64", 1e-12, 1e-6), ("fp32", 2e-5, 2e-5)):
        gF, gX, gT, (t, b, h) = grads(ctx, X, F, W, hh.Params(precision=prec, eta=1e-9))
        assert len(b.export()[0]) == 0
        assert np.abs(gX - gXo).max() <= tx * np.abs(gXo).max(), prec
        assert np.abs(gT - gTo).max() <= tt * np.abs(gTo).max(), prec


def test_width64_gradient():
    th = hh_synth.mlp_params(64, 9)
    c = hh.Context()
    c.set_mlp(th, 64)
    n = 1200
    X = hh_synth.rsa_cube(n, 0.1, seed=46)
    F, W = hh_synth.forces(n, 11), hh_synth.forces(n, 12)
    gFo, gXo, gTo = oracle.dense_grad(X, F, W, oracle.PairKernel("mlp", th, 64))
    p = hh.Params(precision="fp64", eps=1e-6)
    t, b, h = build(c, X, p)
    gX = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    gT = torch.zeros(len(th), dtype=torch.float32, device="cuda")
    c.matvec_backward(h, cuda(W), cuda(F), gX=gX, gtheta=gT)
    gX, gT = gX.cpu().numpy(), gT.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gX - gXo) <= 1e-4 * np.linalg.norm(gXo)
    assert np.linalg.norm(gT - gTo) <= 1e-4 * np.linalg.norm(gTo)


def test_autograd_function_matches_direct_calls(ctx):
    n = 1500
    X0 = hh_synth.rsa_cube(n, 0.1, seed=47)
    F0, W = hh_synth.forces(n, 13), hh_synth.forces(n, 14)
    p = hh.Params(precision="fp64")
    X = cuda(X0).requires_grad_(True)
    F = cuda(F0).requires_grad_(True)
    th = torch.as_tensor(THETA, dtype=torch.float32).cuda().requires_grad_(True)
    c = hh.Context()
    U = hh.hmatvec(X, F, th, c, p)
    L = (U * cuda(W)).sum()
    L.backward()
    gF, gX, gT, _ = grads(ctx, X0, F0, W, p)
    # every sum of the adjoint has a fixed order: the same bits either way
    assert np.array_equal(F.grad.cpu().numpy(), gF)
    assert np.array_equal(X.grad.cpu().numpy(), gX)
    assert np.array_equal(th.grad.cpu().numpy().astype(np.float64), gT)
    Ud, _ = loss(ctx, X0, F0, W, p)
    assert float(L.detach()) == pytest.approx(Ud, rel=1e-14)


def test_pivots_only_hmatrix_gives_the_same_gradients(ctx):
    n = 1500
    X = hh_synth.rsa_cube(n, 0.1, seed=48)
    F, W = hh_synth.forces(n, 15), hh_synth.forces(n, 16)
    p = hh.Params(precision="fp64")
    gF, gX, gT, _ = grads(ctx, X, F, W, p)
    pp = hh.Params(precision="fp64", pivots_only=True)
    t = ctx.build_tree(cuda(X), pp)
    h = ctx.aca(t, ctx.partition(t, pp), pp)
    with pytest.raises(hh.HHError):
        ctx.matvec(h, cuda(F))
    gF2 = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    gX2 = torch.zeros_like(gF2)
    gT2 = torch.zeros(len(THETA), dtype=torch.float32, device="cuda")
    ctx.matvec_backward(h, cuda(W), cuda(F), gF=gF2, gX=gX2, gtheta=gT2)
    # factors rebuilt along the same pivots: equal up to summation order
    assert np.abs(gF2.cpu().numpy() - gF).max() <= 1e-12 * np.abs(gF).max()
    assert np.abs(gX2.cpu().numpy() - gX).max() <= 1e-10 * np.abs(gX).max()
    assert np.abs(gT2.cpu().numpy() - gT).max() <= 1e-5 * np.abs(gT).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradients_are_reproducible_and_budget_independent(ctx, prec):
    # fixed summation orders: a second call gives the same bits; a small
    # memory budget splits the admissible blocks into groups, which changes
    # only the order of the FP64 sums (within rounding)
    n = 6000
    X = hh_synth.gaussian_cloud(n, 30.0, seed=49)[0]
    F, W = hh_synth.forces(n, 17), hh_synth.forces(n, 18)
    p = hh.Params(precision=prec, leaf_size=32, pivots_only=True)
    gF1, gX1, gT1, _ = grads(ctx, X, F, W, p)
    gF2, gX2, gT2, _ = grads(ctx, X, F, W, p)
    assert np.array_equal(gF1, gF2) and np.array_equal(gX1, gX2) and np.array_equal(gT1, gT2)
    pb = hh.Params(precision=prec, leaf_size=32, pivots_only=True, mem_budget=8 << 20)
    gF3, gX3, gT3, _ = grads(ctx, X, F, W, pb)
    assert np.abs(gF3 - gF1).max() <= 1e-12 * np.abs(gF1).max()
    assert np.abs(gX3 - gX1).max() <= 1e-11 * np.abs(gX1).max()
    assert np.abs(gT3 - gT1).max() <= 1e-6 * np.abs(gT1).max()


def _golden_drop20k():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "grad_drop20k.txt")
    with open(path) as f:
        lines = [l for l in f if not l.startswith("#")]
    nt = int(lines[0].split()[1])
    gT = np.array([float(v) for v in lines[1:1 + nt]])
    nr = int(lines[1 + nt].split()[1])
    rows = np.array([[float(v) for v in l.split()] for l in lines[2 + nt:2 + nt + nr]])
    return gT, rows[:, 0].astype(np.int64), rows[:, 1:4], rows[:, 4:7]


def test_gradient_of_the_20k_drop_against_the_dense_oracle():
    # the differentiation workload at N = 20,000 (Gaussian drop, sigma = 30 a):
    # dL/dtheta in full and dL/dX, dL/dF on 128 rows against the FP64 dense
    # gradient over all pairs (tests/golden/make_grad_drop20k.py).  The
    # H-matrix gradient differs from the dense one by the ACA truncation:
    # about zeta in relative norm (measured: see the tolerances)
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "make_grad_drop20k", os.path.join(os.path.dirname(__file__), "golden", "make_grad_drop20k.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    X, F, W, rows, _ = mk.inputs()
    gTo, ro, gXo, gFo = _golden_drop20k()
    assert np.array_equal(ro, rows)
    c = hh.Context()
    c.set_mlp(THETA, 32)
    for prec, eps, tol in (("fp64", 1e-6, 1e-4), ("fp32", 1e-4, 3e-3)):
        p = hh.Params(precision=prec, eps=eps, leaf_size=64, pivots_only=True)
        gF, gX, gT, _ = grads(c, X, F, W, p)
        assert np.linalg.norm(gT - gTo) <= tol * np.linalg.norm(gTo), prec
        assert np.linalg.norm(gX[rows] - gXo) <= tol * np.linalg.norm(gXo), prec
        assert np.linalg.norm(gF[rows] - gFo) <= tol * np.linalg.norm(gFo), prec
