"""Short-range terms of Eq. 6 (M^(s,2) + M^(t,3) + M^(s,3)) on the GPU against
the FP64 oracle, alone and inside hh_predict."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import hh_synth
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402

THETA = hh_synth.mlp_params(32, 7)
TS32 = hh_synth.mlp_params(32, 21)
T332 = hh_synth.mlp_params(32, 22, n_in=7, n_out=12)
TS64 = hh_synth.mlp_params(64, 23)
T364 = hh_synth.mlp_params(64, 24, n_in=7, n_out=12)
TOL = {"fp64": 1e-12, "fp32": 2e-5}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(torch.float64).cuda()


def make_ctx(width=32, ts=True, t3=True, rcut=5.0):
    c = hh.Context()
    c.set_mlp(THETA, 32)
    s, t = (TS32, T332) if width == 32 else (TS64, T364)
    c.set_short_range(s if ts else None, t if t3 else None, width, rcut)
    return c


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("width", [32, 64])
def test_against_oracle(prec, width):
    n = 1500
    X = hh_synth.rsa_cube(n, 0.2, seed=61)
    F = hh_synth.forces(n, 62)
    c = make_ctx(width)
    U = c.short_range(cuda(X), cuda(F), hh.Params(precision=prec)).cpu().numpy()
    ts, t3 = (TS32, T332) if width == 32 else (TS64, T364)
    Uo = oracle.short_range(X, F, ts, width, t3, width, rcut=5.0)
    assert np.abs(Uo).max() > 0
    assert oracle.rel_error(Uo, U) < TOL[prec]
    # neighbour pairs: the directed count within R_cut
    pairs = cKDTree(X).query_pairs(5.0 - 1e-12, output_type="ndarray")
    d = np.linalg.norm(X[pairs[:, 0]] - X[pairs[:, 1]], axis=1)
    assert c.stats()["n_short_pairs"] == 2 * int((d < 5.0).sum())


def test_each_term_and_linearity():
    n = 800
    X = hh_synth.rsa_cube(n, 0.25, seed=63)
    F = hh_synth.forces(n, 64)
    p = hh.Params(precision="fp64")
    U2 = make_ctx(t3=False).short_range(cuda(X), cuda(F), p).cpu().numpy()
    U3 = make_ctx(ts=False).short_range(cuda(X), cuda(F), p).cpu().numpy()
    U = make_ctx().short_range(cuda(X), cuda(F), p).cpu().numpy()
    assert oracle.rel_error(oracle.short_range(X, F, TS32, 32, None, 32), U2) < 1e-12
    assert oracle.rel_error(oracle.short_range(X, F, None, 32, T332, 32), U3) < 1e-12
    assert oracle.rel_error(U, U2 + U3) < 1e-13


def test_batched_suspensions_do_not_interact():
    # two suspensions occupying the same region of space
    sizes = [600, 700]
    Xs = [hh_synth.rsa_cube(s, 0.2, seed=70 + i) for i, s in enumerate(sizes)]
    Fs = [hh_synth.forces(s, 80 + i) for i, s in enumerate(sizes)]
    off = np.array([0, sizes[0], sizes[0] + sizes[1]])
    c = make_ctx()
    p = hh.Params(precision="fp64")
    Ub = c.short_range(cuda(np.concatenate(Xs)), cuda(np.concatenate(Fs)), p, offsets=off).cpu().numpy()
    for i in range(2):
        Ui = c.short_range(cuda(Xs[i]), cuda(Fs[i]), p).cpu().numpy()
        assert np.array_equal(Ub[off[i]:off[i + 1]], Ui)


def test_sparse_and_deterministic():
    X = hh_synth.rsa_cube(300, 0.001, seed=65)        # mean spacing >> R_cut: almost no neighbours
    F = hh_synth.forces(300, 66)
    c = make_ctx()
    p = hh.Params(precision="fp32")
    a = c.short_range(cuda(X), cuda(F), p).cpu().numpy()
    ao = oracle.short_range(X, F, TS32, 32, T332, 32)
    assert np.array_equal(a == 0, ao == 0)                 # the same particles have no neighbours
    assert oracle.rel_error(ao, a) < 2e-5
    X2 = hh_synth.rsa_cube(3000, 0.2, seed=67)
    F2 = hh_synth.forces(3000, 68)
    u1 = c.short_range(cuda(X2), cuda(F2), p).cpu().numpy()
    u2 = c.short_range(cuda(X2), cuda(F2), p).cpu().numpy()
    assert np.array_equal(u1, u2)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_predict_with_short_range(prec):
    n = 2500
    X = hh_synth.rsa_cube(n, 0.1, seed=69)
    F = hh_synth.forces(n, 70)
    c = make_ctx()
    p0 = hh.Params(precision=prec)
    p1 = hh.Params(precision=prec, short_range=True)
    U0 = c.predict(cuda(X), cuda(F), p0).cpu().numpy()
    U1 = c.predict(cuda(X), cuda(F), p1).cpu().numpy()
    st = c.stats()
    assert st["n_short_pairs"] > 0 and st["t_short"] > 0
    Us = oracle.short_range(X, F, TS32, 32, T332, 32)
    tol = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 1e-5}[prec]
    assert oracle.rel_error(Us, U1 - U0) < tol
    # staged product with the flag; its transpose and the adjoint refuse it
    t = c.build_tree(cuda(X), p1)
    h = c.aca(t, c.partition(t, p1), p1)
    Um = c.matvec(h, cuda(F)).cpu().numpy()
    assert oracle.rel_error(U1, Um) < {"fp64": 1e-12, "fp32": 1e-6, "bf16": 1e-6}[prec]
    with pytest.raises(hh.HHError):
        c.matvec(h, cuda(F), transpose=True)
    with pytest.raises(hh.HHError):
        c.matvec_backward(h, cuda(F), cuda(F), gF=torch.zeros((n, 3), dtype=torch.float64, device="cuda"))


def test_flag_needs_networks():
    c = hh.Context()
    c.set_mlp(THETA, 32)
    X = cuda(hh_synth.rsa_cube(100, 0.1, seed=1))
    with pytest.raises(hh.HHError):
        c.predict(X, X, hh.Params(short_range=True))
