"""On-GPU training of the pair MLP (Section 2.3, Eq. 5) against the FP64
oracle: loss, gradient, Adam, the RPY teacher, a short training run, and the
gain of the trained network inside the H-matrix product."""
import numpy as np
import pytest

import hh_synth
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402


def cuda(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()


def rpy_teacher(r, e):
    k = oracle.PairKernel("rpy")
    return np.stack([oracle.pair_block(k, ri) @ ei for ri, ei in zip(r, e)])


@pytest.fixture(scope="module")
def ctx():
    return hh.Context()


@pytest.mark.parametrize("width", [32, 64])
def test_loss_and_gradient_match_oracle(ctx, width):
    r, e = hh_synth.two_particle_samples(513, seed=1)
    U = rpy_teacher(r, e)
    th = hh_synth.mlp_params(width, 3)
    L, g = ctx.train_loss_grad(cuda(th, torch.float32), width, cuda(r), cuda(e), cuda(U))
    Lo, go = oracle.train_loss_grad(th.astype(np.float64), width, r, e, U)
    assert L == pytest.approx(Lo, rel=2e-5)
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - go) <= 2e-4 * np.linalg.norm(go)


def test_gpu_rpy_teacher_matches_oracle(ctx):
    r, e = hh_synth.two_particle_samples(1000, seed=2, dmin=0.5)   # includes the overlapping branch r < 2a
    U = rpy_teacher(r, e)
    th = cuda(hh_synth.mlp_params(32, 3), torch.float32)
    L_given, _ = ctx.train_loss_grad(th, 32, cuda(r), cuda(e), cuda(U), grad=False)
    L_gpu, _ = ctx.train_loss_grad(th, 32, cuda(r), cuda(e), None, grad=False)
    assert L_gpu == pytest.approx(L_given, rel=1e-5)


def test_adam_step_matches_oracle(ctx):
    width = 32
    r, e = hh_synth.two_particle_samples(256, seed=3)
    th = hh_synth.mlp_params(width, 5)
    t = cuda(th, torch.float32)
    m = torch.zeros_like(t); v = torch.zeros_like(t)
    for step in (1, 2, 3):
        thn = t.cpu().numpy().astype(np.float64)
        mn = m.cpu().numpy().astype(np.float64); vn = v.cpu().numpy().astype(np.float64)
        _, go = oracle.train_loss_grad(thn, width, r, e, rpy_teacher(r, e))
        ctx.train_step(t, m, v, step, width, cuda(r), cuda(e), None, lr=1e-3)
        oracle.adam_step(thn, go, mn, vn, step, lr=1e-3)
        assert np.max(np.abs(t.cpu().numpy() - thn)) < 2e-6


def train(ctx, width=32, steps=1500, batch=4096, lr=2e-3, seed=0):
    th = cuda(hh_synth.mlp_params(width, 7), torch.float32)
    m = torch.zeros_like(th); v = torch.zeros_like(th)
    losses = []
    for s in range(1, steps + 1):
        r, e = hh_synth.two_particle_samples(batch, seed=1000 * seed + s)
        lr_s = lr * (0.1 ** (s / steps))
        losses.append(ctx.train_step(th, m, v, s, width, cuda(r), cuda(e), None, lr=lr_s))
    return th, losses


@pytest.fixture(scope="module")
def trained(ctx):
    return train(ctx)


def test_training_reduces_held_out_loss(ctx, trained):
    th, losses = trained
    r, e = hh_synth.two_particle_samples(8192, seed=424242)
    L_end, _ = ctx.train_loss_grad(th, 32, cuda(r), cuda(e), None, grad=False)
    L_0, _ = ctx.train_loss_grad(cuda(hh_synth.mlp_params(32, 7), torch.float32), 32, cuda(r), cuda(e), None,
                                 grad=False)
    print(f"held-out Eq. 5 loss: untrained {L_0:.3e}, trained {L_end:.3e}")
    assert L_end < 1e-2 * L_0 and L_end < 1e-2


def test_gain_of_trained_network_in_hmatrix(ctx, trained):
    """eps against the dense RPY product: trained H-HIGNN << untrained, alpha_1 only."""
    th, _ = trained
    n = 4000
    X = hh_synth.rsa_cube(n, 0.1, seed=31)
    F = hh_synth.forces(n, 0)
    Ud = oracle.dense_matvec(X, F, oracle.PairKernel("rpy"))
    theta_trained = hh_synth.round_bf16(th.cpu().numpy())      # the canonical bf16 network
    errs = {}
    for name, theta in (("trained", theta_trained), ("untrained", hh_synth.mlp_params(32, 7))):
        c = hh.Context()
        c.set_mlp(theta, 32)
        U = c.predict(cuda(X), cuda(F), hh.Params(precision="fp32")).cpu().numpy()
        errs[name] = oracle.rel_error(Ud, U)
    errs["alpha1_only"] = oracle.rel_error(Ud, oracle.self_mobility() * F)
    print("eps vs dense RPY:", errs)
    assert errs["trained"] < 0.1 * errs["untrained"] and errs["trained"] < 0.1 * errs["alpha1_only"]
