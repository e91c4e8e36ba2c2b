"""FP64 CPU oracle for the H-HIGNN mobility product (test infrastructure).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg use
this package.  It wraps ``oracle.c`` (plain C, OpenMP, no FMA contraction)
through ctypes and shares nothing with the CUDA library.

Every function is pinned by ``-m "not gpu"`` tests (tests/test_oracle_*.py)
against closed forms, invariants, brute force or library routines; ``PINS``
lists what pins each part.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

PINS = {
    "pair_block (RPY)": "closed-form RPY values at r = 2, 5, 100; symmetry; continuity at r = 2a",
    "pair_block (MLP)": "SiLU pairs that make the network exactly affine; constant-output network against "
                        "scipy distances; block symmetry; width-32/64 layouts",
    "dense_matvec": "two-particle closed form; rows equal to dense_matrix products; RPY symmetry",
    "dense_matvec_multi": "equals dense_matvec per force vector, bit for bit (same summation order)",
    "morton": "hand-derived codes for grid-aligned points",
    "tree": "Definition 1 invariants; hand-derived 1-D bisection",
    "partition": "exact cover of all (i, j); symmetry; brute-force admissibility over node pairs; "
                 "hand-derived 1-D partition",
    "aca": "exact reproduction of rank-r blocks; error vs numpy SVD (Eckart-Young); lambda^2 = |CQ|_F^2",
    "hmatvec": "equals the dense product when nothing is admissible; eps_r <= zeta; decreasing in zeta",
    "grad": "central finite differences of the dense product; gF against the dense matrix transpose",
    "train": "finite differences of the Eq. 5 loss; Adam step against its closed form",
    "mlp_gen": "equals the pinned 4 -> w -> w -> w -> 6 pair MLP for those sizes",
    "short_range": "constant-output networks against a distance-matrix formulation (numpy); hand-derived "
                   "3-particle cliques; translation invariance; permutation equivariance",
    "filament_energy": "closed forms: stretched bond, right-angle and folded joints, straight chain under gravity",
    "filament_forces": "central differences of filament_energy; the two-bead spring; zero net internal force and "
                       "torque per chain; straight chains at rest length feel gravity only",
    "euler_step": "composition of filament_forces, hmatvec and x + dt U (each pinned)",
    "simulate": "two identical spheres under RPY sediment together at the closed-form velocity; dt = 0 keeps X; "
                "one step equals euler_step",
    "recompress": "matrices of prescribed singular values: the kept rank and the error are the Eckart-Young "
                  "ones; exact for rank-deficient factors; error <= eps_rc ||M||_F on ACA blocks",
}


def build(force: bool = False) -> str:
    """Compile liboracle.so next to this file (gcc, OpenMP, no FMA)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _declare(_lib)
    return _lib


class Kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("width", ctypes.c_int), ("theta", ctypes.c_void_p),
                ("a", ctypes.c_double), ("mu", ctypes.c_double)]


class HStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("n_nodes", "nG", "nH", "n_near_pairs", "n_aca_entries", "rank_sum", "rank_max", "rank_capped")]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double


def _declare(L):
    sig = {
        "or_mlp_forward": (None, [_P, _I, _P, _P]),
        "or_pair_block": (None, [_P, _P, _P]),
        "or_self_mobility": (_D, [_D, _D]),
        "or_dense_matvec": (None, [_I, _P, _P, _P, _P, _I64, _I, _P]),
        "or_dense_matrix": (None, [_I, _P, _P, _I, _P]),
        "or_dense_matvec_multi": (None, [_I, _P, _I, _P, _P, _P, _I64, _I, _P]),
        "or_dense_grad": (None, [_I, _P, _P, _P, _P, _I, _P, _P, _P]),
        "or_train_loss_grad": (_D, [_P, _I, _I64, _P, _P, _P, _D, _P]),
        "or_adam_step": (None, [_P, _P, _P, _P, _I64, _D, _D, _D, _D, _I]),
        "or_morton_codes": (None, [_I, _P, _P]),
        "or_morton_sort": (None, [_I, _P, _P, _P]),
        "or_build_tree": (_I, [_I, _P, _P, _I, _I, _P, _P, _P, _P, _P, _P]),
        "or_admissible": (_I, [_P, _P, _I, _I, _D]),
        "or_partition": (_I, [_I, _P, _P, _P, _P, _P, _I, _D, _P, _I64, _P, _P, _I64, _P]),
        "or_aca_block": (_I, [_P, _P, _I, _I, _I, _I, _D, _I, _I, _P, _P, _P, _P, _P, _P]),
        "or_aca_dense": (_I, [_P, _I, _I, _D, _I, _I, _P, _P, _P, _P, _P, _P]),
        "or_j1": (_I, [_I, ctypes.c_uint64, _I, _I, _I]),
        "or_hmatvec": (_I, [_I, _P, _P, _P, _I, _D, _D, _I, _I, ctypes.c_uint64, _I, _P, _P, _P, _P, _P, _I64]),
        "or_rel_error": (_D, [_I64, _P, _P]),
        "or_num_threads": (_I, []),
        "or_mlp_gen": (None, [_P, _I, _I, _I, _P, _P]),
        "or_short_range": (None, [_I, _P, _P, _P, _I, _P, _I, _D, _D, _P]),
        "or_filament_energy": (_D, [_I, _I, _P, _D, _D, _D, _P]),
        "or_filament_forces": (None, [_I, _I, _P, _D, _D, _D, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class PairKernel:
    """Kernel description for the C side (keeps theta alive)."""

    def __init__(self, kind: str = "mlp", theta=None, width: int = 32, a: float = 1.0, mu: float = 1.0):
        self.kind = kind
        self.theta = _f64(theta) if theta is not None else np.zeros(1)
        self.width = int(width)
        self.a = float(a)
        self.mu = float(mu)
        self.c = Kernel(0 if kind == "mlp" else 1, self.width, self.theta.ctypes.data, self.a, self.mu)

    @property
    def ref(self):
        return ctypes.byref(self.c)


def mlp_forward(theta, width, f):
    o = np.zeros(6)
    lib().or_mlp_forward(_ptr(_f64(theta)), width, _ptr(_f64(f)), _ptr(o))
    return o


def pair_block(kernel: PairKernel, r):
    K = np.zeros(9)
    lib().or_pair_block(kernel.ref, _ptr(_f64(r)), _ptr(K))
    return K.reshape(3, 3)


def self_mobility(a=1.0, mu=1.0):
    return lib().or_self_mobility(a, mu)


def dense_matvec(X, F, kernel: PairKernel, rows=None, with_self=True):
    X = _f64(X); F = _f64(F)
    n = X.shape[0]
    if rows is not None:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        U = np.zeros((len(rows), 3))
        lib().or_dense_matvec(n, _ptr(X), _ptr(F), kernel.ref, _ptr(rows), len(rows), int(with_self), _ptr(U))
    else:
        U = np.zeros((n, 3))
        lib().or_dense_matvec(n, _ptr(X), _ptr(F), kernel.ref, None, n, int(with_self), _ptr(U))
    return U


def dense_matvec_multi(X, Fs, kernel: PairKernel, rows=None, with_self=True):
    """dense_matvec for up to 8 force vectors Fs [nf, n, 3] at once (each pair
    block evaluated once); returns [nf, rows or n, 3]."""
    X = _f64(X); Fs = _f64(Fs)
    n, nf = X.shape[0], Fs.shape[0]
    if not 1 <= nf <= 8:
        raise ValueError("1 to 8 force vectors")
    r = np.ascontiguousarray(rows, dtype=np.int64) if rows is not None else None
    nr = len(r) if r is not None else n
    U = np.zeros((nf, nr, 3))
    lib().or_dense_matvec_multi(n, _ptr(X), nf, _ptr(Fs), kernel.ref, _ptr(r), nr, int(with_self), _ptr(U))
    return U


def dense_matrix(X, kernel: PairKernel, with_self=True):
    X = _f64(X)
    n = X.shape[0]
    M = np.zeros((3 * n, 3 * n))
    lib().or_dense_matrix(n, _ptr(X), kernel.ref, int(with_self), _ptr(M))
    return M


def dense_grad(X, F, W, kernel: PairKernel, with_self=True):
    """(gF, gX, gtheta) of L = sum_i W_i . U_i with U the dense product."""
    X = _f64(X); F = _f64(F); W = _f64(W)
    n = X.shape[0]
    gF = np.zeros((n, 3)); gX = np.zeros((n, 3)); gT = np.zeros(len(kernel.theta))
    lib().or_dense_grad(n, _ptr(X), _ptr(F), _ptr(W), kernel.ref, int(with_self), _ptr(gF), _ptr(gX), _ptr(gT))
    return gF, gX, gT


def train_loss_grad(theta, width, r, e, U, a=1.0, grad=True):
    theta = _f64(theta); r = _f64(r); e = _f64(e); U = _f64(U)
    g = np.zeros(len(theta)) if grad else None
    L = lib().or_train_loss_grad(_ptr(theta), width, r.shape[0], _ptr(r), _ptr(e), _ptr(U), a, _ptr(g))
    return (L, g) if grad else L


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays theta, m, v."""
    lib().or_adam_step(_ptr(theta), _ptr(_f64(g)), _ptr(m), _ptr(v), len(theta), lr, b1, b2, eps, t)


def morton_codes(X):
    X = _f64(X)
    c = np.zeros(X.shape[0], dtype=np.uint64)
    lib().or_morton_codes(X.shape[0], _ptr(X), _ptr(c))
    return c


def morton_sort(codes):
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    n = len(codes)
    perm = np.zeros(n, dtype=np.int32)
    sc = np.zeros(n, dtype=np.uint64)
    lib().or_morton_sort(n, _ptr(codes), _ptr(perm), _ptr(sc))
    return perm, sc


class Tree:
    def __init__(self, perm, codes, Xs, begin, end, child, parent, lo, hi):
        self.perm, self.codes, self.Xs = perm, codes, Xs
        self.begin, self.end, self.child, self.parent, self.lo, self.hi = begin, end, child, parent, lo, hi

    @property
    def n_nodes(self):
        return len(self.begin)

    def size(self, i):
        return int(self.end[i] - self.begin[i])


def build_tree(X, leaf):
    X = _f64(X)
    n = X.shape[0]
    codes = morton_codes(X)
    perm, sc = morton_sort(codes)
    Xs = np.ascontiguousarray(X[perm])
    cap = 2 * n + 1
    nb = np.zeros(cap, np.int32); ne = np.zeros(cap, np.int32)
    ch = np.zeros((cap, 2), np.int32); par = np.zeros(cap, np.int32)
    lo = np.zeros((cap, 3)); hi = np.zeros((cap, 3))
    nn = lib().or_build_tree(n, _ptr(sc), _ptr(Xs), int(leaf), cap, _ptr(nb), _ptr(ne), _ptr(ch), _ptr(par),
                             _ptr(lo), _ptr(hi))
    if nn < 0:
        raise RuntimeError("tree capacity exceeded")
    return Tree(perm, sc, Xs, nb[:nn].copy(), ne[:nn].copy(), ch[:nn].copy(), par[:nn].copy(),
                lo[:nn].copy(), hi[:nn].copy())


def admissible(tree: Tree, t, s, eta):
    return bool(lib().or_admissible(_ptr(tree.lo), _ptr(tree.hi), int(t), int(s), float(eta)))


def partition(tree: Tree, leaf, eta):
    capG = capH = 1 << 14
    while True:
        G = np.zeros((capG, 2), np.int32); H = np.zeros((capH, 2), np.int32)
        nG = ctypes.c_int64(); nH = ctypes.c_int64()
        rc = lib().or_partition(tree.n_nodes, _ptr(tree.begin), _ptr(tree.end), _ptr(tree.child), _ptr(tree.lo),
                                _ptr(tree.hi), int(leaf), float(eta), _ptr(G), capG, ctypes.byref(nG), _ptr(H), capH,
                                ctypes.byref(nH))
        if rc == 0:
            return G[: nG.value].copy(), H[: nH.value].copy()
        capG = max(capG, nG.value) * 4
        capH = max(capH, nH.value) * 4


def aca_block(kernel: PairKernel, Xs, t0, c, s0, q, eps, max_rank, j1=0):
    Xs = _f64(Xs)
    C = np.zeros((max_rank, c, 3, 3)); Q = np.zeros((max_rank, q, 3, 3))
    I = np.zeros(max_rank, np.int32); J = np.zeros(max_rank, np.int32)
    l2 = ctypes.c_double(); fl = ctypes.c_int(0)
    l = lib().or_aca_block(kernel.ref, _ptr(Xs), t0, c, s0, q, eps, max_rank, j1, _ptr(C), _ptr(Q), _ptr(I),
                           _ptr(J), ctypes.byref(l2), ctypes.byref(fl))
    return dict(rank=l, C=C[:l], Q=Q[:l], I=I[:l], J=J[:l], lambda2=l2.value, capped=bool(fl.value & 1))


def aca_dense(G, eps, max_rank, j1=0):
    """ACA of an explicit block G [c, q, 3, 3] of 3x3 elements."""
    G = _f64(G)
    c, q = G.shape[:2]
    C = np.zeros((max_rank, c, 3, 3)); Q = np.zeros((max_rank, q, 3, 3))
    I = np.zeros(max_rank, np.int32); J = np.zeros(max_rank, np.int32)
    l2 = ctypes.c_double(); fl = ctypes.c_int(0)
    l = lib().or_aca_dense(_ptr(G), c, q, eps, max_rank, j1, _ptr(C), _ptr(Q), _ptr(I), _ptr(J),
                           ctypes.byref(l2), ctypes.byref(fl))
    return dict(rank=l, C=C[:l], Q=Q[:l], I=I[:l], J=J[:l], lambda2=l2.value, capped=bool(fl.value & 1))


def j1(rule, seed, t, s, q):
    return lib().or_j1(rule, seed, t, s, q)


def hmatvec(X, F, kernel: PairKernel, leaf=32, eta=1.0, eps=1e-4, max_rank=48, j1_rule=0, seed=0,
            with_self=True, want_ranks=False):
    """H-matrix product in FP64; returns (U, stats)."""
    X = _f64(X); F = _f64(F)
    n = X.shape[0]
    U = np.zeros((n, 3))
    st = HStats()
    ranks = pI = pJ = None
    cap = 0
    if want_ranks:
        tree = build_tree(X, leaf)
        G, _ = partition(tree, leaf, eta)
        cap = len(G)
        ranks = np.zeros(max(cap, 1), np.int32)
        pI = np.zeros(max(cap, 1) * max_rank, np.int32)
        pJ = np.zeros(max(cap, 1) * max_rank, np.int32)
    rc = lib().or_hmatvec(n, _ptr(X), _ptr(F), kernel.ref, leaf, eta, eps, max_rank, j1_rule, seed,
                          int(with_self), _ptr(U), ctypes.byref(st), _ptr(ranks), _ptr(pI), _ptr(pJ), cap)
    if rc != 0:
        raise RuntimeError(f"or_hmatvec failed ({rc})")
    stats = {f[0]: getattr(st, f[0]) for f in HStats._fields_}
    if want_ranks:
        stats["ranks"] = ranks[:cap]
        stats["pivI"] = pI[: cap * max_rank].reshape(cap, max_rank)
        stats["pivJ"] = pJ[: cap * max_rank].reshape(cap, max_rank)
    return U, stats


def rel_error(ref, approx):
    ref = _f64(ref).ravel(); approx = _f64(approx).ravel()
    return lib().or_rel_error(ref.size, _ptr(ref), _ptr(approx))


def num_threads():
    return lib().or_num_threads()


def mlp_gen(theta, n_in, width, n_out, f):
    """MLP n_in -> width x 3 -> n_out (SiLU), FP64."""
    th = _f64(theta)
    f = _f64(f)
    o = np.zeros(n_out)
    lib().or_mlp_gen(_ptr(th), n_in, width, n_out, _ptr(f), _ptr(o))
    return o


def short_range(X, F, theta_s=None, ws=32, theta_3=None, w3=32, rcut=5.0, a=1.0):
    """Short-range terms of Eq. 6 (M^(s,2) + M^(t,3) + M^(s,3)) F for one suspension (FP64)."""
    X, F = _f64(X), _f64(F)
    ts = _f64(theta_s) if theta_s is not None else None
    t3 = _f64(theta_3) if theta_3 is not None else None
    U = np.zeros_like(X)
    lib().or_short_range(len(X), _ptr(X), _ptr(F), _ptr(ts), ws, _ptr(t3), w3, float(rcut), float(a), _ptr(U))
    return U


def filament_energy(X, beads, k=100.0, l0=2.2, kappa=10.0, g=(0.0, 0.0, -1.0)):
    """Bond + bending + gravity energy of chains of `beads` consecutive rows (FP64)."""
    X = _f64(X)
    nch = len(X) // beads if beads > 0 else 0
    return lib().or_filament_energy(nch, beads, _ptr(X), k, l0, kappa, _ptr(_f64(g)))


def filament_forces(X, beads, k=100.0, l0=2.2, kappa=10.0, g=(0.0, 0.0, -1.0)):
    """Bead forces -grad filament_energy, [n, 3] FP64."""
    X = _f64(X)
    nch = len(X) // beads if beads > 0 else 0
    F = np.zeros_like(X)
    lib().or_filament_forces(nch, beads, _ptr(X), k, l0, kappa, _ptr(_f64(g)), _ptr(F))
    return F


def euler_step(X, beads, kernel, dt, leaf=32, eta=1.0, eps=1e-4, max_rank=48, k=100.0, l0=2.2, kappa=10.0,
               g=(0.0, 0.0, -1.0)):
    """One explicit Euler step of the filament suspension: F = F(X),
    U = alpha_1 F + M_H F (the oracle's H-matrix product), X + dt U.
    Returns (X_new, F, U)."""
    X = _f64(X)
    F = filament_forces(X, beads, k, l0, kappa, g)
    U, _ = hmatvec(X, F, kernel, leaf=leaf, eta=eta, eps=eps, max_rank=max_rank)
    return X + dt * U, F, U


def simulate(X, n_chains, beads, kernel, dt, n_steps, dump_every=1, leaf=32, eta=1.0, eps=1e-4, max_rank=48,
             k=100.0, l0=2.2, kappa=10.0, g=(0.0, 0.0, -1.0)):
    """n_steps explicit Euler steps (Section 2.5) of chains (the first
    n_chains * beads rows, forces of filament_forces) and free particles (the
    remaining rows, force g): F = F(X), U = alpha_1 F + M_H F (hmatvec),
    X <- X + dt U.  Returns the list of X at step 0 and at every step
    divisible by dump_every."""
    X = _f64(X).copy()
    nc = n_chains * beads
    dumps = [X.copy()]
    for step in range(1, n_steps + 1):
        F = np.empty_like(X)
        F[:nc] = filament_forces(X[:nc], beads, k, l0, kappa, g) if nc else F[:0]
        F[nc:] = np.asarray(g, dtype=np.float64)
        U, _ = hmatvec(X, F, kernel, leaf=leaf, eta=eta, eps=eps, max_rank=max_rank)
        X = X + dt * U
        if dump_every and step % dump_every == 0:
            dumps.append(X.copy())
    return dumps


def block_matrix(C, Q):
    """The scalar form M = sum_k C_k Q_k (3c x 3q) of a block's 3x3 factors,
    C [l, c, 3, 3] and Q [l, q, 3, 3] as aca_block returns them: entry
    (3m + a, 3n + b) = sum_k sum_x C_k(m)[a][x] Q_k(n)[x][b]."""
    C = _f64(C); Q = _f64(Q)
    l, c = C.shape[:2]
    q = Q.shape[1]
    if l == 0:
        return np.zeros((3 * c, 3 * q))
    Cs = C.transpose(1, 2, 0, 3).reshape(3 * c, 3 * l)      # row 3m + a, column 3k + x
    Qs = Q.transpose(0, 2, 1, 3).reshape(3 * l, 3 * q)      # row 3k + x, column 3n + b
    return Cs @ Qs


def recompress(C, Q, eps_rc):
    """Truncated SVD of a block's ACA approximant (the paper stores the ACA
    factors unchanged; this is the textbook best rank-r approximation,
    Eckart-Young): with M = block_matrix(C, Q) = sum_i s_i u_i v_i^T, the
    smallest r with sum_{i >= r} s_i^2 <= eps_rc^2 sum_i s_i^2.  Returns
    (U [3c, r] = the u_i s_i, V [r, 3q] = the v_i^T, r, s)."""
    M = block_matrix(C, Q)
    if M.size == 0:
        return np.zeros((M.shape[0], 0)), np.zeros((0, M.shape[1])), 0, np.zeros(0)
    u, s, vt = np.linalg.svd(M, full_matrices=False)
    tot = float(np.sum(s * s))
    r, tail = len(s), 0.0
    while r > 0 and tail + s[r - 1] ** 2 <= eps_rc * eps_rc * tot:
        tail += s[r - 1] ** 2
        r -= 1
    return u[:, :r] * s[:r], vt[:r], r, s
