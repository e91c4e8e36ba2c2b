"""B300-native H-HIGNN mobility product: thin Python binding of libhhignn.so.

Argument marshalling only: every step of the computation runs in the CUDA
library (``csrc/``), reached through the C-ABI of ``include/hhignn.h``.
PyTorch supplies device memory and streams.  There is no CPU fallback: if the
shared library is missing or cannot be loaded, ``lib()`` raises.

    import torch, paper_2505_08174_b300 as hh
    ctx = hh.Context()
    ctx.set_mlp(theta, width=32)
    U = ctx.predict(X, F, hh.Params(eps=1e-4))          # X, F: [N,3] float64 cuda
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhhignn.so")

HH_OK, HH_ERR_ARG, HH_ERR_CUDA, HH_ERR_OOM, HH_ERR_TIMEOUT, HH_ERR_NUMERIC, HH_WARN_RANK_CAP = range(7)
HH_FP64, HH_FP32, HH_BF16 = 0, 1, 2
HH_MLP, HH_RPY = 0, 1
STATUS_NAMES = {0: "HH_OK", 1: "HH_ERR_ARG", 2: "HH_ERR_CUDA", 3: "HH_ERR_OOM", 4: "HH_ERR_TIMEOUT",
                5: "HH_ERR_NUMERIC", 6: "HH_WARN_RANK_CAP"}
PRECISIONS = {"fp64": HH_FP64, "fp32": HH_FP32, "bf16": HH_BF16}
KERNELS = {"mlp": HH_MLP, "rpy": HH_RPY}

# Every function the header declares (checked by the CPU test-suite).
EXPORTS = [
    "hh_default_params", "hh_create", "hh_destroy", "hh_last_error", "hh_set_mlp", "hh_build_tree",
    "hh_partition", "hh_aca", "hh_matvec", "hh_predict", "hh_matvec_backward", "hh_export_tree",
    "hh_export_blocks", "hh_export_aca", "hh_export_factors", "hh_stats", "hh_tree_free", "hh_blocks_free", "hh_hmat_free",
    "hh_aca_block_apply_noalloc", "hh_eval_pairs", "hh_train_loss_grad", "hh_train_step",
    "hh_set_launch", "hh_get_launch", "hh_autotune", "hh_set_short_range", "hh_short_range",
    "hh_filament_forces", "hh_filament_step", "hh_probe_throughput", "hh_shard_owners",
    "hh_debug_fail_alloc", "hh_debug_stall_mma_waits", "hh_simulate", "hh_recompress", "hh_export_recompressed",
]


class HHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CParams(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("eta", ctypes.c_double), ("eps", ctypes.c_double),
                ("max_rank", ctypes.c_int32), ("precision", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("radius", ctypes.c_double), ("viscosity", ctypes.c_double), ("j1_rule", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("shard_id", ctypes.c_int32), ("n_shards", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("mem_budget", ctypes.c_int64)]


class CStats(ctypes.Structure):
    _fields_ = [("t_tree", ctypes.c_double), ("t_part", ctypes.c_double), ("t_near", ctypes.c_double),
                ("t_aca", ctypes.c_double), ("t_apply", ctypes.c_double), ("t_acc", ctypes.c_double),
                ("n_near_pairs", ctypes.c_int64), ("n_aca_queries", ctypes.c_int64),
                ("n_blocks_G", ctypes.c_int64), ("n_blocks_H", ctypes.c_int64), ("n_nodes", ctypes.c_int64),
                ("rank_hist", ctypes.c_int64 * 65), ("t_kernel_aca", ctypes.c_double),
                ("t_kernel_near", ctypes.c_double), ("n_launches", ctypes.c_int64), ("t_short", ctypes.c_double),
                ("n_short_pairs", ctypes.c_int64), ("mem_peak_bytes", ctypes.c_int64),
                ("n_aca_rounds", ctypes.c_int64), ("t_aca_tiles", ctypes.c_double), ("t_aca_steps", ctypes.c_double),
                ("n_aca_groups", ctypes.c_int64)]


class CLaunch(ctypes.Structure):
    _fields_ = [("small_max", ctypes.c_int32), ("aca_small_cps", ctypes.c_int32),
                ("aca_large_cps", ctypes.c_int32), ("near_cps", ctypes.c_int32), ("rounds_min_cq", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class CFilament(ctypes.Structure):
    """hh_filament_params: bond spring, rest length, bending stiffness, body force."""
    _fields_ = [("k_bond", ctypes.c_double), ("l0", ctypes.c_double), ("kappa", ctypes.c_double),
                ("g", ctypes.c_double * 3)]


def Filament(k_bond=100.0, l0=2.2, kappa=10.0, g=(0.0, 0.0, -1.0)) -> CFilament:
    return CFilament(float(k_bond), float(l0), float(kappa), (ctypes.c_double * 3)(*[float(v) for v in g]))


_P = ctypes.c_void_p
_lib = None


def lib():
    """Load libhhignn.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built; run `python -m paper_2505_08174_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        i32, i64, st = ctypes.c_int32, ctypes.c_int64, ctypes.c_int
        sig = {
            "hh_default_params": (None, [_P]),
            "hh_create": (st, [_P, ctypes.c_int]),
            "hh_destroy": (None, [_P]),
            "hh_last_error": (ctypes.c_char_p, [_P]),
            "hh_set_mlp": (st, [_P, _P, ctypes.c_int, ctypes.c_int, _P]),
            "hh_build_tree": (st, [_P, _P, _P, i32, _P, _P, _P]),
            "hh_partition": (st, [_P, _P, _P, _P, _P]),
            "hh_aca": (st, [_P, _P, _P, _P, _P, _P]),
            "hh_matvec": (st, [_P, _P, _P, _P, ctypes.c_int, _P]),
            "hh_predict": (st, [_P, _P, _P, _P, i32, _P, _P, _P]),
            "hh_matvec_backward": (st, [_P, _P, _P, _P, _P, _P, _P, _P]),
            "hh_export_tree": (st, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
            "hh_export_blocks": (st, [_P, _P, _P, _P, _P]),
            "hh_export_aca": (st, [_P, _P, _P, _P, _P, _P]),
            "hh_export_factors": (st, [_P, _P, _P, _P, _P]),
            "hh_probe_throughput": (st, [_P, i32, ctypes.c_int64, _P, _P]),
            "hh_shard_owners": (st, [_P, i32, _P, _P]),
            "hh_debug_fail_alloc": (None, [ctypes.c_int64]),
            "hh_recompress": (st, [_P, _P, ctypes.c_double, _P]),
            "hh_export_recompressed": (st, [_P, _P, _P, _P, _P, _P]),
            "hh_simulate": (st, [_P, _P, ctypes.c_int64, i32, ctypes.c_int64, _P, _P, ctypes.c_double, i32, i32, _P,
                                 _P, _P]),
            "hh_debug_stall_mma_waits": (st, [_P, ctypes.c_uint32]),
            "hh_stats": (st, [_P, _P]),
            "hh_tree_free": (None, [_P]),
            "hh_blocks_free": (None, [_P]),
            "hh_hmat_free": (None, [_P]),
            "hh_aca_block_apply_noalloc": (st, [_P, _P, i32, _P, i32, _P, _P, _P, _P, _P]),
            "hh_eval_pairs": (st, [_P, _P, i64, _P, _P, _P]),
            "hh_train_loss_grad": (st, [_P, _P, ctypes.c_int, _P, _P, _P, i64, ctypes.c_double, _P, _P, _P]),
            "hh_train_step": (st, [_P, _P, _P, _P, i64, ctypes.c_int, _P, _P, _P, i64, ctypes.c_double,
                                   ctypes.c_double, _P, _P]),
            "hh_set_launch": (st, [_P, _P]),
            "hh_get_launch": (st, [_P, _P]),
            "hh_autotune": (st, [_P, _P, _P, i32, _P, i32, _P, _P]),
            "hh_set_short_range": (st, [_P, _P, _P, ctypes.c_int, ctypes.c_double, _P]),
            "hh_short_range": (st, [_P, _P, _P, _P, i32, _P, _P, _P]),
            "hh_filament_forces": (st, [_P, _P, ctypes.c_int64, i32, _P, _P, _P]),
            "hh_filament_step": (st, [_P, _P, ctypes.c_int64, i32, _P, _P, ctypes.c_double, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


FLAG_SHORT_RANGE = 1
FLAG_PIVOTS_ONLY = 2


def debug_fail_alloc(n: int):
    """Test hook: the n-th device allocation of the library from now on fails
    (HH_ERR_OOM, with the call's temporaries freed); 0 cancels."""
    lib().hh_debug_fail_alloc(int(n))


def Params(leaf_size=32, eta=1.0, eps=1e-4, max_rank=48, precision="fp32", kernel="mlp", radius=1.0,
           viscosity=1.0, j1_rule=0, seed=0, shard_id=0, n_shards=1, short_range=False,
           pivots_only=False, mem_budget=0) -> CParams:
    p = CParams()
    lib().hh_default_params(ctypes.byref(p))
    p.leaf_size, p.eta, p.eps, p.max_rank = leaf_size, eta, eps, max_rank
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
    p.kernel = KERNELS[kernel] if isinstance(kernel, str) else kernel
    p.radius, p.viscosity, p.j1_rule, p.seed = radius, viscosity, j1_rule, seed
    p.shard_id, p.n_shards = shard_id, n_shards
    p.flags = (FLAG_SHORT_RANGE if short_range else 0) | (FLAG_PIVOTS_ONLY if pivots_only else 0)
    p.mem_budget = int(mem_budget)
    return p


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_xyz(t, name):
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 2 and t.shape[1] == 3 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous [N,3] float64 CUDA tensor")


class Context:
    """One hh_ctx on a CUDA device (owns the MLP copy, counters, status)."""

    def __init__(self, device: int | None = None):
        import torch
        self.device = torch.cuda.current_device() if device is None else device
        self._h = ctypes.c_void_p()
        self._check(lib().hh_create(ctypes.byref(self._h), self.device), "hh_create")
        self.width = None

    def _check(self, st, what, allow_warn=True):
        if st == HH_OK or (allow_warn and st == HH_WARN_RANK_CAP):
            return st
        msg = lib().hh_last_error(self._h).decode() if getattr(self, "_h", None) else ""
        raise HHError(st, f"{what}: {msg}")

    def close(self):
        if getattr(self, "_h", None):
            lib().hh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mlp(self, theta, width: int, stream=None):
        import torch
        th = torch.as_tensor(theta, dtype=torch.float32).to(f"cuda:{self.device}").contiguous()
        self._check(lib().hh_set_mlp(self._h, _dptr(th), width, 3, _stream(stream)), "hh_set_mlp")
        torch.cuda.current_stream().synchronize()
        self.width = width

    def predict(self, X, F, params: CParams, offsets=None, out=None, stream=None):
        """U = alpha_1 F + M_H F end to end (tree, partition, fused ACA, near, FP64 sum)."""
        import torch
        _check_xyz(X, "X"); _check_xyz(F, "F")
        n = X.shape[0]
        off = np.asarray([0, n] if offsets is None else offsets, dtype=np.int64)
        U = torch.empty_like(X) if out is None else out
        st = lib().hh_predict(self._h, _dptr(X), _dptr(F), off.ctypes.data_as(_P), len(off) - 1,
                              ctypes.byref(params), _stream(stream), _dptr(U))
        self.last_status = self._check(st, "hh_predict")
        return U

    def eval_pairs(self, r, params: CParams, stream=None):
        """K(r) [n, 3, 3] for separations r [n, 3] (float64 CUDA) in the params' precision."""
        import torch
        _check_xyz(r, "r")
        K = torch.empty((r.shape[0], 9), dtype=torch.float64, device=r.device)
        self._check(lib().hh_eval_pairs(self._h, _dptr(r), r.shape[0], ctypes.byref(params), _stream(stream),
                                        _dptr(K)), "hh_eval_pairs")
        return K.view(-1, 3, 3)

    # -- training (Eq. 5) -------------------------------------------------------
    def train_loss_grad(self, theta, width, r, e, U=None, radius=1.0, grad=True, stream=None):
        """(loss, grad) of Eq. 5 on the GPU; theta float32 CUDA, r/e/U float64 [B,3] CUDA."""
        import torch
        g = torch.empty_like(theta) if grad else None
        loss = ctypes.c_double()
        self._check(lib().hh_train_loss_grad(self._h, _dptr(theta), width, _dptr(r), _dptr(e),
                                             _dptr(U) if U is not None else None, r.shape[0], radius,
                                             _dptr(g) if g is not None else None, _stream(stream),
                                             ctypes.byref(loss)), "hh_train_loss_grad")
        return loss.value, g

    def train_step(self, theta, m, v, step, width, r, e, U=None, radius=1.0, lr=1e-3, stream=None):
        """One Adam step in place on theta, m, v (float32 CUDA); returns the loss before the step."""
        loss = ctypes.c_double()
        self._check(lib().hh_train_step(self._h, _dptr(theta), _dptr(m), _dptr(v), step, width, _dptr(r), _dptr(e),
                                        _dptr(U) if U is not None else None, r.shape[0], radius, lr,
                                        _stream(stream), ctypes.byref(loss)), "hh_train_step")
        return loss.value

    # -- short-range terms (Eq. 6: M^(s,2) + M^(t,3) + M^(s,3)) -------------------
    def set_short_range(self, theta_s, theta_3, width: int, r_cut: float = 5.0, stream=None):
        import torch
        dev = f"cuda:{self.device}"
        ts = None if theta_s is None else torch.as_tensor(theta_s, dtype=torch.float32).to(dev).contiguous()
        t3 = None if theta_3 is None else torch.as_tensor(theta_3, dtype=torch.float32).to(dev).contiguous()
        p = lambda t: _dptr(t) if t is not None else None
        self._check(lib().hh_set_short_range(self._h, p(ts), p(t3), int(width), float(r_cut), _stream(stream)),
                    "hh_set_short_range")

    def short_range(self, X, F, params: CParams, offsets=None, out=None, stream=None):
        """U (+)= the short-range terms for X, F (caller order); out is accumulated into when given."""
        import torch
        _check_xyz(X, "X"); _check_xyz(F, "F")
        off = np.asarray([0, X.shape[0]] if offsets is None else offsets, dtype=np.int64)
        U = torch.zeros_like(X) if out is None else out
        self._check(lib().hh_short_range(self._h, _dptr(X), _dptr(F), off.ctypes.data_as(_P), len(off) - 1,
                                         ctypes.byref(params), _stream(stream), _dptr(U)), "hh_short_range")
        return U

    # -- filament suspension: bead forces and the explicit Euler step -------------
    def filament_forces(self, X, beads, fil: CFilament = None, out=None, stream=None):
        """Bead forces of chains of `beads` consecutive rows of X (bond, bending, body force)."""
        import torch
        _check_xyz(X, "X")
        if beads < 1 or X.shape[0] % beads:
            raise ValueError("X must hold whole chains of `beads` rows")
        fil = Filament() if fil is None else fil
        F = torch.empty_like(X) if out is None else out
        self._check(lib().hh_filament_forces(self._h, _dptr(X), X.shape[0] // beads, int(beads), ctypes.byref(fil),
                                             _stream(stream), _dptr(F)), "hh_filament_forces")
        return F

    def filament_step(self, X, beads, params: CParams, dt, fil: CFilament = None, F=None, U=None, stream=None):
        """One explicit Euler step in place on X: F = forces(X), U = M(X) F, X += dt U.  Returns (F, U)."""
        import torch
        _check_xyz(X, "X")
        if beads < 1 or X.shape[0] % beads:
            raise ValueError("X must hold whole chains of `beads` rows")
        fil = Filament() if fil is None else fil
        F = torch.empty_like(X) if F is None else F
        U = torch.empty_like(X) if U is None else U
        st = lib().hh_filament_step(self._h, _dptr(X), X.shape[0] // beads, int(beads), ctypes.byref(fil),
                                    ctypes.byref(params), float(dt), _stream(stream), _dptr(F), _dptr(U))
        self.last_status = self._check(st, "hh_filament_step")
        return F, U

    def simulate(self, X, params: CParams, dt, n_steps, n_chains=0, beads=1, fil: CFilament = None, dump_every=0,
                 stream=None):
        """n_steps explicit Euler steps in place on X (chains first, then free
        particles feeling g only; see hh_simulate).  Returns (dumps, t_step_ms):
        dumps [n_steps // dump_every + 1, N, 3] float64 (None when dump_every
        is 0), t_step_ms [n_steps]."""
        _check_xyz(X, "X")
        n_free = X.shape[0] - n_chains * beads
        if n_chains < 0 or beads < 1 or n_free < 0:
            raise ValueError("X must hold n_chains chains of `beads` rows, then the free particles")
        fil = Filament() if fil is None else fil
        dumps = np.zeros((n_steps // dump_every + 1, X.shape[0], 3)) if dump_every > 0 else None
        ts = np.zeros(max(n_steps, 1))
        st = lib().hh_simulate(self._h, _dptr(X), int(n_chains), int(beads), int(n_free), ctypes.byref(fil),
                               ctypes.byref(params), float(dt), int(n_steps), int(dump_every),
                               dumps.ctypes.data_as(_P) if dumps is not None else None, ts.ctypes.data_as(_P),
                               _stream(stream))
        self.last_status = self._check(st, "hh_simulate")
        return dumps, ts[:n_steps]

    # -- launch shape and autotuner ---------------------------------------------
    def set_launch(self, small_max=0, aca_small_cps=0, aca_large_cps=0, near_cps=0, rounds_min_cq=0):
        c = CLaunch(small_max, aca_small_cps, aca_large_cps, near_cps, rounds_min_cq)
        self._check(lib().hh_set_launch(self._h, ctypes.byref(c)), "hh_set_launch")

    def get_launch(self) -> dict:
        c = CLaunch()
        self._check(lib().hh_get_launch(self._h, ctypes.byref(c)), "hh_get_launch")
        return c.as_dict()

    def autotune(self, X, params: CParams, reps=1, offsets=None, stream=None) -> dict:
        """Time hh_predict on X for candidate launch shapes; keep the fastest on this context."""
        _check_xyz(X, "X")
        off = np.asarray([0, X.shape[0]] if offsets is None else offsets, dtype=np.int64)
        c = CLaunch()
        self._check(lib().hh_autotune(self._h, _dptr(X), off.ctypes.data_as(_P), len(off) - 1, ctypes.byref(params),
                                      int(reps), _stream(stream), ctypes.byref(c)), "hh_autotune")
        return c.as_dict()

    PROBES = {"mufu_ex2": 0, "mufu_rcp": 1, "mufu_tanh": 2, "ffma": 3, "dfma": 4, "silu": 5}

    def probe(self, kind: str, iters: int = 1 << 16, stream=None) -> float:
        """Operations per second of one arithmetic unit (see hh_probe_throughput)."""
        v = ctypes.c_double()
        self._check(lib().hh_probe_throughput(self._h, self.PROBES[kind], int(iters), _stream(stream),
                                              ctypes.byref(v)), "hh_probe_throughput")
        return v.value

    def debug_stall_mma_waits(self, polls: int):
        """Test hook: MMA completion waits watch a barrier nothing arrives at
        for `polls` polls, so they run out (0: normal waits)."""
        self._check(lib().hh_debug_stall_mma_waits(self._h, int(polls)), "hh_debug_stall_mma_waits")

    def stats(self) -> dict:
        s = CStats()
        self._check(lib().hh_stats(self._h, ctypes.byref(s)), "hh_stats")
        d = {f: getattr(s, f) for f, _ in CStats._fields_ if f != "rank_hist"}
        d["rank_hist"] = list(s.rank_hist)
        return d

    # -- staged API -----------------------------------------------------------
    def build_tree(self, X, params: CParams, offsets=None, stream=None):
        _check_xyz(X, "X")
        off = np.asarray([0, X.shape[0]] if offsets is None else offsets, dtype=np.int64)
        h = ctypes.c_void_p()
        self._check(lib().hh_build_tree(self._h, _dptr(X), off.ctypes.data_as(_P), len(off) - 1,
                                        ctypes.byref(params), _stream(stream), ctypes.byref(h)), "hh_build_tree")
        return Tree(self, h)

    def partition(self, tree, params: CParams, stream=None):
        h = ctypes.c_void_p()
        self._check(lib().hh_partition(self._h, tree._h, ctypes.byref(params), _stream(stream), ctypes.byref(h)),
                    "hh_partition")
        return Blocks(self, h, tree)

    def aca(self, tree, blocks, params: CParams, stream=None):
        h = ctypes.c_void_p()
        st = lib().hh_aca(self._h, tree._h, blocks._h, ctypes.byref(params), _stream(stream), ctypes.byref(h))
        self._check(st, "hh_aca")
        hm = HMatrix(self, h, tree, blocks, params)
        hm.status = st
        return hm

    def matvec(self, hmat, F, transpose=False, out=None, stream=None):
        import torch
        _check_xyz(F, "F")
        U = torch.empty_like(F) if out is None else out
        self._check(lib().hh_matvec(self._h, hmat._h, _dptr(F), _dptr(U), int(transpose), _stream(stream)),
                    "hh_matvec")
        return U

    def matvec_backward(self, hmat, gU, F, gF=None, gX=None, gtheta=None, stream=None):
        p = lambda t: _dptr(t) if t is not None else None
        self._check(lib().hh_matvec_backward(self._h, hmat._h, _dptr(gU), _dptr(F), p(gF), p(gX), p(gtheta),
                                             _stream(stream)), "hh_matvec_backward")


class _Owned:
    _free = None

    def __init__(self, ctx, h):
        self.ctx, self._h = ctx, h

    def close(self):
        if getattr(self, "_h", None):
            getattr(lib(), self._free)(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tree(_Owned):
    _free = "hh_tree_free"

    def export(self):
        nn, n = ctypes.c_int64(), ctypes.c_int64()
        self.ctx._check(lib().hh_export_tree(self._h, None, None, None, None, None, None, None,
                                             ctypes.byref(nn), ctypes.byref(n)), "hh_export_tree")
        nn, n = nn.value, n.value
        perm = np.zeros(n, np.int32); codes = np.zeros(n, np.uint64)
        nb = np.zeros(nn, np.int32); ne = np.zeros(nn, np.int32); ch = np.zeros((nn, 2), np.int32)
        lo = np.zeros((nn, 3)); hi = np.zeros((nn, 3))
        q = lambda a: a.ctypes.data_as(_P)
        self.ctx._check(lib().hh_export_tree(self._h, q(perm), q(codes), q(nb), q(ne), q(ch), q(lo), q(hi),
                                             None, None), "hh_export_tree")
        return dict(perm=perm, codes=codes, begin=nb, end=ne, child=ch, lo=lo, hi=hi)


class Blocks(_Owned):
    _free = "hh_blocks_free"

    def __init__(self, ctx, h, tree):
        super().__init__(ctx, h)
        self.tree = tree    # keep the tree alive

    def export(self):
        nG, nH = ctypes.c_int64(), ctypes.c_int64()
        self.ctx._check(lib().hh_export_blocks(self._h, None, ctypes.byref(nG), None, ctypes.byref(nH)),
                        "hh_export_blocks")
        G = np.zeros((nG.value, 2), np.int32); H = np.zeros((nH.value, 2), np.int32)
        self.ctx._check(lib().hh_export_blocks(self._h, G.ctypes.data_as(_P), None, H.ctypes.data_as(_P), None),
                        "hh_export_blocks")
        return G, H

    def shard_owners(self, n_shards: int):
        """(block_owner [nG], node_owner [n_nodes]): the shard of each admissible
        block and of each target node's near field (see hh_shard_owners)."""
        G, _ = self.export()
        nn = self.tree.export()["begin"].shape[0]
        bo = np.zeros(len(G), np.int32)
        no = np.zeros(nn, np.int32)
        self.ctx._check(lib().hh_shard_owners(self._h, int(n_shards), bo.ctypes.data_as(_P), no.ctypes.data_as(_P)),
                        "hh_shard_owners")
        return bo, no


class HMatrix(_Owned):
    _free = "hh_hmat_free"

    def __init__(self, ctx, h, tree, blocks, params):
        super().__init__(ctx, h)
        self.tree, self.blocks, self.params = tree, blocks, params

    def export(self):
        nG, mr = ctypes.c_int64(), ctypes.c_int32()
        self.ctx._check(lib().hh_export_aca(self._h, None, None, None, ctypes.byref(nG), ctypes.byref(mr)),
                        "hh_export_aca")
        ranks = np.zeros(nG.value, np.int32)
        pI = np.zeros((nG.value, mr.value), np.int32); pJ = np.zeros((nG.value, mr.value), np.int32)
        self.ctx._check(lib().hh_export_aca(self._h, ranks.ctypes.data_as(_P), pI.ctypes.data_as(_P),
                                            pJ.ctypes.data_as(_P), None, None), "hh_export_aca")
        return ranks, pI, pJ

    def export_factors(self):
        """(fofs [nG + 1], factors [n_factor * 9]) as stored: block b holds C
        [l][9][c] then Q [l][9][q] from element fofs[b] on."""
        nG = ctypes.c_int64()
        self.ctx._check(lib().hh_export_aca(self._h, None, None, None, ctypes.byref(nG), None), "hh_export_aca")
        nf, rb = ctypes.c_int64(), ctypes.c_int32()
        self.ctx._check(lib().hh_export_factors(self._h, None, None, ctypes.byref(nf), ctypes.byref(rb)),
                        "hh_export_factors")
        fofs = np.zeros(nG.value + 1, np.int64)
        fac = np.zeros(9 * max(nf.value, 1), np.float64 if rb.value == 8 else np.float32)
        self.ctx._check(lib().hh_export_factors(self._h, fofs.ctypes.data_as(_P), fac.ctypes.data_as(_P), None,
                                                None), "hh_export_factors")
        return fofs, fac[: 9 * nf.value]

    def factor_count(self) -> int:
        """Stored factor elements (9 reals each; hh_export_factors' n_factor)."""
        nf = ctypes.c_int64()
        self.ctx._check(lib().hh_export_factors(self._h, None, None, ctypes.byref(nf), None), "hh_export_factors")
        return nf.value

    def recompress(self, eps_rc: float, stream=None):
        """Truncated-SVD recompression of the stored factors (hh_recompress)."""
        self.ctx._check(lib().hh_recompress(self.ctx._h, self._h, float(eps_rc), _stream(stream)), "hh_recompress")

    def export_recompressed(self):
        """(srank [nG], sofs [nG + 1], sfac): block b holds U [r][3c] then V
        [r][3q] from sofs[b] on (hh_export_recompressed)."""
        nG = ctypes.c_int64()
        self.ctx._check(lib().hh_export_aca(self._h, None, None, None, ctypes.byref(nG), None), "hh_export_aca")
        ns, rb = ctypes.c_int64(), ctypes.c_int32()
        self.ctx._check(lib().hh_export_recompressed(self._h, None, None, None, ctypes.byref(ns), ctypes.byref(rb)),
                        "hh_export_recompressed")
        sr = np.zeros(max(nG.value, 1), np.int32)
        so = np.zeros(nG.value + 1, np.int64)
        sf = np.zeros(max(ns.value, 1), np.float64 if rb.value == 8 else np.float32)
        self.ctx._check(lib().hh_export_recompressed(self._h, sr.ctypes.data_as(_P), so.ctypes.data_as(_P),
                                                     sf.ctypes.data_as(_P), None, None), "hh_export_recompressed")
        return sr[:nG.value], so, sf


def _width_of(n_theta: int) -> int:
    # 4W + W + 2 (W^2 + W) + 6W + 6 parameters (Eq. 4 MLP 4 -> W -> W -> W -> 6)
    for w in (32, 64):
        if 2 * w * w + 13 * w + 6 == n_theta:
            return w
    raise ValueError(f"theta has {n_theta} entries: not a 4-W-W-W-6 MLP with W in (32, 64)")


_HMATVEC = None


def _hmatvec_class():
    global _HMATVEC
    if _HMATVEC is not None:
        return _HMATVEC
    import torch

    class HMatvec(torch.autograd.Function):
        """U = alpha_1 F + M_H(X; theta) F through the C-ABI, with the hand-written
        adjoint hh_matvec_backward as its backward (tree, partition and ACA pivots
        frozen at the forward's X)."""

        @staticmethod
        def forward(ctx, X, F, theta, context, params):
            context.set_mlp(theta.detach(), _width_of(theta.numel()))
            Xd = X.detach().contiguous()
            Fd = F.detach().to(torch.float64).contiguous()
            t = context.build_tree(Xd, params)
            b = context.partition(t, params)
            h = context.aca(t, b, params)
            U = context.matvec(h, Fd)
            ctx.context, ctx.h, ctx.keep = context, h, (t, b)
            ctx.theta_dtype, ctx.n_theta = theta.dtype, theta.numel()
            ctx.save_for_backward(Fd)
            return U

        @staticmethod
        def backward(ctx, gU):
            (Fd,) = ctx.saved_tensors
            gU = gU.detach().to(torch.float64).contiguous()
            need_x, need_f, need_t = ctx.needs_input_grad[:3]
            gF = torch.empty_like(Fd) if need_f else None
            gX = torch.zeros_like(Fd) if need_x else None
            gT = torch.zeros(ctx.n_theta, dtype=torch.float32, device=Fd.device) if need_t else None
            if need_x or need_f or need_t:
                ctx.context.matvec_backward(ctx.h, gU, Fd, gF=gF, gX=gX, gtheta=gT)
            return gX, gF, (gT.to(ctx.theta_dtype) if gT is not None else None), None, None

    _HMATVEC = HMatvec
    return HMatvec


def hmatvec(X, F, theta, context: "Context", params: CParams):
    """Differentiable U = alpha_1 F + M_H(X; theta) F (torch.autograd): gradients
    with respect to X, F and theta come from hh_matvec_backward."""
    return _hmatvec_class().apply(X, F, theta, context, params)
