"""Seeded synthetic inputs for the H-matrix mobility product.

This module produces the data that both sides of every comparison consume:
particle positions, forces, and the pair-MLP parameter vector.  It holds none
of the method's arithmetic (no pair kernel, no tree, no admissibility, no
low-rank approximation); it only places particles, draws forces and draws
network weights.  Both the CUDA path and the CPU oracle read its outputs.

Workload recipes (the paper's suspensions of Section 4, replaced by seeded
synthetic equivalents):

* ``rsa_cube``       -- random sequential addition of spheres of radius ``a``
                        in a cube at volume fraction ``phi`` (centre distance
                        >= 2a); stands in for the paper's perturbed lattices.
* ``gaussian_cloud`` -- spherical Gaussian "suspension drop" with overlap
                        rejection; sigma is raised to the smallest value whose
                        peak volume fraction is <= 0.25.
* ``filaments``      -- straight bead chains at random orientation, placed
                        without overlap; ``perturb`` gives a displaced variant
                        (the bead forces belong to the time step, not here).
* ``forces``         -- i.i.d. N(0,1) force components.
* ``mlp_params``     -- Xavier-uniform weights drawn from SplitMix64, zero
                        biases, every value rounded to bfloat16 so that the
                        FP64, FP32 and BF16 paths evaluate the same network.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "cube_side", "rsa_cube", "sigma_min", "gaussian_cloud", "filaments",
    "perturb",
    "forces", "splitmix64", "uniform01", "mlp_params", "mlp_param_count",
    "round_bf16", "GEOMETRY_SEED",
]

GEOMETRY_SEED = 1234

# SplitMix64 (Steele, Lea & Flood 2014): state_k = seed + k * golden, then the
# three-round mixer.  Counter based, so any draw can be recomputed from k.
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs ``start+1 .. start+n`` of SplitMix64 seeded with ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """53-bit doubles in [0, 1) from SplitMix64 (top 53 bits times 2^-53)."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def round_bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) through float32; float32 out."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32)


def mlp_param_count(width: int, depth: int = 3, n_in: int = 4, n_out: int = 6) -> int:
    dims = [n_in] + [width] * depth + [n_out]
    return sum(dims[i + 1] * dims[i] + dims[i + 1] for i in range(len(dims) - 1))


def mlp_params(width: int, seed: int, depth: int = 3, n_in: int = 4, n_out: int = 6,
               bf16: bool = True) -> np.ndarray:
    """Packed pair-MLP parameters (float32).

    Per layer (input -> hidden x depth -> output): weight [out, in] row-major,
    then bias [out].  Weights Xavier uniform U(-b, b), b = sqrt(6/(fan_in +
    fan_out)), drawn in layer order from one SplitMix64 stream; zero biases.
    With ``bf16`` every value is rounded to bfloat16.
    """
    dims = [n_in] + [width] * depth + [n_out]
    out = []
    pos = 0
    for li in range(len(dims) - 1):
        fi, fo = dims[li], dims[li + 1]
        bound = math.sqrt(6.0 / (fi + fo))
        u = uniform01(seed, fo * fi, pos)
        pos += fo * fi
        out.append((2.0 * u - 1.0) * bound)
        out.append(np.zeros(fo))
    theta = np.concatenate(out)
    return round_bf16(theta) if bf16 else theta.astype(np.float32)


def cube_side(n: int, phi: float, a: float = 1.0) -> float:
    return (n * (4.0 / 3.0) * math.pi * a ** 3 / phi) ** (1.0 / 3.0)


def _rsa(n: int, propose, a: float, rng) -> np.ndarray:
    """Random sequential addition in batches: a candidate is kept when no kept
    centre, and no other candidate of its batch with a lower index, lies
    closer than 2a."""
    from scipy.spatial import cKDTree

    pts = np.empty((0, 3))
    d2 = 2.0 * a
    stall = 0
    while len(pts) < n:
        need = n - len(pts)
        cand = propose(rng, int(need * 1.25) + 64)
        if len(pts):
            dist, _ = cKDTree(pts).query(cand, k=1, distance_upper_bound=d2)
            cand = cand[~(dist < d2)]
        if len(cand) > 1:
            pairs = cKDTree(cand).query_pairs(d2, output_type="ndarray")
            if len(pairs):
                bad = np.zeros(len(cand), dtype=bool)
                bad[np.maximum(pairs[:, 0], pairs[:, 1])] = True
                cand = cand[~bad]
        cand = cand[:need]
        stall = stall + 1 if len(cand) == 0 else 0
        if stall > 50:
            raise RuntimeError("random sequential addition stalled")
        pts = np.concatenate([pts, cand]) if len(pts) else cand
    return np.ascontiguousarray(pts[:n])


def rsa_cube(n: int, phi: float = 0.1, a: float = 1.0, seed: int = GEOMETRY_SEED) -> np.ndarray:
    """n sphere centres, uniform in [0, L]^3 with L set by the volume fraction."""
    side = cube_side(n, phi, a)
    rng = np.random.Generator(np.random.PCG64(seed))
    return _rsa(n, lambda g, m: g.uniform(0.0, side, size=(m, 3)), a, rng)


def sigma_min(n: int, a: float = 1.0, peak_phi: float = 0.25) -> float:
    """Smallest Gaussian width whose peak volume fraction is <= peak_phi."""
    return (n * (4.0 / 3.0) * math.pi * a ** 3 / (peak_phi * (2.0 * math.pi) ** 1.5)) ** (1.0 / 3.0)


def gaussian_cloud(n: int, sigma: float, a: float = 1.0, seed: int = GEOMETRY_SEED):
    """Spherical Gaussian cloud; returns (X, sigma_eff)."""
    s = max(sigma, sigma_min(n, a))
    rng = np.random.Generator(np.random.PCG64(seed))
    return _rsa(n, lambda g, m: g.normal(0.0, s, size=(m, 3)), a, rng), s


def filaments(n_chains: int, beads: int, bond: float = 2.2, a: float = 1.0, phi: float = 0.1,
              min_gap: float = 2.1, seed: int = GEOMETRY_SEED):
    """Straight chains of ``beads`` beads spaced ``bond`` apart, uniformly random
    orientation, placed one at a time in a cube (random sequential addition of
    whole chains) so that beads of different chains stay >= min_gap apart.
    The cube starts at the side of volume fraction ``phi``.  A chain's start
    point is uniform over the positions where the whole chain fits in the cube.
    After 1000 consecutive failed placements the cube grows by 5% in place:
    the start points of the chains already placed are scaled by 1.05 (a rigid
    chain then still fits), any bead pair that this brings closer than min_gap
    (rare) removes the later chain, and placement continues.  Random straight
    rods this long jam far below phi = 0.1, so the cube grows several times.

    Candidates are drawn in batches of 256 and tested against the placed beads
    together, then accepted in draw order, each also tested against those of
    its batch accepted before it; the failure count runs in draw order.

    Beads of chain c are rows c*beads .. c*beads+beads-1, in order along the
    chain.  Returns (X, chain_id, side); the volume fraction reached is
    n_chains * beads * (4/3) pi a^3 / side^3.

    Overlap test: a cell grid of side >= min_gap with an empty border layer,
    so every bead closer than min_gap to a candidate bead sits in one of the
    27 cells around it; each cell keeps a linked list of its beads."""
    from scipy.spatial import cKDTree

    rng = np.random.Generator(np.random.PCG64(seed))
    side = cube_side(n_chains * beads, phi, a)
    offs = np.arange(beads) * bond
    g2 = min_gap * min_gap
    nbead = n_chains * beads
    starts = np.empty((n_chains, 3))
    dirs = np.empty((n_chains, 3))
    placed = 0

    def beads_of(st, dv):
        return (st[:, None, :] + offs[None, :, None] * dv[:, None, :]).reshape(-1, 3)

    while True:
        nc = max(1, int(side // min_gap))
        h = side / nc
        P = nc + 2
        stencil = ((np.arange(-1, 2)[:, None, None] * P + np.arange(-1, 2)[None, :, None]) * P
                   + np.arange(-1, 2)[None, None, :]).ravel()

        def cell_of(x):
            c = np.clip((x // h).astype(np.int64), 0, nc - 1) + 1
            return (c[..., 0] * P + c[..., 1]) * P + c[..., 2]

        head = np.full(P * P * P, -1, dtype=np.int64)
        nxt = np.full(nbead, -1, dtype=np.int64)
        X = np.empty((nbead, 3))
        if placed:
            X[:placed * beads] = beads_of(starts[:placed], dirs[:placed])
            f = cell_of(X[:placed * beads])
            order = np.argsort(f, kind="stable")
            fs = f[order]
            last = np.r_[fs[1:] != fs[:-1], True]
            nxt[order[:-1]] = np.where(last[:-1], -1, order[1:])
            first = np.r_[True, fs[1:] != fs[:-1]]
            head[fs[first]] = order[first]
        fails = 0
        while placed < n_chains and fails < 1000:
            m = 256
            V = rng.normal(size=(m, 3))
            V /= np.linalg.norm(V, axis=1)[:, None]
            U = rng.uniform(0.0, 1.0, size=(m, 3))
            E = offs[-1] * V
            lo = np.maximum(0.0, -E)
            hi = side - np.maximum(0.0, E)
            fits = (hi >= lo).all(1)
            ST = lo + U * (hi - lo)
            C = ST[:, None, :] + offs[None, :, None] * V[:, None, :]
            fc = cell_of(C)                                         # [m, beads]
            idx = head[fc[:, :, None] + stencil[None, None, :]]     # [m, beads, 27]
            jm, jb, _ = np.nonzero(idx >= 0)
            idx = idx[idx >= 0]
            clash = np.zeros(m, dtype=bool)
            while len(idx):
                d = X[idx] - C[jm, jb]
                clash[jm[np.einsum("ij,ij->i", d, d) < g2]] = True
                idx = nxt[idx]
                keep = idx >= 0
                idx, jm, jb = idx[keep], jm[keep], jb[keep]
            ok = fits & ~clash
            acc = []
            for j in range(m):
                if ok[j] and acc:
                    Q = C[acc].reshape(-1, 3)
                    d = Q[:, None, :] - C[j][None, :, :]
                    ok[j] = not (np.einsum("ijk,ijk->ij", d, d) < g2).any()
                if not ok[j]:
                    fails += 1
                    if fails >= 1000:
                        break
                    continue
                acc.append(j)
                base = placed * beads
                X[base:base + beads] = C[j]
                for k in range(beads):
                    nxt[base + k] = head[fc[j, k]]
                    head[fc[j, k]] = base + k
                starts[placed], dirs[placed] = ST[j], V[j]
                placed += 1
                fails = 0
                if placed == n_chains:
                    break
        if placed == n_chains:
            return X, np.repeat(np.arange(n_chains), beads), side
        # grow in place; drop the later chain of any pair brought too close
        side *= 1.05
        starts[:placed] *= 1.05
        B = beads_of(starts[:placed], dirs[:placed])
        pr = cKDTree(B).query_pairs(min_gap, output_type="ndarray")
        if len(pr):
            pr = pr[pr[:, 0] // beads != pr[:, 1] // beads]
            if len(pr):
                d = B[pr[:, 0]] - B[pr[:, 1]]
                close = np.einsum("ij,ij->i", d, d) < g2
                drop = np.unique(np.maximum(pr[close, 0], pr[close, 1]) // beads)
                keep = np.setdiff1d(np.arange(placed), drop)
                starts[:len(keep)], dirs[:len(keep)] = starts[keep], dirs[keep]
                placed = len(keep)


def perturb(X: np.ndarray, scale: float, seed: int) -> np.ndarray:
    """X plus i.i.d. N(0, scale^2) displacements (a bent, stretched variant
    of a chain configuration that exercises the bond and bending forces)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return X + scale * rng.standard_normal(X.shape)


def two_particle_samples(batch: int, seed: int, dmin: float = 2.0, dmax: float = 1000.0):
    """Training configurations of two particles (Section 2.3): separation
    r = x_1 - x_2 with |r| log-uniform in [dmin, dmax] and uniform direction,
    and a unit force on particle 2 drawn from {e_x, e_y, e_z}.  Returns
    (r [B,3], e [B,3]) float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.standard_normal((batch, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    d = np.exp(rng.uniform(np.log(dmin), np.log(dmax), size=batch))
    e = np.eye(3)[rng.integers(0, 3, size=batch)]
    return u * d[:, None], e


def forces(n: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) force components, shape [n, 3], float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, 3))
