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
* ``lattice_sphere`` -- the sites of a primitive cubic lattice (one at the
                        centre) inside a ball, each moved by a small uniform
                        jitter: the paper's suspension drop; ``two_drops``
                        stacks two of them on the z axis.
* ``lattice_cube`` / ``lattice_subset`` -- a perturbed n^3 lattice and seeded
                        random subsets of its sites (fixed domain, varying
                        concentration).
* ``filament_sphere`` -- the paper's filament suspension: bead chains placed
                        in an inner ball, free particles in the shell around
                        it, centre distances >= a minimum gap.
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
    "perturb", "lattice_sphere", "two_drops", "lattice_cube", "lattice_subset", "filament_sphere",
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


def lattice_sphere(radius: float, spacing: float = 3.5, center=(0.0, 0.0, 0.0), jitter: float = 0.2,
                   seed: int = GEOMETRY_SEED) -> np.ndarray:
    """Sites of a primitive cubic lattice of the given spacing, one of them at
    the centre, with |site - centre| <= radius (selected before the jitter),
    each then moved by an i.i.d. uniform [-jitter, jitter] offset per
    component.  Rows in lattice order (x-major).  With jitter <=
    (spacing - 2a) / (2 sqrt 3) no two spheres of radius a overlap.  The
    paper's drop (radius 175, about 10% volume fraction) is spacing 3.5:
    the 523,305 lattice points of a ball of radius 50 lattice units."""
    m = int(radius // spacing) + 1
    g = np.arange(-m, m + 1, dtype=np.float64) * spacing
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    P = P[np.einsum("ij,ij->i", P, P) <= radius * radius]
    rng = np.random.Generator(np.random.PCG64(seed))
    P = P + rng.uniform(-jitter, jitter, size=P.shape)
    return np.ascontiguousarray(P + np.asarray(center, dtype=np.float64))


def two_drops(radius: float = 175.0, spacing: float = 3.5, separation: float = 3.0, jitter: float = 0.2,
              seed: int = GEOMETRY_SEED) -> np.ndarray:
    """Two equal lattice drops on the z axis, vertically aligned, centres
    separation * radius apart (the upper, trailing drop first in the rows);
    each from lattice_sphere with its own seed."""
    up = lattice_sphere(radius, spacing, (0.0, 0.0, separation * radius), jitter, seed)
    down = lattice_sphere(radius, spacing, (0.0, 0.0, 0.0), jitter, seed + 1)
    return np.ascontiguousarray(np.concatenate([up, down]))


def lattice_cube(n_side: int, spacing: float = 3.5, jitter: float = 0.2, seed: int = GEOMETRY_SEED) -> np.ndarray:
    """n_side^3 sites of a primitive cubic lattice, origin at a corner, each
    moved by a uniform [-jitter, jitter] offset per component."""
    g = np.arange(n_side, dtype=np.float64) * spacing
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(P + rng.uniform(-jitter, jitter, size=P.shape))


def lattice_subset(n: int, n_side: int = 100, spacing: float = 3.5, jitter: float = 0.2, seed: int = GEOMETRY_SEED,
                   subset_seed: int = 0) -> np.ndarray:
    """n distinct sites drawn uniformly (seeded) from the perturbed
    n_side^3 lattice of lattice_cube, in lattice order: the domain stays
    fixed while the concentration grows with n."""
    P = lattice_cube(n_side, spacing, jitter, seed)
    rng = np.random.Generator(np.random.PCG64(subset_seed))
    idx = np.sort(rng.choice(len(P), size=n, replace=False))
    return np.ascontiguousarray(P[idx])


def filament_sphere(n_fil: int = 5120, beads: int = 21, rb: float = 3.0, n_free: int = 107520,
                    min_gap: float = 2.1, seed: int = GEOMETRY_SEED):
    """The paper's filament suspension: straight chains of `beads` beads
    spaced rb apart, random orientation, placed whole and one batch at a time
    inside the inner ball R_in = (1/2)^(1/3) R_out, R_out = 4 * 10^(1/3) *
    (beads - 1) * rb (a chain's midpoint uniform in the ball of radius
    R_in - (beads - 1) rb / 2, so every bead is inside R_in); then n_free
    particles uniform in the shell R_in <= |x| <= R_out.  Every centre
    distance between different chains, or involving a free particle, is
    >= min_gap (candidates are checked against everything placed before
    and against the earlier candidates of their batch).  Rows: chain c at
    c*beads .. c*beads + beads - 1 in order along the chain, then the free
    particles.  Returns (X, R_in, R_out)."""
    from scipy.spatial import cKDTree

    rng = np.random.Generator(np.random.PCG64(seed))
    r_out = 4.0 * 10.0 ** (1.0 / 3.0) * (beads - 1) * rb
    r_in = 0.5 ** (1.0 / 3.0) * r_out
    half = 0.5 * (beads - 1) * rb
    offs = (np.arange(beads) - 0.5 * (beads - 1)) * rb

    def in_ball(m, rad):
        v = rng.normal(size=(m, 3))
        v /= np.linalg.norm(v, axis=1)[:, None]
        return v * (rad * rng.uniform(0.0, 1.0, size=m) ** (1.0 / 3.0))[:, None]

    chains = np.empty((0, beads, 3))
    stall = 0
    while len(chains) < n_fil:
        m = 256
        mid = in_ball(m, r_in - half)
        d = rng.normal(size=(m, 3))
        d /= np.linalg.norm(d, axis=1)[:, None]
        C = mid[:, None, :] + offs[None, :, None] * d[:, None, :]
        ok = np.ones(m, dtype=bool)
        if len(chains):
            dist, _ = cKDTree(chains.reshape(-1, 3)).query(C.reshape(-1, 3), k=1, distance_upper_bound=min_gap)
            ok &= ~(dist.reshape(m, beads) < min_gap).any(1)
        keep = []
        for j in range(m):
            if not ok[j]:
                continue
            if keep:
                Q = C[keep].reshape(-1, 3)
                dd = Q[:, None, :] - C[j][None, :, :]
                if (np.einsum("ijk,ijk->ij", dd, dd) < min_gap * min_gap).any():
                    continue
            keep.append(j)
            if len(chains) + len(keep) == n_fil:
                break
        stall = stall + 1 if not keep else 0
        if stall > 50:
            raise RuntimeError("filament placement stalled")
        chains = np.concatenate([chains, C[keep]])
    beadsX = chains.reshape(-1, 3)
    tree_b = cKDTree(beadsX)
    free = np.empty((0, 3))
    stall = 0
    while len(free) < n_free:
        need = n_free - len(free)
        m = int(need * 1.25) + 64
        v = rng.normal(size=(m, 3))
        v /= np.linalg.norm(v, axis=1)[:, None]
        rad = (r_in ** 3 + rng.uniform(0.0, 1.0, size=m) * (r_out ** 3 - r_in ** 3)) ** (1.0 / 3.0)
        cand = v * rad[:, None]
        dist, _ = tree_b.query(cand, k=1, distance_upper_bound=min_gap)
        cand = cand[~(dist < min_gap)]
        if len(free) and len(cand):
            dist, _ = cKDTree(free).query(cand, k=1, distance_upper_bound=min_gap)
            cand = cand[~(dist < min_gap)]
        if len(cand) > 1:
            pairs = cKDTree(cand).query_pairs(min_gap, output_type="ndarray")
            if len(pairs):
                bad = np.zeros(len(cand), dtype=bool)
                bad[np.maximum(pairs[:, 0], pairs[:, 1])] = True
                cand = cand[~bad]
        cand = cand[:need]
        stall = stall + 1 if len(cand) == 0 else 0
        if stall > 50:
            raise RuntimeError("free-particle placement stalled")
        free = np.concatenate([free, cand]) if len(free) else cand
    return np.ascontiguousarray(np.concatenate([beadsX, free[:n_free]])), r_in, r_out


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
