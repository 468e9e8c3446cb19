"""Seeded synthetic inputs for the two-site QC-DMRG hot path.

This module only draws random numbers and arranges them into arrays: it holds
none of the method's arithmetic.  Both the CUDA path (through the C ABI) and
the CPU oracle consume what it produces, so the two sides always see the same
inputs.

Integrals (the stand-in for the paper's molecular active spaces, which are not
available here): restricted-orbital one- and two-electron integrals of the
electronic Hamiltonian of Sec. 2.1, Eq. H2q, with
    h_ii = -2 + 4 i / L                       (0-based i, no noise)
    h_ij ~ N(0, 0.1^2) * exp(-|i-j|/4)        (i < j, row-major, mirrored)
    B^P_ij ~ N(0, 0.15^2)                     (P = 0..2L-1, i <= j row-major, mirrored)
    v_ijkl = sum_P B^P_ij B^P_kl              (chemists' (ij|kl), 8-fold symmetric)
drawn in that order from numpy.random.default_rng(seed) (PCG64).
"""
from __future__ import annotations

import numpy as np


def integrals(L: int, seed: int = 0, rng: np.random.Generator | None = None):
    """Return (h, v) as float64 arrays of shape (L, L) and (L, L, L, L)."""
    if rng is None:
        rng = np.random.default_rng(seed)
    h = np.zeros((L, L))
    for i in range(L):
        h[i, i] = -2.0 + 4.0 * i / L
    iu, ju = np.triu_indices(L, k=1)
    off = rng.normal(0.0, 0.1, size=iu.size) * np.exp(-np.abs(iu - ju) / 4.0)
    h[iu, ju] = off
    h[ju, iu] = off
    iu2, ju2 = np.triu_indices(L, k=0)
    B = np.zeros((2 * L, L, L))
    for P in range(2 * L):
        b = rng.normal(0.0, 0.15, size=iu2.size)
        B[P, iu2, ju2] = b
        B[P, ju2, iu2] = b
    v = np.einsum("pij,pkl->ijkl", B, B)
    return h, np.ascontiguousarray(v)


def batched_instance(seed: int):
    """One instance of the batched workload: (L, M, h, v) for a given seed.

    L is uniform in {10..20}, M uniform in {64..256}, then the integrals, all
    drawn from the same generator.
    """
    rng = np.random.default_rng(seed)
    L = int(rng.integers(10, 21))
    M = int(rng.integers(64, 257))
    h, v = integrals(L, rng=rng)
    return L, M, h, v


def hubbard_dimer(t: float, U: float):
    """Two-orbital Hubbard dimer: h = [[0,-t],[-t,0]], (11|11) = (22|22) = U."""
    h = np.array([[0.0, -t], [-t, 0.0]])
    v = np.zeros((2, 2, 2, 2))
    v[0, 0, 0, 0] = U
    v[1, 1, 1, 1] = U
    return h, v


def gaussian(shape, seed: int):
    """Standard-normal float64 array of the given shape (seeded)."""
    return np.random.default_rng(seed).standard_normal(shape)


def orthonormal_columns(rows: int, cols: int, rng: np.random.Generator):
    """rows x cols matrix with orthonormal columns: Q factor of a Gaussian matrix.

    Used to draw random block bases (renormalization matrices) for tests and
    for growing the middle-bond blocks of the large workloads; cols <= rows.
    """
    if cols == 0:
        return np.zeros((rows, 0))
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    # fix the sign gauge so the draw is reproducible across LAPACK builds
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def sector_dims_profile(k: int, n_up_tot: int, n_dn_tot: int, L: int, M: int,
                        caps: dict):
    """Deterministic sector-dimension profile of a k-orbital block with bond dimension M.

    m(nu, nd) is proportional to exp(-[(nu - k Nu/L)^2 + (nd - k Nd/L)^2] / (2 s^2)),
    s = sqrt(k)/2, capped by caps[(nu, nd)] (the number of states the enlarged
    block offers in that sector), then normalised to sum M by largest remainder.
    Returns a dict {(nu, nd): m} over the keys of caps (zeros dropped).
    """
    keys = sorted(caps)
    s = max(np.sqrt(k) / 2.0, 0.5)
    cu, cd = k * n_up_tot / L, k * n_dn_tot / L
    w = np.array([np.exp(-((nu - cu) ** 2 + (nd - cd) ** 2) / (2 * s * s)) for nu, nd in keys])
    cap = np.array([caps[key] for key in keys], dtype=np.int64)
    total = min(M, int(cap.sum()))
    alloc = np.zeros(len(keys), dtype=np.int64)
    remaining = total
    active = cap > 0
    # water-filling with caps, then largest remainder
    while remaining > 0 and active.any():
        ww = np.where(active, w, 0.0)
        if ww.sum() <= 0:
            ww = active.astype(float)
        share = ww / ww.sum() * remaining
        base = np.minimum(np.floor(share).astype(np.int64), cap - alloc)
        if base.sum() == 0:
            frac = np.where(active, share - np.floor(share), -1.0)
            order = np.lexsort((np.arange(len(keys)), -frac))
            for idx in order:
                if remaining == 0:
                    break
                if active[idx] and alloc[idx] < cap[idx]:
                    alloc[idx] += 1
                    remaining -= 1
        else:
            alloc += base
            remaining -= int(base.sum())
        active = alloc < cap
    return {key: int(m) for key, m in zip(keys, alloc) if m > 0}


def middle_bond_sectors(L: int, n_up: int, n_dn: int, M: int, k: int, M_right: int | None = None):
    """Sector tables {(nu, nd): dim} of the two middle-bond blocks grow_middle_bond builds.

    Dimensions only (no operators): each enlarged block offers, per sector, the
    sum of the old block's sector dimensions over the four site states, and the
    kept dimensions follow sector_dims_profile.  Returns (left, right): the
    left block of sites 0..k-1 and the right block of sites k+2..L-1.
    """
    if M_right is None:
        M_right = M
    site = ((0, 0), (1, 0), (0, 1), (1, 1))

    def grow(blk, n_sites, m):
        caps = {}
        for (a, b), d in blk.items():
            for su, sd in site:
                caps[(a + su, b + sd)] = caps.get((a + su, b + sd), 0) + d
        return sector_dims_profile(n_sites, n_up, n_dn, L, m, caps)

    left, right = {(0, 0): 1}, {(0, 0): 1}
    for s in range(k):
        left = grow(left, s + 1, M)
    for s in range(L - 1, k + 1, -1):
        right = grow(right, L - s, M_right)
    return left, right


def grow_middle_bond(ctx, L: int, n_up: int, n_dn: int, M: int, k: int, seed: int = 0,
                     release: bool = False, M_right: int | None = None):
    """Grow the left blocks 0..k-1 and right blocks k+2..L-1 of a context with seeded random O.

    Each renormalization keeps, per enlarged sector, the number of states given
    by sector_dims_profile (normalised to M) and draws a random orthonormal O.
    Returns the list of (direction, kept, O_flat) applied, in order, so the same
    bases can be replayed elsewhere.  Leaves ctx at position k.  With release,
    each block is freed once the next one is built (ctx.release_block), so only
    the middle-bond blocks stay resident.  M_right (default M) is the bond
    dimension of the right blocks (asymmetric M).
    """
    if M_right is None:
        M_right = M
    rng = np.random.default_rng(seed)
    applied = []
    ctx.set_position(0, 1)
    for s in range(k):
        lay = ctx.enlarged_layout(+1)
        caps = {(int(a), int(b)): int(d) for a, b, d in lay}
        prof = sector_dims_profile(s + 1, n_up, n_dn, L, M, caps)
        kept = [prof.get((int(a), int(b)), 0) for a, b, _ in lay]
        O = np.concatenate([orthonormal_columns(int(d), m, rng).ravel() for (_, _, d), m in zip(lay, kept)])
        ctx.renormalize(+1, O, kept)
        applied.append((+1, kept, O))
        if release and s >= 1:
            ctx.release_block(0, s)
    ctx.set_position(L - 2, -1)
    for s in range(L - 1, k + 1, -1):
        n_sites = L - s
        lay = ctx.enlarged_layout(-1)
        caps = {(int(a), int(b)): int(d) for a, b, d in lay}
        prof = sector_dims_profile(n_sites, n_up, n_dn, L, M_right, caps)
        kept = [prof.get((int(a), int(b)), 0) for a, b, _ in lay]
        O = np.concatenate([orthonormal_columns(int(d), m, rng).ravel() for (_, _, d), m in zip(lay, kept)])
        ctx.renormalize(-1, O, kept)
        applied.append((-1, kept, O))
        if release and n_sites >= 2:
            ctx.release_block(1, n_sites - 1)
    ctx.set_position(k, 1)
    return applied
