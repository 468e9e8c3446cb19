"""Shared test helpers: grow identical random block bases on the GPU library and in the oracle.

The random renormalization matrices are inputs (seeded, from workloads); both
sides receive the same O, and the enlarged-sector layouts they each compute
independently are checked to agree before use.
"""
from __future__ import annotations

import numpy as np

from oracle import blocks as ob
from paper_2001_04890_gb300 import workloads


def choose_kept(dims, M):
    tot = int(sum(dims))
    if tot <= M:
        return [int(d) for d in dims]
    kept = [min(int(d), max(1, int(d * M / tot))) if d > 0 else 0 for d in dims]
    while sum(kept) > M:
        i = int(np.argmax(kept))
        kept[i] -= 1
    return kept


def random_O(layout_dims, M, rng):
    kept = choose_kept(layout_dims, M)
    blocks = [workloads.orthonormal_columns(int(n), int(m), rng) for n, m in zip(layout_dims, kept)]
    flat = np.concatenate([b.ravel() for b in blocks]) if blocks else np.zeros(0)
    return kept, blocks, flat


def _check_layout(gpu_layout, oracle_layout):
    dims = ob.enlarged_dims(oracle_layout)
    ref = np.array([(E[0], E[1], dims[E]) for E in oracle_layout], dtype=np.int64).reshape(-1, 3)
    assert np.array_equal(np.asarray(gpu_layout, dtype=np.int64).reshape(-1, 3), ref), (gpu_layout, ref)


def build_random_position(ctx, h, v, k, M, seed=0, left_M=None, right_M=None):
    """Grow left blocks 0..k-1 and right blocks k+2..L-1 with the same random O on both sides.

    Leaves ctx at position k and returns the oracle blocks (lb, rb).
    """
    L = h.shape[0]
    rng = np.random.default_rng(seed)
    left_M = left_M or M
    right_M = right_M or M
    lb = ob.empty_block()
    ctx.set_position(0, 1)
    for s in range(k):
        lay = ob.enlarged_left(lb)
        _check_layout(ctx.enlarged_layout(+1), lay)
        dims = [ob.enlarged_dims(lay)[E] for E in lay]
        kept, blocks, flat = random_O(dims, left_M, rng)
        ctx.renormalize(+1, flat, kept)
        lb = ob.grow_left(lb, s, {E: b for E, b in zip(lay, blocks)})
    rb = ob.empty_block()
    ctx.set_position(L - 2, -1)
    for s in range(L - 1, k + 1, -1):
        lay = ob.enlarged_right(rb)
        _check_layout(ctx.enlarged_layout(-1), lay)
        dims = [ob.enlarged_dims(lay)[E] for E in lay]
        kept, blocks, flat = random_O(dims, right_M, rng)
        ctx.renormalize(-1, flat, kept)
        rb = ob.grow_right(rb, s, {E: b for E, b in zip(lay, blocks)})
    ctx.set_position(k, 1)
    return lb, rb


def rebuild_blocks(exports, L, side, n_sites):
    """Explicit-basis block (oracle/blocks.py) of n_sites sites rebuilt from exported
    renormalization matrices: exports[j] = (kept per enlarged sector, flat O) of the
    block of j sites, in the format dmrg_renormalize takes (dmrg_block_basis)."""
    blk = ob.empty_block()
    for j in range(1, n_sites + 1):
        kept, O = exports[j]
        lay = ob.enlarged_left(blk) if side == 0 else ob.enlarged_right(blk)
        dims = [ob.enlarged_dims(lay)[E] for E in lay]
        assert len(kept) == len(lay)
        blocks, pos = {}, 0
        for E, d, m in zip(lay, dims, kept):
            blocks[E] = np.asarray(O[pos:pos + d * m]).reshape(d, m)
            pos += d * m
        assert pos == len(O)
        blk = ob.grow_left(blk, j - 1, blocks) if side == 0 else ob.grow_right(blk, L - j, blocks)
    return blk


def oracle_middle_bond(h, v, n_up, n_dn, M, k, seed):
    """The operator-based FP64 oracle at position k, its blocks grown from the same
    seeded random O as workloads.grow_middle_bond gives a GPU context."""
    from oracle import baseline
    from oracle import dmrg as od
    L = h.shape[0]
    b = baseline.OracleBuilder(h, v)
    workloads.grow_middle_bond(b, L, n_up, n_dn, M, k, seed=seed)
    lb, rb = b._blocks()
    return od.HPsi(b.I, k, lb, rb, n_up, n_dn)
