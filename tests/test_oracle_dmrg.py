"""The operator-based oracle DMRG (oracle/dmrg.py) pinned to the explicit-basis oracle and to full CI."""
import numpy as np
import pytest

from oracle import blocks as ob
from oracle import dmrg as od
from oracle import fock
from paper_2001_04890_gb300 import workloads
from tests.helpers import random_O


def grow_both(h, v, k, M, seed):
    """Same random O on the explicit-basis oracle (O2) and the operator oracle (O3)."""
    I = od.Ints(h, v)
    L = h.shape[0]
    rng = np.random.default_rng(seed)
    lb, lo = ob.empty_block(), od.empty_oblock(0)
    for s in range(k):
        lay = ob.enlarged_left(lb)
        dims = [ob.enlarged_dims(lay)[E] for E in lay]
        kept, blocks, _ = random_O(dims, M, rng)
        lo = od.renormalize(I, s, lo, od.empty_oblock(1), +1, blocks, kept)
        lb = ob.grow_left(lb, s, {E: b for E, b in zip(lay, blocks)})
    rb, ro = ob.empty_block(), od.empty_oblock(1)
    for s in range(L - 1, k + 1, -1):
        lay = ob.enlarged_right(rb)
        dims = [ob.enlarged_dims(lay)[E] for E in lay]
        kept, blocks, _ = random_O(dims, M, rng)
        ro = od.renormalize(I, s - 1, od.empty_oblock(0), ro, -1, blocks, kept)
        rb = ob.grow_right(rb, s, {E: b for E, b in zip(lay, blocks)})
    return I, lb, rb, lo, ro


# L = 8: blocks of up to five sites on either side, so both halves hold several
# orbitals when the complementary operators are formed on the larger one (k = 1:
# the right block is larger, k = 5: the left one, k = 3: equal halves)
@pytest.mark.parametrize("L,N,two_sz,M,k", [(5, 4, 0, 16, 1), (6, 6, 0, 40, 2), (6, 5, 1, 24, 3),
                                            (6, 6, 0, 30, 0), (6, 6, 0, 30, 4), (8, 8, 0, 40, 1),
                                            (8, 8, 0, 40, 3), (8, 8, 0, 40, 5)])
def test_operator_oracle_hpsi_equals_explicit_projection(L, N, two_sz, M, k):
    h, v = workloads.integrals(L, seed=200 + k)
    nu, nd = (N + two_sz) // 2, (N - two_sz) // 2
    I, lb, rb, lo, ro = grow_both(h, v, k, M, seed=k)
    P = ob.Projected(h, v, lb, rb, nu, nd)
    hp = od.HPsi(I, k, lo, ro, nu, nd)
    assert hp.dim == P.dim
    psi = workloads.gaussian(P.dim, seed=3)
    ref = P.apply(psi)
    assert np.max(np.abs(hp.apply(psi) - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_operator_oracle_block_ops_equal_exact():
    L, M, k = 6, 30, 3
    h, v = workloads.integrals(L, seed=17)
    I, lb, rb, lo, ro = grow_both(h, v, k, M, seed=5)
    for blk, oblk, keys in ((lb, lo, [("H",), ("C", 3), ("T", 9), ("A", 0, 5), ("B", 4, 1)]),
                            (rb, ro, [("H",), ("C", 11), ("V", 2), ("A", 10, 11), ("B", 11, 10)])):
        for key in keys:
            idx = None if len(key) == 1 else tuple(key[1:])
            ex = ob.renormalized(blk, ob.block_fock_operator(blk, key[0], idx, h, v))
            got = oblk.op(key)
            for (kb, ka), M_ in ex.items():
                g = got.get((blk.sectors.index(kb), blk.sectors.index(ka)))
                assert g is not None and np.max(np.abs(g - M_)) < 1e-12, key
            for (b, a), g in got.items():
                assert (blk.sectors[b], blk.sectors[a]) in ex or np.max(np.abs(g)) < 1e-12


def test_operator_oracle_sweeps_reach_fci():
    L, N, M = 6, 6, 64
    h, v = workloads.integrals(L, seed=12)
    e_fci = fock.fci_ground(h, v, 3, 3)[0]
    dm = od.OracleDMRG(h, v, N, 0, M)
    E = dm.sweep(4)
    assert np.all(E >= e_fci - 1e-10)
    assert abs(E[2 * 2 * (L - 2):].min() - e_fci) < 1e-10


def test_baseline_builder_replays_on_explicit_bases():
    """The CPU baseline's middle-bond builder (oracle/baseline.py, driven by
    workloads.grow_middle_bond) against the explicit Fock-space oracle: the same
    recorded O sequence replayed on explicit bases gives the same H.psi."""
    from oracle import baseline
    L, N, M, k = 6, 6, 20, 2
    h, v = workloads.integrals(L, seed=0)
    b = baseline.OracleBuilder(h, v)
    applied = workloads.grow_middle_bond(b, L, 3, 3, M, k, seed=4)
    lo, ro = b._blocks()
    it = iter(applied)

    def split(O, dims, kept):
        out, pos = [], 0
        for d, m in zip(dims, kept):
            out.append(np.asarray(O[pos:pos + d * m]).reshape(d, m))
            pos += d * m
        assert pos == len(O)
        return out

    lb, rb = ob.empty_block(), ob.empty_block()
    for s in range(k):
        d, kept, O = next(it)
        assert d == +1
        lay = ob.enlarged_left(lb)
        blocks = split(O, [ob.enlarged_dims(lay)[E] for E in lay], kept)
        lb = ob.grow_left(lb, s, {E: blk for E, blk in zip(lay, blocks)})
    for s in range(L - 1, k + 1, -1):
        d, kept, O = next(it)
        assert d == -1
        lay = ob.enlarged_right(rb)
        blocks = split(O, [ob.enlarged_dims(lay)[E] for E in lay], kept)
        rb = ob.grow_right(rb, s, {E: blk for E, blk in zip(lay, blocks)})
    P = ob.Projected(h, v, lb, rb, 3, 3)
    hp = od.HPsi(b.I, k, lo, ro, 3, 3)
    assert hp.dim == P.dim
    psi = workloads.gaussian(P.dim, seed=9)
    ref = P.apply(psi)
    assert np.max(np.abs(hp.apply(psi) - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("L,nu,nd,M,k", [(8, 4, 4, 30, 3), (9, 5, 3, 24, 3), (10, 4, 5, 40, 2)])
def test_middle_bond_sector_tables_match_the_grown_blocks(L, nu, nd, M, k):
    """The dimension-only sector tables (used to describe the large workloads) equal
    those of blocks actually grown by renormalization with the seeded O."""
    from oracle import baseline
    h, v = workloads.integrals(L, seed=0)
    b = baseline.OracleBuilder(h, v)
    workloads.grow_middle_bond(b, L, nu, nd, M, k, seed=2)
    lb, rb = b._blocks()
    left, right = workloads.middle_bond_sectors(L, nu, nd, M, k)
    assert {tuple(s): d for s, d in zip(lb.sectors, lb.dims) if d > 0} == left
    assert {tuple(s): d for s, d in zip(rb.sectors, rb.dims) if d > 0} == right
