"""Host checks of the tensor-core launch plan (the grouped products of Eq.
dgemm, Sec. 2.2.1, on the tcgen05 kernel): blocks ordered by kernel shape,
tasks stacked by shared psi block, and every operator view and psi block
staged once as a tile, in order of first use, at the offset each task reads.
No GPU: the plan is dumped by the library's planner."""
import numpy as np
import pytest

from paper_2001_04890_gb300 import binding, workloads

CASES = [(12, 12, 0, 200, 5), (13, 13, 1, 150, 5), (10, 10, 0, 256, 4), (12, 12, 0, 1024, 5)]
# target_chunks, min_chunk, tc_min, by_work[, tc_tiny]
TUNES = [[8192.0, 2e5, 1, 0], [64.0, 0.0, 9, 1], [4096.0, 5e4, 17, 0], [8192.0, 2e5, 1, 1, 1]]


def _c16(x):
    return (x + 15) // 16 * 16


def _tables(L, N, tsz, M, k):
    nu, nd = (N + tsz) // 2, (N - tsz) // 2
    l, r = workloads.middle_bond_sectors(L, nu, nd, M, k)
    return [(a, b, d) for (a, b), d in sorted(l.items())], [(a, b, d) for (a, b), d in sorted(r.items())]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("tune", TUNES)
def test_tensor_core_plan(case, tune):
    L, N, tsz, M, k = case
    sl, sr = _tables(*case)
    h, v = workloads.integrals(L, seed=0)
    assert _check_tc(h, v, N, tsz, k, sl, sr, tune) > 0


@pytest.mark.parametrize("seed", range(8))
def test_tensor_core_plan_on_random_layouts(seed):
    rng = np.random.default_rng(300 + seed)
    L = int(rng.integers(5, 9))
    k = int(rng.integers(0, L - 1))
    N = int(rng.integers(2, 2 * L - 1))
    tsz = int(rng.choice([x for x in range(-N, N + 1, 2) if (N - x) // 2 <= L and (N + x) // 2 <= L]))

    def table(n_sites):
        if n_sites == 0:
            return [(0, 0, 1)]
        out = [(a, b, int(rng.integers(1, 90))) for a in range(n_sites + 1) for b in range(n_sites + 1)
               if rng.random() < 0.7]
        return out or [(0, 0, 1)]
    sl, sr = table(k), table(L - k - 2)
    h, v = workloads.integrals(L, seed=seed)
    for tune in ([8192.0, 2e5, 1, 0], [64.0, 0.0, 17, 1], [64.0, 0.0, 1, 0, 1]):
        _check_tc(h, v, N, tsz, k, sl, sr, tune)


def _check_tc(h, v, N, tsz, k, sl, sr, tune):
    cnt, te, tg, ts, ps = binding.debug_tc(h, v, N, tsz, k, sl, sr, tune=tune)
    _, xs, ch, _ = binding.debug_exec(h, v, N, tsz, k, sl, sr, tensor_cores=True, tune=tune)
    if cnt["tasks"] == 0:
        assert len(tg) == 0 and cnt["op_bytes"] == 0
        return 0
    # blocks: the tensor-core chunks of the execution plan, by shape 64x32, 64x64, 128x128
    tc_chunks = ch[ch[:, 0] == 2]
    assert len(tg) == len(tc_chunks) == cnt["blocks"]
    assert cnt["shape64x32"] + cnt["shape64x64"] + cnt["shape128"] == len(tg)
    pmax = {}
    for c in tc_chunks:
        pmax[int(c[1])] = int(xs[c[6]:c[6] + c[7], 2].max())
    fits = lambda g, lim: g[3] <= 64 and g[4] <= lim and pmax[int(g[0])] <= lim
    # the 32-column shape: when every block fits it, or (tc_tiny) for each block that fits it
    all_tiny = all(fits(g, 32) for g in tg)
    tiny = len(tune) > 4 and tune[4] == 1
    shapes = [2 if (all_tiny or (tiny and fits(g, 32))) else (1 if fits(g, 64) else 0) for g in tg]
    assert shapes == sorted(shapes, reverse=True)
    assert shapes.count(2) == cnt["shape64x32"] and shapes.count(1) == cnt["shape64x64"]
    want = {}
    for c in tc_chunks:
        want.setdefault((int(c[1]), int(c[2]), int(c[3]), int(c[4]), int(c[5])), []).append(set(range(c[6], c[6] + c[7])))
    first = 0
    op_seen, ps_seen = [], []
    op_set, ps_set = set(), set()
    for g, sh in zip(tg, shapes):
        d, drs, dcs, m, q, gfirst, count = (int(x) for x in g)
        assert gfirst == first
        first += count
        tasks = te[gfirst:gfirst + count]
        # the same execution-list entries as the chunk it came from
        assert set(tasks[:, 4].tolist()) in want[(d, drs, dcs, m, q)]
        # grouped by psi block (stable), stacks = runs on one psi block, capped
        ys = tasks[:, 11]
        assert np.all(np.diff(ys) >= 0)
        cap = max(1, min(8, (128 if sh == 0 else 64) // _c16(m)))
        i = 0
        while i < count:
            run = int(tasks[i, 3])
            assert 1 <= run <= cap and np.all(tasks[i + 1:i + run, 3] == 0)
            assert np.all(ys[i:i + run] == ys[i])
            nxt = i + run
            if nxt < count and ys[nxt] == ys[i]:
                assert run == cap   # a run is split only at the cap
            i = nxt
        for t in tasks:
            xt, yt, zt, stack, src, x, xrs, xcs, z, zrs, zcs, y, n, p = (int(a) for a in t)
            xv = (-1, 0, 0, n, n) if x == -1 else (4 * x, xrs, xcs, m, n)
            zv = (-1, 0, 0, p, p) if z == -1 else (4 * z, zcs, zrs, q, p)
            for view in (xv, zv):
                if view not in op_set:
                    op_set.add(view)
                    op_seen.append(view)
            if y not in ps_set:
                ps_set.add(y)
                ps_seen.append(y)
    assert first == cnt["tasks"]
    # operator tiles: one per distinct view, laid out in order of first use
    assert [tuple(int(a) for a in (r[0], r[2], r[3], r[4], r[5])) for r in ts] == op_seen
    off = 0
    for r in ts:
        assert r[1] == off
        off += _c16(int(r[4])) * _c16(int(r[5])) * 4
    assert off == cnt["op_bytes"]
    tile_of = {tuple(int(a) for a in (r[0], r[2], r[3], r[4], r[5])): int(r[1]) for r in ts}
    # psi tiles: one per psi block read, in order of first use, rows p and columns n
    assert [int(r[0]) for r in ps] == ps_seen
    off = 0
    for r in ps:
        assert r[1] == off
        off += _c16(int(r[3])) * _c16(int(r[2])) * 4
    assert off == cnt["psi_bytes"]
    psi_of = {int(r[0]): (int(r[1]), int(r[2]), int(r[3])) for r in ps}
    # every task reads the tiles of its own views
    for g in tg:
        m, q, gfirst, count = int(g[3]), int(g[4]), int(g[5]), int(g[6])
        for t in te[gfirst:gfirst + count]:
            xt, yt, zt, stack, src, x, xrs, xcs, z, zrs, zcs, y, n, p = (int(a) for a in t)
            xv = (-1, 0, 0, n, n) if x == -1 else (4 * x, xrs, xcs, m, n)
            zv = (-1, 0, 0, p, p) if z == -1 else (4 * z, zcs, zrs, q, p)
            assert tile_of[xv] == xt and tile_of[zv] == zt
            assert psi_of[y] == (yt, n, p)
    return cnt["tasks"]
