"""Host checks of the execution plan the GPU runs for one H.psi (Sec. 2.2.1,
Eq. dgemm): every task of every output block runs exactly once, in the
association the cost rule picks, inside equal-work chunks whose scratch slots
the ordered reduction adds back into that block; chunks go to the kernel the
routing rule names.  No GPU: the plan is dumped by the library's planner."""
import collections

import numpy as np
import pytest

from paper_2001_04890_gb300 import binding, workloads

CASES = [(10, 10, 0, 60, 4), (12, 13, 1, 100, 5), (9, 9, -1, 40, 3), (14, 14, 0, 160, 6), (10, 10, 0, 256, 4)]
TUNES = [None, [64.0, 0.0, 33, 0], [1e9, 0.0, 1, 1], [8.0, 1e12, 64, 0], [4096.0, 5e4, 17, 1]]


def _tables(L, N, tsz, M, k):
    nu, nd = (N + tsz) // 2, (N - tsz) // 2
    l, r = workloads.middle_bond_sectors(L, nu, nd, M, k)
    return [(a, b, d) for (a, b), d in sorted(l.items())], [(a, b, d) for (a, b), d in sorted(r.items())]


def _flops(m, n, p, q, xid, zid):
    if xid and zid:
        return 0.0
    if xid:
        return 2.0 * n * p * q
    if zid:
        return 2.0 * m * n * p
    return 2.0 * min(m * n * p + m * p * q, n * p * q + m * n * q)


def _transposed_cheaper(m, n, p, q):
    return n * p * q + m * n * q < m * n * p + m * p * q


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("tune", TUNES)
@pytest.mark.parametrize("tc", [False, True])
def test_execution_plan_runs_every_task_once(case, tune, tc):
    L, N, tsz, M, k = case
    sl, sr = _tables(L, N, tsz, M, k)
    h, v = workloads.integrals(L, seed=0)
    _check_plan(h, v, N, tsz, k, sl, sr, tc, tune)


@pytest.mark.parametrize("seed", range(8))
def test_execution_plan_on_random_layouts(seed):
    rng = np.random.default_rng(200 + seed)
    L = int(rng.integers(5, 9))
    k = int(rng.integers(0, L - 1))
    N = int(rng.integers(2, 2 * L - 1))
    tsz = int(rng.choice([x for x in range(-N, N + 1, 2) if (N - x) // 2 <= L and (N + x) // 2 <= L]))

    def table(n_sites):
        if n_sites == 0:
            return [(0, 0, 1)]
        out = [(a, b, int(rng.integers(1, 40))) for a in range(n_sites + 1) for b in range(n_sites + 1)
               if rng.random() < 0.7]
        return out or [(0, 0, 1)]
    sl, sr = table(k), table(L - k - 2)
    h, v = workloads.integrals(L, seed=seed)
    for tc in (False, True):
        for tune in (None, [64.0, 0.0, 9, 1]):
            _check_plan(h, v, N, tsz, k, sl, sr, tc, tune)


def _check_plan(h, v, N, tsz, k, sl, sr, tc, tune):
    tasks = binding.debug_tasks(h, v, N, tsz, k, sl, sr, grouped=True)
    cnt, xs, ch, red = binding.debug_exec(h, v, N, tsz, k, sl, sr, tensor_cores=tc, tune=tune)
    target, min_chunk, tc_min, by_work = (8192.0, 2e5, 33, 0) if tune is None else tune
    assert cnt["entries"] == len(tasks) == len(xs)
    if len(tasks) == 0:
        assert len(ch) == 0 and len(red) == 0
        return

    # output blocks in grouped order, each with its tasks
    blocks = []
    for g, m, n, p, q, fl, y in tasks:
        if not blocks or blocks[-1][0] != g:
            blocks.append((g, m, q, []))
        blocks[-1][3].append((int(y), int(n), int(p), int(fl)))
    assert len(red) == len(blocks) == cnt["reduce_groups"]
    total = sum(1.0 + _flops(m, n, p, q, fl & 1, fl & 2) for _, m, q, ts in blocks for (_, n, p, fl) in ts)
    chunk_work = max(total / target, min_chunk)

    # reduction: contiguous reduced elements and scratch slots, block by block
    e0 = soff = 0
    slot_of = {}
    for r, (g, m, q, ts) in zip(red, blocks):
        r_e0, r_soff, r_d, drs, dcs, rm, rq, nsplit = (int(x) for x in r)
        assert (r_e0, r_soff, rm, rq, drs, dcs) == (e0, soff, m, q, q, 1)
        assert nsplit >= 1
        for i in range(nsplit):
            slot_of[soff + i * m * q] = (len(slot_of), g)
        e0 += m * q
        soff += nsplit * m * q
    assert (cnt["reduced"], cnt["scratch"]) == (e0, soff)

    # chunks: every slot written by exactly one chunk; entries back in the stored association
    red_of_block = {b[0]: (int(r[5]), int(r[6])) for b, r in zip(blocks, red)}
    seen_slots = collections.Counter()
    per_block = collections.defaultdict(collections.Counter)
    tiles = 0
    kinds = {0: [], 1: [], 2: []}
    for kind, d, drs, dcs, m, q, first, count in ch:
        assert int(d) in slot_of
        seen_slots[int(d)] += 1
        _, g = slot_of[int(d)]
        bm, bq = red_of_block[g]
        # a transposed chunk writes the m x q slot through (1, q) strides as a q x m block;
        # for a 1 x 1 block only its entries tell: they read Y^T, strides (1, n) not (p, 1)
        if (bm, bq) != (1, 1):
            transposed = (int(m), int(q), int(drs), int(dcs)) != (bm, bq, bq, 1)
        else:
            ent = xs[first:first + count]
            transposed = bool(np.any((ent[:, 3] != ent[:, 2]) | (ent[:, 4] != 1)))
        if transposed:
            assert (m, q, drs, dcs) == (bq, bm, 1, bq)
        else:
            assert (m, q) == (bm, bq)
        assert count >= 1
        work = 0.0
        ok_tc = True
        for y, n, p, yrs, ycs, fl, x, z in xs[first:first + count]:
            if transposed:
                assert fl == 0 and (yrs, ycs) == (1, n)
                key = (int(y), int(p), int(n), 0)
                assert _transposed_cheaper(bm, int(p), int(n), bq)
            else:
                assert (yrs, ycs) == (p, 1)
                key = (int(y), int(n), int(p), int(fl))
            per_block[g][key] += 1
            w = 1.0 + _flops(int(m), int(n), int(p), int(q), fl & 1, fl & 2)
            work += w
            ok_tc &= 1 <= n <= 128 and 1 <= p <= 128 and (not fl & 1 or n == m) and (not fl & 2 or p == q)
        assert count == 1 or work <= chunk_work
        shape_tc = tc and m <= 128 and q <= 128 and (m >= tc_min or q >= tc_min)
        if kind == 2:
            assert shape_tc and ok_tc and not transposed
        elif kind == 1:
            assert m <= 32 and q <= 32 and not (shape_tc and ok_tc)
        else:
            assert not (m <= 32 and q <= 32) and not (shape_tc and ok_tc)
            tiles += -(-int(m) // 32) * -(-int(q) // 32)
        kinds[int(kind)].append(work)
    assert all(c == 1 for c in seen_slots.values()) and len(seen_slots) == len(slot_of)
    assert cnt["tiles"] == tiles
    for g, m, q, ts in blocks:
        assert per_block[g] == collections.Counter(ts)
        # the cost rule: an entry of a non-tensor-core block with no identity side runs transposed
        # exactly when that association is strictly cheaper
    for kd in (1, 2):
        if by_work:
            assert kinds[kd] == sorted(kinds[kd], key=lambda w: -w)


def test_execution_plan_orientation_rule_is_applied():
    # at least one entry of a realistic layout runs transposed, and never on the tensor-core kernel
    L, N, tsz, M, k = 14, 14, 0, 160, 6
    sl, sr = _tables(L, N, tsz, M, k)
    h, v = workloads.integrals(L, seed=0)
    tasks = binding.debug_tasks(h, v, N, tsz, k, sl, sr, grouped=True)
    cnt, xs, ch, red = binding.debug_exec(h, v, N, tsz, k, sl, sr)
    want = sum(1 for g, m, n, p, q, fl, y in tasks if fl == 0 and _transposed_cheaper(m, n, p, q))
    # transposed chunks: slot written as q x m through (1, q) strides
    red_shape = {}
    for r in red:
        for i in range(int(r[7])):
            red_shape[int(r[1]) + i * int(r[5]) * int(r[6])] = (int(r[5]), int(r[6]))
    got = 0
    for kind, d, drs, dcs, m, q, first, count in ch:
        bm, bq = red_shape[int(d)]
        if (bm, bq) != (1, 1) and (int(m), int(q), int(drs), int(dcs)) == (bq, bm, 1, bq):
            got += int(count)
        elif (bm, bq) == (1, 1):
            e = xs[first:first + count]
            got += int(np.sum((e[:, 3] != e[:, 2]) | (e[:, 4] != 1)))
    assert want > 0 and got == want


@pytest.mark.parametrize("case", CASES + [(24, 24, 0, 512, 11)])
@pytest.mark.parametrize("tc", [False, True])
def test_every_operand_view_stays_inside_its_array(case, tc):
    """Host bounds check of the execution plan (the descriptors the kernels read): every
    X / Z view inside its operator arena, every psi view inside psi, every chunk slot and
    reduction inside the scratch array."""
    L, N, tsz, M, k = case
    sl, sr = _tables(L, N, tsz, M, k)
    h, v = workloads.integrals(L, seed=0)
    checked, bad, first = binding.debug_validate(h, v, N, tsz, k, sl, sr, tensor_cores=tc)
    assert checked > 0 and bad == 0, first


@pytest.mark.parametrize("seed", range(10))
def test_operand_views_in_bounds_on_random_layouts(seed):
    rng = np.random.default_rng(400 + seed)
    L = int(rng.integers(4, 10))
    k = int(rng.integers(0, L - 1))
    N = int(rng.integers(1, 2 * L))
    tsz = int(rng.choice([x for x in range(-N, N + 1, 2) if (N - x) // 2 <= L and (N + x) // 2 <= L]))

    def table(n_sites):
        if n_sites == 0:
            return [(0, 0, 1)]
        out = [(a, b, int(rng.integers(1, 70))) for a in range(n_sites + 1) for b in range(n_sites + 1)
               if rng.random() < 0.7]
        return out or [(0, 0, 1)]
    sl, sr = table(k), table(L - k - 2)
    h, v = workloads.integrals(L, seed=seed)
    # the default launch shape and shapes the autotuner can pick (split granularity,
    # tensor-core routing threshold, group order); with tensor cores, the tile plan too
    tunes = [None, [1.0, 0.0, 1, 1], [32768.0, 5.0e4, 17, 0], [8192.0, 2.0e5, 1, 1], [64.0, 1.0e7, 65, 1],
             [8192.0, 2.0e5, 1, 1, 1]]
    for tc in (False, True):
        for tune in tunes:
            checked, bad, first = binding.debug_validate(h, v, N, tsz, k, sl, sr, tensor_cores=tc, tune=tune)
            assert checked > 0 and bad == 0, (tune, first)
