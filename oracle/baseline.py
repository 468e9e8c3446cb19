"""CPU baseline and reference arm of bench.py: the FP64 oracle timed on host cores.

TEST INFRASTRUCTURE ONLY (see oracle/fock.py).  The oracle is used as it
stands (no tuning for speed).  It builds the same middle-bond blocks as the
GPU run (the same seeded random O, drawn by paper_2001_04890_gb300.workloads
from this oracle's own enlarged layouts) and times H.psi applications of
Eq. h_mat at the middle bond; a bounded sample keeps the CPU time to about
10-30 s.
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import dmrg as od


class OracleBuilder:
    """Duck-typed stand-in for the library context used by workloads.grow_middle_bond."""

    def __init__(self, h, v):
        self.I = od.Ints(h, v)
        self.L = h.shape[0]
        self.left = {0: od.empty_oblock(0)}
        self.right = {0: od.empty_oblock(1)}
        self.k = 0

    def set_position(self, k, direction=1):
        self.k = k

    def _blocks(self):
        lb = self.left.get(self.k, od.empty_oblock(0))
        rb = self.right.get(self.L - self.k - 2, od.empty_oblock(1))
        return lb, rb

    def enlarged_layout(self, direction):
        lb, rb = self._blocks()
        E = od.Enl(lb if direction > 0 else rb, 0 if direction > 0 else 1)
        return np.array([(Ek[0], Ek[1], d) for Ek, d in zip(E.E, E.dim)], dtype=np.int64).reshape(-1, 3)

    def renormalize(self, direction, O, kept):
        lb, rb = self._blocks()
        E = od.Enl(lb if direction > 0 else rb, 0 if direction > 0 else 1)
        blocks, pos = [], 0
        for d, m in zip(E.dim, kept):
            blocks.append(np.asarray(O[pos:pos + d * m]).reshape(d, m))
            pos += d * m
        nb = od.renormalize(self.I, self.k, lb, rb, direction, blocks, kept)
        if direction > 0:
            self.left[self.k + 1] = nb
            self.k += 1
        else:
            self.right[self.L - self.k - 1] = nb
            self.k -= 1


def _threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def middle_bond(wl, seed=0):
    from paper_2001_04890_gb300 import workloads
    L, N, two_sz, M = wl["L"], wl["N"], wl["two_sz"], wl["M"]
    nu, nd = (N + two_sz) // 2, (N - two_sz) // 2
    k = (L - 2) // 2
    h, v = workloads.integrals(L, seed=0)
    b = OracleBuilder(h, v)
    workloads.grow_middle_bond(b, L, nu, nd, M, k, seed=seed)
    lb, rb = b._blocks()
    return b.I, k, lb, rb, nu, nd


def sector_tables(lb, rb):
    """(n_up, n_dn, dim) rows of the two middle-bond blocks."""
    tl = [(a, b, d) for (a, b), d in zip(lb.sectors, lb.dims)]
    tr = [(a, b, d) for (a, b), d in zip(rb.sectors, rb.dims)]
    return tl, tr


def cpu_baseline(wl, flops, budget_s=20.0, note=""):
    """Oracle H.psi at the middle bond, timed on the host cores for about budget_s seconds.

    flops: the algorithmic FLOPs of one H.psi of this workload (the count the GPU
    arm uses, recorded with the workload), so value is in the GPU arm's unit.
    """
    I, k, lb, rb, nu, nd = middle_bond(wl)
    t0 = time.perf_counter()
    hp = od.HPsi(I, k, lb, rb, nu, nd)
    t_build = time.perf_counter() - t0
    from paper_2001_04890_gb300 import workloads
    psi = workloads.gaussian(hp.dim, seed=1)
    n, t = 0, 0.0
    while (t < budget_s or n == 0) and n < 50:
        t1 = time.perf_counter()
        hp.apply(psi)
        t += time.perf_counter() - t1
        n += 1
    s = t / n
    return {"value": flops / s / 1e12, "unit": "TFLOP/s", "cores": _threads(), "kind": "oracle",
            "sample": (f"{n} oracle H.psi applications at the middle bond of {wl['name']} (psi dim "
                       f"{hp.dim}, {len(hp.terms)} two-half terms), {s:.3f} s each; block growth and "
                       f"the oracle's operator pre-summation ({t_build:.1f} s) not timed" + note),
            "s_per_hpsi": s}


def reference_line(wl, steps, warmup, metric, flops, note=""):
    """bench.py --impl reference: the oracle timed on the host cores, same metric and config."""
    I, k, lb, rb, nu, nd = middle_bond(wl)
    hp = od.HPsi(I, k, lb, rb, nu, nd)
    from paper_2001_04890_gb300 import workloads
    psi = workloads.gaussian(hp.dim, seed=1)
    for _ in range(warmup):
        hp.apply(psi)
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        hp.apply(psi)
        ts.append(time.perf_counter() - t0)
    s = float(np.mean(ts))
    value = flops / s / 1e12
    cores = _threads()
    return {"impl": "reference", "metric": metric, "value": value, "unit": "TFLOP/s", "n_gpus": 0,
            "steps": steps, "warmup": warmup, "ms_per_step": s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "L": wl["L"], "N": wl["N"], "two_sz": wl["two_sz"],
                       "M": wl["M"], "position": k, "psi_dim": hp.dim,
                       "step": "one FP64 oracle H.psi application at the middle bond (bounded sample)" + note},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} oracle H.psi applications at the middle bond after "
                                       f"{warmup} untimed ones"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
