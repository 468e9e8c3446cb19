"""The library's density-matrix truncation rule (Sec. 2.1: keep the eigenvectors
with the largest eigenvalues over all sectors) against the oracle's, on the
host: the same spectra give the same kept set, in the same order, including
exact ties, near-degenerate clusters across the cut and eigenvalues at the
drop threshold; the kept count also against a brute-force statement of the
rule."""
import numpy as np
import pytest

from oracle import blocks as ob
from paper_2001_04890_gb300 import binding


def _oracle_choice(spectra, M):
    # diagonal rho per sector: eigh returns the spectrum itself, ascending
    rho = {(s, 0): np.diag(np.asarray(ev, dtype=np.float64)) for s, ev in enumerate(spectra)}
    O, kept, dw, eig = ob.truncate(rho, M)
    asc = [eig[E][0][::-1].copy() for E in rho]
    cols = []
    for E, ev in zip(rho, asc):
        n = len(ev)
        # kept columns of O are unit vectors: recover each one's ascending index
        js = [int(np.argmax(np.abs(O[E][:, c]))) for c in range(O[E].shape[1])]
        cols.append(js)
    return asc, kept, dw, cols


def _gap(spectra, kept_total, drop=1e-13):
    # brute force over (value, sector, rank from the top) in the documented order
    allv = []
    for s, ev in enumerate(spectra):
        top = sorted(ev, reverse=True)
        allv += [(-x, s, j) for j, x in enumerate(top)]
    allv.sort()
    if kept_total == 0 or kept_total >= len(allv) or -allv[kept_total][0] <= drop:
        return np.inf
    return -allv[kept_total - 1][0] - -allv[kept_total][0]


CASES = []
rng = np.random.default_rng(7)
for t in range(60):
    ns = int(rng.integers(1, 6))
    if t % 3 == 0:
        pool = np.array([0.0, 1e-14, 1e-13, 0.05, 0.1, 0.2])   # exact ties and the drop threshold
        spectra = [np.sort(rng.choice(pool, size=int(rng.integers(0, 6)))) for _ in range(ns)]
    elif t % 3 == 1:
        spectra = [np.sort(rng.random(int(rng.integers(0, 7)))) for _ in range(ns)]
    else:
        spectra = [np.sort(np.round(rng.random(int(rng.integers(1, 7))), 1)) for _ in range(ns)]
    CASES.append(spectra)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_library_truncation_equals_oracle(case):
    spectra = CASES[case]
    total = sum(len(s) for s in spectra)
    for M in range(0, total + 2):
        asc, kept_o, dw_o, cols_o = _oracle_choice(spectra, M)
        kept, cols, trace, kw, gap = binding.debug_truncation(asc, M)
        assert list(kept) == list(kept_o), (spectra, M)
        for c_lib, c_or in zip(cols, cols_o):
            # same columns; the library lists the largest eigenvalue first
            assert sorted(c_lib.tolist()) == sorted(c_or)
            assert list(c_lib) == sorted(c_lib.tolist(), reverse=True)
        assert abs((trace - kw) - dw_o) <= 1e-15 * max(1.0, trace)
        g = _gap(asc, int(np.sum(kept)))
        assert (np.isinf(gap) and np.isinf(g)) or abs(gap - g) <= 1e-15


def _brute_kept_count(spectra, M, drop=1e-13, cluster=1e-10):
    """The documented rule by brute force: the largest prefix of the global order
    with at most M states whose cut does not split a cluster (gap >= 1e-10 to the
    next eigenvalue above drop); M itself (capped) if that prefix is empty."""
    vals = sorted([x for ev in spectra for x in ev if x > drop], reverse=True)
    n = min(M, len(vals))
    for c in range(n, 0, -1):
        if c == len(vals) or vals[c - 1] - vals[c] >= cluster:
            return c
    return n


@pytest.mark.parametrize("case", range(len(CASES)))
def test_library_truncation_count_equals_brute_force(case):
    spectra = [np.asarray(s, dtype=np.float64) for s in CASES[case]]
    total = sum(len(s) for s in spectra)
    for M in range(0, total + 2):
        kept = binding.debug_truncation(spectra, M)[0]
        assert int(np.sum(kept)) == _brute_kept_count(spectra, M), (spectra, M)


def test_library_truncation_gap_flags_straddling_cluster():
    # 0.3 kept in one sector, its exact twin cut in another: gap 0
    kept, cols, trace, kw, gap = binding.debug_truncation([np.array([0.1, 0.3]), np.array([0.3])], 1)
    assert list(kept) == [1, 0] and gap == 0.0
    kept, cols, trace, kw, gap = binding.debug_truncation([np.array([0.1, 0.3]), np.array([0.3])], 2)
    assert list(kept) == [1, 1] and abs(gap - 0.2) < 1e-15
    # a straddling tie below the top cluster: the cut moves above it
    kept, cols, trace, kw, gap = binding.debug_truncation([np.array([0.3, 0.5]), np.array([0.3])], 2)
    assert list(kept) == [1, 0] and abs(gap - 0.2) < 1e-15
    # nothing above the drop threshold cut: no gap
    kept, cols, trace, kw, gap = binding.debug_truncation([np.array([0.0, 1e-13, 0.5])], 1)
    assert list(kept) == [1] and np.isinf(gap)


def test_library_truncation_rejects_bad_arguments():
    with pytest.raises(binding.DMRGError):
        binding.debug_truncation([np.array([0.5])], -1)
