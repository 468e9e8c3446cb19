"""The synthetic workload generators (no arithmetic of the method): the sector-dimension
profile of grown block bases and the seeded integrals keep the properties the
measurements rely on."""
import numpy as np
import pytest

from paper_2001_04890_gb300 import workloads


@pytest.mark.parametrize("seed", range(6))
def test_sector_profile_respects_caps_and_total(seed):
    rng = np.random.default_rng(seed)
    k, L = int(rng.integers(1, 12)), 24
    caps = {(a, b): int(rng.integers(0, 40)) for a in range(k + 2) for b in range(k + 2) if rng.random() < 0.7}
    M = int(rng.integers(1, 300))
    prof = workloads.sector_dims_profile(k, 12, 12, L, M, caps)
    assert all(0 < m <= caps[key] for key, m in prof.items())
    assert sum(prof.values()) == min(M, sum(caps.values()))


def test_sector_profile_follows_the_gaussian_weights():
    # without binding caps the kept dimensions decrease away from the profile's centre
    k, L, nu, nd = 8, 16, 8, 8
    caps = {(a, b): 10 ** 6 for a in range(k + 1) for b in range(k + 1)}
    prof = workloads.sector_dims_profile(k, nu, nd, L, 2000, caps)
    centre = (k * nu / L, k * nd / L)
    dist = lambda key: (key[0] - centre[0]) ** 2 + (key[1] - centre[1]) ** 2
    keys = sorted(prof, key=dist)
    assert keys[0] == (4, 4)
    assert all(prof[a] >= prof[b] for a, b in zip(keys, keys[1:]) if dist(a) < dist(b))


def test_integrals_are_symmetric_and_seeded():
    h, v = workloads.integrals(7, seed=3)
    h2, v2 = workloads.integrals(7, seed=3)
    assert np.array_equal(h, h2) and np.array_equal(v, v2)
    assert np.allclose(h, h.T, atol=0)
    # chemists' 8-fold symmetry and positive semi-definiteness over pair indices
    for perm in ("jikl", "ijlk", "klij"):
        assert np.allclose(v, np.einsum(f"ijkl->{perm}", v), atol=1e-15)
    w = np.linalg.eigvalsh(v.reshape(49, 49))
    assert w.min() > -1e-12
    assert np.allclose(np.diag(h), -2 + 4 * np.arange(7) / 7)


@pytest.mark.parametrize("key", ["c1", "c2", "c3", "c5a", "c5b"])
def test_recorded_hpsi_flops_equal_the_planner_count(key):
    """bench.py records each workload's algorithmic H.psi FLOPs (so that its oracle arm
    loads no library); they equal the host planner's count on the same sector tables."""
    import importlib.util
    import os
    from paper_2001_04890_gb300 import binding
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    wl = bench.WORKLOADS[key]
    L, N, tsz, M = wl["L"], wl["N"], wl["two_sz"], wl["M"]
    k = (L - 2) // 2
    left, right = workloads.middle_bond_sectors(L, (N + tsz) // 2, (N - tsz) // 2, M, k)
    tl = [(a, b, d) for (a, b), d in sorted(left.items()) if d > 0]
    tr = [(a, b, d) for (a, b), d in sorted(right.items()) if d > 0]
    h, v = workloads.integrals(L, seed=0)
    assert binding.plan_hpsi_flops(h, v, N, tsz, k, tl, tr)[0] == wl["hpsi_flops"]
