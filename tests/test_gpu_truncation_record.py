"""GPU: the record of density-matrix truncations (Sec. 2.1) that sweeps leave
in a context (dmrg_truncation_stats): one entry per RDM truncation, none for a
caller-given basis, gaps between the kept and the cut spectrum non-negative."""
import numpy as np
import pytest

from paper_2001_04890_gb300 import binding, workloads
from tests.helpers import build_random_position

pytestmark = pytest.mark.gpu


def test_sweeps_record_every_truncation():
    L, N, M, nsw = 8, 8, 16, 2
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, 0, M)
    s0 = ctx.truncation_stats()
    ctx.sweep(nsw, tol=1e-10)
    s = ctx.truncation_stats()
    ctx.close()
    assert s["truncations"] - s0["truncations"] == nsw * 2 * (L - 2)
    assert 0 <= s["straddled"] <= s["truncations"]
    assert s["min_gap"] >= 0.0 and s["last_gap"] >= s["min_gap"]


def test_caller_basis_is_not_a_truncation():
    L, N, M = 6, 6, 12
    h, v = workloads.integrals(L, seed=2)
    ctx = binding.DMRG(h, v, N, 0, M)
    s0 = ctx.truncation_stats()
    build_random_position(ctx, h, v, 2, M, seed=1)
    s = ctx.truncation_stats()
    ctx.close()
    assert s["truncations"] == s0["truncations"]
