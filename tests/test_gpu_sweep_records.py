"""GPU: what sweeps leave in a context besides energies.

The record of density-matrix truncations (Sec. 2.1, dmrg_truncation_stats):
one entry per RDM truncation, none for a caller-given basis, gaps between the
kept and the cut spectrum non-negative.  The orbital entropies of the
converged two-site wave function (dmrg_orbital_entropies) against full CI."""
import numpy as np
import pytest

from oracle import fock
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


def test_orbital_entropies_of_the_converged_state_match_full_ci():
    L, N, M, k = 6, 6, 64, 2
    h, v = workloads.integrals(L, seed=12)
    e_fci, x, D = fock.fci_ground(h, v, 3, 3)
    ctx = binding.DMRG(h, v, N, 0, M)
    ctx.sweep(4, tol=1e-10)
    ctx.set_position(k, 1)   # two-site blocks on both sides: the superblock is the full space
    e, _ = ctx.davidson(tol=1e-12, max_iter=400, allow_noconv=True)
    ent = ctx.orbital_entropies()
    lay, _ = ctx.psi_layout()
    psi = ctx.get_psi()
    ctx.close()
    assert abs(e - e_fci) < 1e-9
    ref = fock.orbital_entropies(fock.pair_rdm_dets(x, D, k))
    got = (ent["s_left"], ent["s_right"], ent["s_pair"])
    assert np.max(np.abs(np.array(got) - np.array(ref))) < 1e-5, (got, ref)
    assert ent["s_left"] + ent["s_right"] - ent["s_pair"] >= -1e-12  # mutual information >= 0
    # the context's routine and the host-only one agree on the same vector
    rho, s3 = binding.debug_pair_rdm(lay, psi)
    assert np.array_equal(rho, ent["rho2"]) and np.allclose(s3, got, rtol=0, atol=0)
