"""GPU: post-processing of converged sweeps.  The exported renormalization
matrices (dmrg_block_basis; the MPS tensors of Sec. 2.1) rebuild the converged
wave function in the determinant basis, where it is the full-CI ground state;
the per-step records of dmrg_sweep_record (energies as dmrg_sweep, discarded
weights, the entropies of every step's two sites) against full CI."""
import numpy as np
import pytest

from oracle import blocks as ob
from oracle import fock
from paper_2001_04890_gb300 import binding, workloads
from tests.helpers import rebuild_blocks

pytestmark = pytest.mark.gpu


def test_exported_bases_rebuild_the_full_ci_state():
    L, N, M, k = 6, 6, 64, 2
    h, v = workloads.integrals(L, seed=12)
    e_fci, x_fci, D = fock.fci_ground(h, v, 3, 3)
    ctx = binding.DMRG(h, v, N, 0, M)
    ctx.sweep(4, tol=1e-10)
    ctx.set_position(k, 1)
    e, _ = ctx.davidson(tol=1e-12, max_iter=400, allow_noconv=True)
    left = {j: ctx.block_basis(0, j) for j in range(1, k + 1)}
    right = {j: ctx.block_basis(1, j) for j in range(1, L - k - 1)}
    psi = ctx.get_psi()
    ctx.close()
    lb = rebuild_blocks(left, L, 0, k)
    rb = rebuild_blocks(right, L, 1, L - k - 2)
    P = ob.Projected(h, v, lb, rb, 3, 3)
    assert P.dim == len(psi)
    assert np.allclose(P.V.T @ P.V, np.eye(P.dim), atol=1e-12)   # orthonormal block bases
    x = P.V @ psi
    assert abs(np.linalg.norm(x) - 1.0) < 1e-12
    assert abs(abs(x @ x_fci) - 1.0) < 1e-9
    assert abs(psi @ P.apply(psi) - e_fci) < 1e-9 and abs(e - e_fci) < 1e-9


def test_sweep_record_matches_sweep_and_full_ci():
    L, N, M, nsw = 6, 6, 64, 4
    h, v = workloads.integrals(L, seed=12)
    e_fci, x_fci, D = fock.fci_ground(h, v, 3, 3)
    a = binding.DMRG(h, v, N, 0, M)
    E = a.sweep(nsw, tol=1e-10)
    a.close()
    b = binding.DMRG(h, v, N, 0, M)
    rec = b.sweep_record(nsw, tol=1e-10)
    b.close()
    assert np.max(np.abs(rec["energies"] - E)) < 1e-10   # the same steps
    assert np.all(rec["discarded"] >= -1e-14) and np.all(rec["discarded"] <= 1.0)
    steps = 2 * (L - 2)
    last = slice((nsw - 1) * steps, nsw * steps)
    assert np.all(np.abs(rec["energies"][last] - e_fci) < 1e-9)   # exact in the last sweep
    assert np.all(rec["discarded"][last] < 1e-10)
    positions = list(range(0, L - 2)) + list(range(L - 2, 0, -1))
    for j, k in enumerate(positions):
        ref = fock.orbital_entropies(fock.pair_rdm_dets(x_fci, D, k))
        got = rec["entropies"][(nsw - 1) * steps + j]
        assert np.max(np.abs(got - np.array(ref))) < 1e-6, (k, got, ref)


def test_mutual_information_matrix_matches_full_ci():
    """dmrg_mutual_information once the sweeps are exact (L=6, M covering every Schmidt
    rank): every two-orbital matrix, adjacent or not, equals the oracle's from the full-CI
    vector (pair_rdm_dets_ij, Jordan-Wigner strings across the orbitals between), and the
    entropies and mutual information follow."""
    L, N = 6, 6
    h, v = workloads.integrals(L, seed=12)
    e_fci, x, D = fock.fci_ground(h, v, 3, 3)
    ctx = binding.DMRG(h, v, N, 0, 4096)
    ctx.sweep(4, tol=1e-11)
    assert ctx.position()[0] == 0
    e, _ = ctx.davidson(tol=1e-12, max_iter=400, allow_noconv=True)
    assert abs(e - e_fci) < 1e-9
    mi = ctx.mutual_information(pair_matrices=True)
    ctx.close()
    for i in range(L):
        for j in range(i + 1, L):
            ref = fock.pair_rdm_dets_ij(x, D, i, j)
            got = mi["rho"][i, j]
            assert np.max(np.abs(got / np.trace(got) - ref)) < 1e-8, (i, j)
            si, sj, sij = fock.orbital_entropies(ref)
            assert abs(mi["s1"][i] - si) < 1e-6 and abs(mi["s1"][j] - sj) < 1e-6
            assert abs(mi["I"][i, j] - (si + sj - sij)) < 1e-6 and mi["I"][i, j] == mi["I"][j, i]
    assert np.all(np.diag(mi["I"]) == 0.0)
