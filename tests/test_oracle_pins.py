"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Closed forms, textbook special cases, first-quantized rewrites and invariants,
chosen so that a dropped term, a wrong sign, a transposed integral index or a
wrong 1/2 in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import fock
from oracle import blocks as ob
from paper_2001_04890_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ground(h, v, nu, nd):
    H, D = fock.hamiltonian_dets(h, v, nu, nd)
    if H.shape[0] == 0:
        return None
    return float(np.linalg.eigvalsh(H.toarray())[0])


# ---------------------------------------------------------------- site basis

def test_site_matrices_match_printed_eq_creation_ops_up_to_labels():
    """Eq. creation_ops as printed equals our matrices after swapping the labels of states 1 and 2."""
    printed = np.loadtxt(os.path.join(GOLDEN, "creation_ops_printed.txt"))
    up_printed, dn_printed = printed[:4], printed[4:]
    cu, cd, _ = fock.site_ops()
    perm = [0, 2, 1, 3]  # stated order {0,up,dn,updn} <-> order where the printed matrices hold
    P = np.eye(4)[perm]
    assert np.array_equal(P @ cu @ P.T, up_printed)
    assert np.array_equal(P @ cd @ P.T, dn_printed)


def test_canonical_anticommutators_on_three_sites():
    cdag = fock.fock_creation(3)
    c = [m.T for m in cdag]
    dim = 4 ** 3
    I = np.eye(dim)
    for m in range(6):
        for n in range(6):
            ac = (c[m] @ cdag[n] + cdag[n] @ c[m]).toarray()
            assert np.allclose(ac, I if m == n else 0 * I)
            cc = (cdag[m] @ cdag[n] + cdag[n] @ cdag[m]).toarray()
            assert np.allclose(cc, 0 * I)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("t,U", [(1.0, 4.0), (0.3, 1.7), (2.0, 0.0)])
def test_hubbard_dimer_closed_form(t, U):
    h, v = workloads.hubbard_dimer(t, U)
    E = _ground(h, v, 1, 1)
    assert abs(E - (U - np.sqrt(U * U + 16 * t * t)) / 2) < 1e-12


def test_single_orbital_double_occupancy():
    h = np.array([[-1.3]])
    v = np.full((1, 1, 1, 1), 0.77)
    assert abs(_ground(h, v, 1, 1) - (2 * -1.3 + 0.77)) < 1e-14


@pytest.mark.parametrize("L,nu,nd", [(6, 3, 3), (6, 4, 2), (5, 2, 1)])
def test_noninteracting_limit_is_orbital_sum(L, nu, nd):
    h, _ = workloads.integrals(L, seed=3)
    v = np.zeros((L,) * 4)
    eps = np.linalg.eigvalsh(h)
    E = _ground(h, v, nu, nd)
    assert abs(E - (eps[:nu].sum() + eps[:nd].sum())) < 1e-11


def test_one_electron_is_lowest_orbital_energy():
    h, v = workloads.integrals(5, seed=4)
    assert abs(_ground(h, v, 1, 0) - np.linalg.eigvalsh(h)[0]) < 1e-12


def test_closed_shell_full_filling_energy():
    """N = 2L: a single determinant, E = 2 sum h_ii + sum_ij [2 (ii|jj) - (ij|ji)]."""
    L = 4
    h, v = workloads.integrals(L, seed=5)
    ref = 2 * np.trace(h) + sum(2 * v[i, i, j, j] - v[i, j, j, i] for i in range(L) for j in range(L))
    assert abs(_ground(h, v, L, L) - ref) < 1e-12


def test_single_determinant_diagonal_matches_textbook_energy():
    """<D|H|D> = sum_occ h_ii + 1/2 sum_{occ a,b} [(aa|bb) - d(sa,sb) (ab|ba)]."""
    L = 5
    h, v = workloads.integrals(L, seed=6)
    H, D = fock.hamiltonian_dets(h, v, 2, 2)
    diag = H.diagonal()
    for k in range(0, D.size, 7):
        occ = [(m // 2, m % 2) for m in range(2 * L) if (int(D[k]) >> m) & 1]
        e = sum(h[i, i] for i, _ in occ)
        for i, si in occ:
            for j, sj in occ:
                e += 0.5 * v[i, i, j, j] - (0.5 * v[i, j, j, i] if si == sj else 0.0)
        assert abs(diag[k] - e) < 1e-12


def test_two_electron_first_quantized_rewrite():
    """One up + one dn electron: H = h(x)1 + 1(x)h + V with V[(k,l),(i,j)] = (ki|lj) in first quantization."""
    L = 4
    h, v = workloads.integrals(L, seed=7)
    I = np.eye(L)
    H1 = np.kron(h, I) + np.kron(I, h) + np.einsum("kilj->klij", v).reshape(L * L, L * L)
    e_first = np.linalg.eigvalsh(H1)
    H, _ = fock.hamiltonian_dets(h, v, 1, 1)
    e_second = np.linalg.eigvalsh(H.toarray())
    assert np.allclose(np.sort(e_first), np.sort(e_second), atol=1e-11)


def test_two_up_electrons_antisymmetric_first_quantized():
    L = 4
    h, v = workloads.integrals(L, seed=8)
    I = np.eye(L)
    H1 = np.kron(h, I) + np.kron(I, h) + np.einsum("kilj->klij", v).reshape(L * L, L * L)
    # antisymmetric subspace basis (i<j): (|ij> - |ji>)/sqrt2
    cols = []
    for i in range(L):
        for j in range(i + 1, L):
            x = np.zeros(L * L)
            x[i * L + j] = 1 / np.sqrt(2)
            x[j * L + i] = -1 / np.sqrt(2)
            cols.append(x)
    A = np.array(cols).T
    e_first = np.linalg.eigvalsh(A.T @ H1 @ A)
    H, _ = fock.hamiltonian_dets(h, v, 2, 0)
    assert np.allclose(np.sort(e_first), np.linalg.eigvalsh(H.toarray()), atol=1e-11)


def test_spin_multiplets_shared_between_sz_sectors():
    """SU(2): every S>=1 level of the Sz=1 sector appears in the Sz=0 sector of the same N."""
    L = 4
    h, v = workloads.integrals(L, seed=9)
    H0, _ = fock.hamiltonian_dets(h, v, 2, 2)
    H1, _ = fock.hamiltonian_dets(h, v, 3, 1)
    e0 = np.linalg.eigvalsh(H0.toarray())
    e1 = np.linalg.eigvalsh(H1.toarray())
    for e in e1:
        assert np.min(np.abs(e0 - e)) < 1e-10


def test_linear_scaling_and_hermiticity():
    L = 5
    h, v = workloads.integrals(L, seed=10)
    H, _ = fock.hamiltonian_dets(h, v, 3, 2)
    A = H.toarray()
    assert np.allclose(A, A.T, atol=1e-14)
    E1 = _ground(h, v, 3, 2)
    E2 = _ground(2.5 * h, 2.5 * v, 3, 2)
    assert abs(E2 - 2.5 * E1) < 1e-11


def test_fock_and_determinant_constructions_agree():
    L = 3
    h, v = workloads.integrals(L, seed=11)
    Hf = fock.hamiltonian_fock(h, v, fock.fock_creation(L))
    Hd, D = fock.hamiltonian_dets(h, v, 2, 1)
    masks = fock.fock_to_mask(L)
    order = np.argsort(masks)
    pos = order[np.searchsorted(masks[order], D)]
    assert np.allclose(Hf.toarray()[np.ix_(pos, pos)], Hd.toarray(), atol=1e-13)


def test_lanczos_matches_dense():
    h, v = workloads.integrals(6, seed=12)
    H, _ = fock.hamiltonian_dets(h, v, 3, 3)
    e, x = fock.lanczos_ground(lambda y: H @ y, H.shape[0])
    assert abs(e - np.linalg.eigvalsh(H.toarray())[0]) < 1e-10
    assert np.linalg.norm(H @ x - e * x) < 1e-6


# ---------------------------------------------------------------- explicit block bases (O2)

def _complete_blocks(L, k):
    """Left block of sites 0..k-1 and right block of k+2..L-1 with complete (identity-like) bases."""
    lb = ob.empty_block()
    for s in range(k):
        lay = ob.enlarged_left(lb)
        O = {E: np.eye(n) for E, n in ob.enlarged_dims(lay).items()}
        lb = ob.grow_left(lb, s, O)
    rb = ob.empty_block()
    for s in range(L - 1, k + 1, -1):
        lay = ob.enlarged_right(rb)
        O = {E: np.eye(n) for E, n in ob.enlarged_dims(lay).items()}
        rb = ob.grow_right(rb, s, O)
    return lb, rb


def test_complete_projection_reproduces_fci_spectrum():
    L = 5
    h, v = workloads.integrals(L, seed=13)
    lb, rb = _complete_blocks(L, 1)
    P = ob.Projected(h, v, lb, rb, 3, 2)
    assert P.dim == P.H.shape[0]
    assert np.allclose(P.V.T @ P.V, np.eye(P.dim), atol=1e-13)
    assert np.allclose(np.linalg.eigvalsh(P.dense()), np.linalg.eigvalsh(P.H.toarray()), atol=1e-11)


def test_truncated_projection_is_variational():
    L = 6
    h, v = workloads.integrals(L, seed=14)
    rng = np.random.default_rng(1)
    lb = ob.empty_block()
    for s in range(2):
        lay = ob.enlarged_left(lb)
        O = {E: workloads.orthonormal_columns(n, max(1, n // 2), rng)
             for E, n in ob.enlarged_dims(lay).items()}
        lb = ob.grow_left(lb, s, O)
    rb = ob.empty_block()
    for s in (5, 4):
        lay = ob.enlarged_right(rb)
        O = {E: workloads.orthonormal_columns(n, max(1, n // 2), rng)
             for E, n in ob.enlarged_dims(lay).items()}
        rb = ob.grow_right(rb, s, O)
    P = ob.Projected(h, v, lb, rb, 3, 3)
    assert np.allclose(P.V.T @ P.V, np.eye(P.dim), atol=1e-12)
    e = P.ground()[0]
    assert e >= _ground(h, v, 3, 3) - 1e-12


def test_rdm_left_right_spectra_agree_and_trace_one():
    L = 6
    h, v = workloads.integrals(L, seed=15)
    lb, rb = _complete_blocks(L, 2)
    P = ob.Projected(h, v, lb, rb, 3, 3)
    e, psi = P.ground()
    rl, _ = ob.rdm_blocks(psi, lb, rb, 3, 3, +1)
    rr, _ = ob.rdm_blocks(psi, lb, rb, 3, 3, -1)
    evl = np.sort(np.concatenate([np.linalg.eigvalsh(R) for R in rl.values()]))
    evr = np.sort(np.concatenate([np.linalg.eigvalsh(R) for R in rr.values()]))
    assert abs(evl.sum() - 1) < 1e-12 and abs(evr.sum() - 1) < 1e-12
    nz = lambda x: np.sort(x[x > 1e-12])
    assert np.allclose(nz(evl), nz(evr), atol=1e-12)
    # Schmidt: the rho^L spectrum is the squared singular values of psi as (l s_l) x (s_r r)
    O, kept, dw, _ = ob.truncate(rl, 10)
    assert sum(kept) == 10
    assert abs(dw - (1 - np.sort(evl)[::-1][:10].sum())) < 1e-12


def test_renormalized_product_equals_product_on_complete_basis():
    L = 4
    h, v = workloads.integrals(L, seed=16)
    lb, _ = _complete_blocks(L, 2)
    A = ob.block_fock_operator(lb, "C", (1,), h, v)
    B = ob.block_fock_operator(lb, "C", (2,), h, v)
    AB = ob.block_fock_operator(lb, "A", (1, 2), h, v)
    rA, rB, rAB = ob.renormalized(lb, A), ob.renormalized(lb, B), ob.renormalized(lb, AB)
    for (kb, ka), blk in rAB.items():
        mid = (ka[0] + 1, ka[1])  # mode 2 is site 1 up: B raises n_up first
        prod = rA[(kb, mid)] @ rB[(mid, ka)]
        assert np.allclose(prod, blk, atol=1e-13)


def test_truncation_rule_on_a_known_spectrum():
    """Reading of "keep the M largest eigenvalues": global order, ties by (sector
    order, in-sector order), eigenvalues <= 1e-13 never kept, a near-degenerate
    cluster across the cut is cut as a whole unless nothing would remain,
    discarded weight = trace - kept.  Checked on density matrices with known
    eigenpairs."""
    import numpy as np
    from oracle import blocks as ob
    rng = np.random.default_rng(5)

    # diagonal density matrices: eigenvalues exact, so the ties below are exact ties
    spectra = {(0, 0): [0.30, 0.05, 1e-14], (0, 1): [0.20, 0.05], (1, 0): [0.30, 0.10, 0.0]}
    rho = {E: np.diag(ev) for E, ev in spectra.items()}
    # M = 4: 0.30 (sector 0), 0.30 (sector 2: later sector), 0.20, 0.10 -> the two 0.05 are cut
    O, kept, dw, _ = ob.truncate(rho, 4)
    assert kept == [1, 1, 2]
    trace = sum(sum(ev) for ev in spectra.values())
    assert abs(dw - (trace - 0.90)) < 1e-12
    # M = 5: the two 0.05 straddle the cut, so both are cut (the 4 above remain)
    O, kept, dw, _ = ob.truncate(rho, 5)
    assert kept == [1, 1, 2]
    assert abs(dw - (trace - 0.90)) < 1e-12
    # M = 1: the top cluster (0.30 twice) holds more than M: the cut stays at M and
    # the tie goes to the earlier sector
    O, kept, dw, _ = ob.truncate(rho, 1)
    assert kept == [1, 0, 0]
    # near-equal (within 1e-10) is one cluster too; 1e-9 apart is not
    near = {(0, 0): np.diag([0.4, 0.2 + 5e-11]), (1, 0): np.diag([0.2])}
    assert ob.truncate(near, 2)[1] == [1, 0]
    apart = {(0, 0): np.diag([0.4, 0.2 + 1e-9]), (1, 0): np.diag([0.2])}
    assert ob.truncate(apart, 2)[1] == [2, 0]
    # M large: 1e-14 and 0.0 are never kept
    O, kept, dw, _ = ob.truncate(rho, 100)
    assert kept == [2, 2, 2]
    assert abs(dw - 1e-14) < 1e-12
    # rotated density matrices (distinct eigenvalues): the kept columns span the
    # eigenvectors of the kept eigenvalues
    spectra = {(0, 0): [0.40, 0.06, 0.01], (1, 1): [0.35, 0.12, 0.06]}
    rho, vecs = {}, {}
    for E, ev in spectra.items():
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        rho[E], vecs[E] = (Q * np.asarray(ev)) @ Q.T, Q
    O, kept, dw, _ = ob.truncate(rho, 3)
    assert kept == [1, 2]
    for (E, ev), k in zip(spectra.items(), kept):
        order = np.argsort(ev)[::-1][:k]
        assert np.allclose(O[E] @ O[E].T, vecs[E][:, order] @ vecs[E][:, order].T, atol=1e-10)
    assert abs(dw - (0.06 + 0.01 + 0.06)) < 1e-12
