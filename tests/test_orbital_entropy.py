"""One- and two-orbital entropies of a two-site wave function (the single-site
entropies and mutual information the paper uses for orbital ordering, Sec. 3).

The oracle (oracle/fock.py) forms the pair's reduced density matrix from a
determinant-basis vector; it is pinned to the Hubbard-dimer closed form, to
zero entropy for a single determinant, to the Schmidt symmetry of pure
two-site states and to subadditivity.  The library's host routine
(dmrg_debug_pair_rdm, the arithmetic behind dmrg_orbital_entropies) is then
compared with the oracle on block-basis wave functions mapped back to
determinants."""
import numpy as np
import pytest

from oracle import blocks as ob
from oracle import fock
from paper_2001_04890_gb300 import binding, workloads
from tests.helpers import random_O


@pytest.mark.parametrize("U", [0.0, 1.0, 3.0, 8.0])
def test_oracle_hubbard_dimer_entropy_closed_form(U):
    t = 1.0
    h, v = workloads.hubbard_dimer(t, U)
    e, x, D = fock.fci_ground(h, v, 1, 1)
    sl, sr, sp = fock.orbital_entropies(fock.pair_rdm_dets(x, D, 0))
    # singlet ground state a |cov> + b |ion>: site weights b^2/2 (empty, double), a^2/2 (up, dn)
    E = (U - np.sqrt(U * U + 16 * t * t)) / 2
    r2 = E * E / (4 * t * t)
    a2, b2 = 1 / (1 + r2), r2 / (1 + r2)
    s_ref = -a2 * np.log(a2 / 2) - b2 * np.log(b2 / 2)
    assert abs(e - E) < 1e-12
    assert abs(sl - s_ref) < 1e-12 and abs(sr - s_ref) < 1e-12
    assert abs(sp) < 1e-12   # the pair is the whole system: a pure state


def test_oracle_single_determinant_has_no_entropy():
    L, nu, nd = 5, 2, 3
    D = fock.determinants(L, nu, nd)
    x = np.zeros(len(D))
    x[7] = 1.0
    for i in range(L - 1):
        assert np.allclose(fock.orbital_entropies(fock.pair_rdm_dets(x, D, i)), 0.0, atol=1e-14)


def test_oracle_pair_matrix_labels_and_two_site_definition():
    # site 0 holds up, site 1 holds dn: the pair state (b, c) = (up, dn) = index 4*1 + 2
    D = fock.determinants(3, 1, 1)
    x = np.zeros(len(D))
    x[np.nonzero(D == ((1 << 0) | (1 << 3)))[0][0]] = 1.0
    rho = fock.pair_rdm_dets(x, D, 0)
    assert rho[6, 6] == 1.0 and np.count_nonzero(rho) == 1
    # two sites are the whole system: rho is the outer product of the state written over (b, c)
    rng = np.random.default_rng(3)
    D = fock.determinants(2, 1, 1)
    x = rng.normal(size=len(D))
    v = np.zeros(16)
    for d, c in zip(D, x):
        b0 = (d & 1) + 2 * ((d >> 1) & 1)
        b1 = ((d >> 2) & 1) + 2 * ((d >> 3) & 1)
        v[4 * b0 + b1] = c
    assert np.allclose(fock.pair_rdm_dets(x, D, 0), np.outer(v, v), atol=0, rtol=0)


def test_oracle_two_site_pure_state_and_subadditivity():
    rng = np.random.default_rng(5)
    D = fock.determinants(2, 1, 1)
    x = rng.normal(size=len(D))
    x /= np.linalg.norm(x)
    sl, sr, sp = fock.orbital_entropies(fock.pair_rdm_dets(x, D, 0))
    assert abs(sl - sr) < 1e-12 and abs(sp) < 1e-12   # Schmidt: equal spectra, pure pair
    D = fock.determinants(5, 3, 2)
    for _ in range(5):
        x = rng.normal(size=len(D))
        x /= np.linalg.norm(x)
        for i in range(4):
            sl, sr, sp = fock.orbital_entropies(fock.pair_rdm_dets(x, D, i))
            assert sl + sr - sp >= -1e-12            # mutual information >= 0
            assert sp >= abs(sl - sr) - 1e-12          # Araki-Lieb


def _bases(L, k, M, seed):
    rng = np.random.default_rng(seed)
    lb = ob.empty_block()
    for s in range(k):
        lay = ob.enlarged_left(lb)
        kept, blocks, _ = random_O([ob.enlarged_dims(lay)[E] for E in lay], M, rng)
        lb = ob.grow_left(lb, s, {E: b for E, b in zip(lay, blocks)})
    rb = ob.empty_block()
    for s in range(L - 1, k + 1, -1):
        lay = ob.enlarged_right(rb)
        kept, blocks, _ = random_O([ob.enlarged_dims(lay)[E] for E in lay], M, rng)
        rb = ob.grow_right(rb, s, {E: b for E, b in zip(lay, blocks)})
    return lb, rb


@pytest.mark.parametrize("L,N,two_sz,M,k", [(6, 6, 0, 16, 2), (6, 5, 1, 12, 1), (7, 7, 1, 20, 2), (5, 4, 0, 64, 0)])
def test_library_pair_rdm_equals_oracle(L, N, two_sz, M, k):
    nu, nd = (N + two_sz) // 2, (N - two_sz) // 2
    h, v = workloads.integrals(L, seed=3)
    lb, rb = _bases(L, k, M, seed=L + k)
    P = ob.Projected(h, v, lb, rb, nu, nd)
    layout = np.array(P.layout, dtype=np.int64)
    _, ground = P.ground()
    rng = np.random.default_rng(1)
    for psi in (ground, rng.normal(size=P.dim)):
        rho_lib, s_lib = binding.debug_pair_rdm(layout, psi)
        x = P.V @ psi   # the same state in the determinant basis
        rho_or = fock.pair_rdm_dets(x, P.D, k)
        assert np.max(np.abs(rho_lib - rho_or)) < 1e-12 * np.trace(rho_or)
        assert np.max(np.abs(np.array(s_lib) - np.array(fock.orbital_entropies(rho_or)))) < 1e-11


def test_library_pair_rdm_rejects_inconsistent_blocks():
    layout = np.array([[0, 1, 2, 0, 2, 2, 0], [0, 2, 1, 0, 1, 2, 4]])   # same (a, d), sizes 4 and 2
    with pytest.raises(binding.DMRGError):
        binding.debug_pair_rdm(layout, np.ones(6))
    with pytest.raises(binding.DMRGError):
        binding.debug_pair_rdm(np.array([[0, 4, 0, 0, 1, 1, 0]]), np.ones(1))


def test_basis_export_format_rebuilds_the_blocks():
    """Chained renormalization matrices in the dmrg_renormalize / dmrg_block_basis format
    rebuild the explicit block bases (the MPS tensors of the sites, Sec. 2.1)."""
    from tests.helpers import rebuild_blocks
    L, k, M = 7, 3, 10
    rng = np.random.default_rng(4)
    exports = {0: {}, 1: {}}
    lb = ob.empty_block()
    for s in range(k):
        lay = ob.enlarged_left(lb)
        kept, blocks, flat = random_O([ob.enlarged_dims(lay)[E] for E in lay], M, rng)
        exports[0][s + 1] = (kept, flat)
        lb = ob.grow_left(lb, s, {E: b for E, b in zip(lay, blocks)})
    rb = ob.empty_block()
    for j, s in enumerate(range(L - 1, k + 1, -1), start=1):
        lay = ob.enlarged_right(rb)
        kept, blocks, flat = random_O([ob.enlarged_dims(lay)[E] for E in lay], M, rng)
        exports[1][j] = (kept, flat)
        rb = ob.grow_right(rb, s, {E: b for E, b in zip(lay, blocks)})
    lb2 = rebuild_blocks(exports[0], L, 0, k)
    rb2 = rebuild_blocks(exports[1], L, 1, L - k - 2)
    for a, b in ((lb, lb2), (rb, rb2)):
        assert a.sectors == b.sectors and a.dims == b.dims
        for E in a.sectors:
            assert np.array_equal(a.V[E], b.V[E])


def _pair_operator(ops):
    """16 x 16 matrix of a mode-operator string on the pair space alone (modes 0, 1 =
    first orbital up, dn; 2, 3 = second orbital up, dn; index 4 b + c)."""
    D = np.arange(16, dtype=np.int64)
    D2, sign, ok = fock.apply_string(D, ops)
    M = np.zeros((16, 16))
    idx = lambda d: 4 * ((d & 1) + 2 * ((d >> 1) & 1)) + (((d >> 2) & 1) + 2 * ((d >> 3) & 1))  # noqa: E731
    for d, d2, sg, k in zip(D, D2, sign, ok):
        if k:
            M[idx(int(d2)), idx(int(d))] = sg
    return M


def test_oracle_nonadjacent_pair_matrix_reproduces_expectation_values():
    """For every orbital pair of a random L=5 state, tr(rho_ij O) equals <x|O|x> evaluated
    on the whole determinant basis (Jordan-Wigner strings across the orbitals between
    included) for hopping, pair-hopping and number operators between the two orbitals;
    adjacent pairs equal pair_rdm_dets."""
    rng = np.random.default_rng(11)
    L = 5
    D = fock.determinants(L, 3, 2)
    x = rng.normal(size=len(D))
    x /= np.linalg.norm(x)
    lookup = {int(d): k for k, d in enumerate(D)}

    def expect(ops):
        D2, sign, ok = fock.apply_string(D, ops)
        return sum(x[lookup[int(d2)]] * sg * x[k] for k, (d2, sg, o) in enumerate(zip(D2, sign, ok)) if o)

    for i in range(L):
        for j in range(i + 1, L):
            rho = fock.pair_rdm_dets_ij(x, D, i, j)
            assert abs(np.trace(rho) - 1.0) < 1e-12 and np.allclose(rho, rho.T, atol=1e-14)
            if j == i + 1:
                assert np.allclose(rho, fock.pair_rdm_dets(x, D, i), atol=1e-14)
            for ops_full, ops_pair in [
                ([(2 * i, True), (2 * j, False)], [(0, True), (2, False)]),          # c+_i,up c_j,up
                ([(2 * j + 1, True), (2 * i + 1, False)], [(3, True), (1, False)]),  # c+_j,dn c_i,dn
                ([(2 * i, True), (2 * i + 1, True), (2 * j + 1, False), (2 * j, False)],
                 [(0, True), (1, True), (3, False), (2, False)]),                    # pair hopping
                ([(2 * i, True), (2 * i, False), (2 * j + 1, True), (2 * j + 1, False)],
                 [(0, True), (0, False), (3, True), (3, False)]),                    # n_i,up n_j,dn
                ([(2 * i + 1, True), (2 * j, True), (2 * j + 1, False), (2 * i, False)],
                 [(1, True), (2, True), (3, False), (0, False)]),                    # spin exchange
            ]:
                want = expect(ops_full)
                got = np.trace(rho @ _pair_operator(ops_pair))
                assert abs(got - want) < 1e-12, (i, j, ops_full, got, want)
