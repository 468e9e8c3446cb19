"""The normal/complementary operator identities (Sec. 2.1, pre-summed operators), on explicit Fock spaces.

Both the CUDA host planner and the oracle DMRG rely on one decomposition of
Eq. H2q over two consecutive groups of orbitals X (first in Jordan-Wigner
order) and Y:

  H^{XY} = H^X + H^Y + sum_{j in Y} (T^X_j c_j + h.c.) + sum_{i in X} (c+_i V^Y_i + h.c.)
         + sum_{p<q in X} (A_pq Pa^Y_pq + h.c.) + sum_{p,s in X} B_ps Q^Y_ps
         = ... + sum_{r<s in Y} (Pc^X_rs (c_s c_r) + h.c.) + sum_{q,r in Y} Q^X_qr c+_q c_r

and on the blocking rules for the complementary operators T, V, Pc, Pa, Q.
Each identity is checked here as an equality of sparse matrices on the Fock
space of X u Y, where operator products carry their Jordan-Wigner strings.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fock
from oracle.blocks import fock_op
from paper_2001_04890_gb300 import workloads

LINT = 6
X = [1, 2]
Y = [3, 4]
XY = X + Y
OUT = [0, 5]


@pytest.fixture(scope="module")
def setup():
    h, v = workloads.integrals(LINT, seed=21)
    t, w = fock.spin_orbital_integrals(h, v)
    cache = {}
    op = lambda kind, idx, sub: fock_op(kind, idx, sub, XY, h, v, cache)
    return h, v, t, w, op


def modes(sites):
    return [2 * s + sg for s in sites for sg in range(2)]


def close(A, B):
    d = (A - B)
    d = d.toarray() if sp.issparse(d) else d
    return np.max(np.abs(d)) < 1e-12


def test_bipartition_of_hamiltonian_normal_on_x(setup):
    h, v, t, w, op = setup
    H = op("H", None, XY)
    Z = op("H", None, X) + op("H", None, Y)
    for j in modes(Y):
        term = op("T", (j,), X) @ op("C", (j,), Y).T
        Z = Z + term + term.T
    for i in modes(X):
        term = op("C", (i,), X) @ op("V", (i,), Y)
        Z = Z + term + term.T
    for p in modes(X):
        for q in modes(X):
            if p < q:
                term = op("A", (p, q), X) @ op("Pa", (p, q), Y)
                Z = Z + term + term.T
            term = op("B", (p, q), X) @ op("Q", (p, q), Y)
            Z = Z + term
    assert close(H, Z)


def test_bipartition_of_hamiltonian_complementary_on_x(setup):
    h, v, t, w, op = setup
    H = op("H", None, XY)
    Z = op("H", None, X) + op("H", None, Y)
    for j in modes(Y):
        term = op("T", (j,), X) @ op("C", (j,), Y).T
        Z = Z + term + term.T
    for i in modes(X):
        term = op("C", (i,), X) @ op("V", (i,), Y)
        Z = Z + term + term.T
    for r in modes(Y):
        for s in modes(Y):
            if r < s:
                term = op("Pc", (r, s), X) @ op("A", (r, s), Y).T
                Z = Z + term + term.T
            Z = Z + op("Q", (r, s), X) @ op("B", (r, s), Y)
    assert close(H, Z)


@pytest.mark.parametrize("j", [0, 1, 10, 11])
def test_blocking_of_T(setup, j):
    h, v, t, w, op = setup
    lhs = op("T", (j,), XY)
    Z = op("T", (j,), X) + op("T", (j,), Y)
    for r in modes(Y):
        Z = Z - op("Pc", (r, j), X) @ op("C", (r,), Y).T
    for q in modes(Y):
        Z = Z + op("Q", (q, j), X) @ op("C", (q,), Y)
    for p in modes(X):
        Z = Z + op("C", (p,), X) @ op("Q", (p, j), Y)
    for r in modes(X):
        Z = Z - op("C", (r,), X).T @ op("Pc", (r, j), Y)
    assert close(lhs, Z)


@pytest.mark.parametrize("i", [0, 1, 10, 11])
def test_blocking_of_V(setup, i):
    h, v, t, w, op = setup
    lhs = op("V", (i,), XY)
    Z = op("V", (i,), X) + op("V", (i,), Y)
    for q in modes(X):
        Z = Z + op("C", (q,), X) @ op("Pa", (i, q), Y)
    for q in modes(Y):
        Z = Z + op("Pa", (i, q), X) @ op("C", (q,), Y)
    for q in modes(X):
        for s in modes(X):
            R = sp.csr_matrix(lhs.shape)
            for r in modes(Y):
                coef = w[i, q, r, s] - w[i, q, s, r]
                if coef != 0.0:
                    R = R + coef * op("C", (r,), Y).T
            Z = Z + op("B", (q, s), X) @ R
    for s in modes(X):
        Z = Z + op("C", (s,), X).T @ op("Q", (i, s), Y)
    assert close(lhs, Z)


@pytest.mark.parametrize("pair", [(0, 1), (0, 10), (1, 11), (10, 11), (0, 2)])
def test_blocking_of_pair_complementaries(setup, pair):
    h, v, t, w, op = setup
    a, b = pair
    W = lambda p, q, r, s: w[p, q, r, s] - w[p, q, s, r]
    # creation pair Pc_{ab}
    Z = op("Pc", (a, b), X) + op("Pc", (a, b), Y)
    for p in modes(X):
        for q in modes(Y):
            Z = Z + W(p, q, a, b) * (op("C", (p,), X) @ op("C", (q,), Y))
    assert close(op("Pc", (a, b), XY), Z)
    # annihilation pair Pa_{ab}
    Z = op("Pa", (a, b), X) + op("Pa", (a, b), Y)
    for r in modes(X):
        for s in modes(Y):
            Z = Z + W(a, b, r, s) * (op("C", (s,), Y).T @ op("C", (r,), X).T)
    assert close(op("Pa", (a, b), XY), Z)
    # Q_{ab}
    Z = op("Q", (a, b), X) + op("Q", (a, b), Y)
    for q in modes(XY):
        for r in modes(XY):
            if (q in modes(X)) != (r in modes(X)):
                coef = w[a, q, b, r] - w[a, q, r, b]
                if coef != 0.0:
                    Z = Z + coef * (op("C", (q,), XY) @ op("C", (r,), XY).T)
    assert close(op("Q", (a, b), XY), Z)


def test_pair_complementaries_are_linear_in_normal_pairs(setup):
    """Pc^X_rs = sum_{p<q} W_pqrs A_pq and Q^X_qr = sum_{p,s} (w_pqsr - w_pqrs) B_ps (holds after any projection)."""
    h, v, t, w, op = setup
    for r, s in [(0, 1), (1, 10), (0, 11)]:
        Z = sp.csr_matrix((4 ** 4, 4 ** 4))
        for p in modes(X):
            for q in modes(X):
                if p < q:
                    Z = Z + (w[p, q, r, s] - w[p, q, s, r]) * op("A", (p, q), X)
        assert close(op("Pc", (r, s), X), Z)
        Z = sp.csr_matrix((4 ** 4, 4 ** 4))
        for p in modes(X):
            for q in modes(X):
                Z = Z + (w[p, r, q, s] - w[p, r, s, q]) * op("B", (p, q), X)
        assert close(op("Q", (r, s), X), Z)
