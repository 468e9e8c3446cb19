"""FP64 CPU oracle, part 1: Fock space, determinants and full CI.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use it.
It shares no code with the CUDA path.

Conventions (the paper's Sec. 2.1; readings where it is silent or garbled):
  * Hamiltonian, Eq. H2q, read in spin-orbital form as
        H = sum_pq t_pq c+_p c_q + 1/2 sum_pqrs w_pqrs c+_p c+_q c_s c_r,
    t_pq = h_ij d(sp,sq), w_pqrs = <pq|rs> = (ik|jl) d(sp,sr) d(sq,ss) for
    p=(i,sp), q=(j,sq), r=(k,sr), s=(l,ss), with v the chemists' integrals
    (ik|jl).  No core energy.  The 1/2 is fixed by the Hubbard-dimer pin.
  * Site basis of Eq. creation_ops taken in the stated order {0, up, dn, updn}
    with |updn> = a+_up a+_dn |0>: a+_up maps 0->up and dn->updn (+1), a+_dn
    maps 0->dn (+1) and up->updn (-1).  (As printed, the two matrices hold
    for the order {0, dn, up, updn}; energies do not depend on the choice.)
  * Jordan-Wigner order: lattice order of the sites; on a site, up before dn.
    Spin-orbital (mode) number m = 2 i + s, s = 0 for up, 1 for dn.
  * A Fock state of n sites is indexed site-major in base 4: the index is
    sum_i s_i 4^(n-1-i) with s_i in {0,1,2,3} the site state above, so the
    state of a block followed by a site is the Kronecker product.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# site state -> (n_up, n_dn)
SITE_NUP = np.array([0, 1, 0, 1])
SITE_NDN = np.array([0, 0, 1, 1])


def site_ops():
    """4x4 site creation operators a+_up, a+_dn and the site parity (Eq. creation_ops)."""
    cu = np.zeros((4, 4))
    cu[1, 0] = 1.0
    cu[3, 2] = 1.0
    cd = np.zeros((4, 4))
    cd[2, 0] = 1.0
    cd[3, 1] = -1.0
    par = np.diag([1.0, -1.0, -1.0, 1.0])
    return cu, cd, par


# --------------------------------------------------------------------------
# Fock space of n sites (small n): sparse Jordan-Wigner operators
# --------------------------------------------------------------------------

def fock_creation(n_sites: int):
    """Sparse c+_m for the 2 n modes of an n-site Fock space (dimension 4^n)."""
    cu, cd, par = site_ops()
    I4 = sp.identity(4, format="csr")
    P = sp.csr_matrix(par)
    out = []
    for i in range(n_sites):
        for local in (cu, cd):
            m = sp.identity(1, format="csr")
            for j in range(n_sites):
                if j < i:
                    f = P
                elif j == i:
                    f = sp.csr_matrix(local)
                else:
                    f = I4
                m = sp.kron(m, f, format="csr")
            out.append(m)
    return out


def fock_numbers(n_sites: int):
    """(n_up, n_dn) of every Fock index of an n-site space."""
    nu = np.zeros(4 ** n_sites, dtype=np.int64)
    nd = np.zeros(4 ** n_sites, dtype=np.int64)
    idx = np.arange(4 ** n_sites)
    for i in range(n_sites):
        s = (idx // 4 ** (n_sites - 1 - i)) % 4
        nu += SITE_NUP[s]
        nd += SITE_NDN[s]
    return nu, nd


def fock_to_mask(n_sites: int):
    """Occupation bitmask (bit m = mode m) of every Fock index of an n-site space."""
    idx = np.arange(4 ** n_sites)
    mask = np.zeros(4 ** n_sites, dtype=np.int64)
    for i in range(n_sites):
        s = (idx // 4 ** (n_sites - 1 - i)) % 4
        mask |= (s & 1).astype(np.int64) << (2 * i)
        mask |= ((s >> 1) & 1).astype(np.int64) << (2 * i + 1)
    return mask


# --------------------------------------------------------------------------
# spin-orbital integrals
# --------------------------------------------------------------------------

def spin_orbital_integrals(h: np.ndarray, v: np.ndarray):
    """t (2L x 2L) and w = <pq|rs> ((2L)^4) from spatial h and chemists' v."""
    L = h.shape[0]
    n = 2 * L
    t = np.zeros((n, n))
    w = np.zeros((n, n, n, n))
    for s in range(2):
        t[s::2, s::2] = h
    for sp_ in range(2):
        for sq in range(2):
            # w[p,q,r,s] = v[i,k,j,l] for spins (sp_, sq, sp_, sq)
            w[sp_::2, sq::2, sp_::2, sq::2] = np.transpose(v, (0, 2, 1, 3))
    return t, w


def hamiltonian_fock(h, v, cdag):
    """Literal second-quantized H (Eq. H2q) as a sparse matrix over a small Fock space.

    cdag are the creation operators of the space (fock_creation); the integrals
    must be those of exactly these modes.
    """
    t, w = spin_orbital_integrals(h, v)
    n = len(cdag)
    c = [m.T.tocsr() for m in cdag]
    dim = cdag[0].shape[0]
    H = sp.csr_matrix((dim, dim))
    for p in range(n):
        for q in range(n):
            if t[p, q] != 0.0:
                H = H + t[p, q] * (cdag[p] @ c[q])
    for p in range(n):
        for q in range(n):
            if p == q:
                continue
            cc = cdag[p] @ cdag[q]
            for r in range(n):
                for s in range(n):
                    if r == s or w[p, q, r, s] == 0.0:
                        continue
                    H = H + 0.5 * w[p, q, r, s] * (cc @ (c[s] @ c[r]))
    return H.tocsr()


# --------------------------------------------------------------------------
# determinant basis of one (N_up, N_dn) sector (full CI)
# --------------------------------------------------------------------------

def popcount(x: np.ndarray) -> np.ndarray:
    return np.bitwise_count(x.astype(np.uint64)).astype(np.int64)


def determinants(L: int, n_up: int, n_dn: int) -> np.ndarray:
    """All occupation bitmasks over 2L modes with the given numbers of up and dn electrons, ascending."""
    from itertools import combinations
    ups = [sum(1 << (2 * i) for i in c) for c in combinations(range(L), n_up)]
    dns = [sum(1 << (2 * i + 1) for i in c) for c in combinations(range(L), n_dn)]
    d = np.array(sorted(u | dd for u in ups for dd in dns), dtype=np.int64)
    return d


def _annihilate(D, sign, ok, m):
    bit = np.int64(1) << m
    has = (D & bit) != 0
    ok = ok & has
    below = popcount(D & (bit - 1))
    sign = sign * np.where(below % 2 == 1, -1.0, 1.0)
    return D & ~bit, sign, ok


def _create(D, sign, ok, m):
    bit = np.int64(1) << m
    has = (D & bit) != 0
    ok = ok & ~has
    below = popcount(D & (bit - 1))
    sign = sign * np.where(below % 2 == 1, -1.0, 1.0)
    return D | bit, sign, ok


def apply_string(D: np.ndarray, ops):
    """Apply a product of mode operators to all determinants D.

    ops is the operator string written left to right as in the formula, each
    item (mode, is_creation); it acts right to left.  Returns (D', sign, ok).
    """
    sign = np.ones(D.shape[0])
    ok = np.ones(D.shape[0], dtype=bool)
    cur = D.copy()
    for m, is_cr in reversed(ops):
        if is_cr:
            cur, sign, ok = _create(cur, sign, ok, m)
        else:
            cur, sign, ok = _annihilate(cur, sign, ok, m)
    return cur, sign, ok


def hamiltonian_dets(h: np.ndarray, v: np.ndarray, n_up: int, n_dn: int):
    """Literal second-quantized H (Eq. H2q) in the determinant basis of one sector (sparse CSR)."""
    L = h.shape[0]
    D = determinants(L, n_up, n_dn)
    t, w = spin_orbital_integrals(h, v)
    n = 2 * L
    rows, cols, vals = [], [], []
    col_idx = np.arange(D.shape[0])

    def emit(coef, ops):
        Dp, sg, ok = apply_string(D, ops)
        if not ok.any():
            return
        Dp, sg, cidx = Dp[ok], sg[ok], col_idx[ok]
        ridx = np.searchsorted(D, Dp)
        rows.append(ridx)
        cols.append(cidx)
        vals.append(coef * sg)

    for p in range(n):
        for q in range(n):
            if t[p, q] != 0.0:
                emit(t[p, q], [(p, True), (q, False)])
    for p in range(n):
        for q in range(n):
            if p == q:
                continue
            for r in range(n):
                for s in range(n):
                    if r == s or w[p, q, r, s] == 0.0:
                        continue
                    emit(0.5 * w[p, q, r, s], [(p, True), (q, True), (s, False), (r, False)])
    dim = D.shape[0]
    if rows:
        H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(dim, dim)).tocsr()
    else:
        H = sp.csr_matrix((dim, dim))
    H.sum_duplicates()
    return H, D


def lanczos_ground(matvec, dim: int, tol: float = 1e-12, max_iter: int = 500, seed: int = 0):
    """Lowest eigenpair by Lanczos with full reorthogonalisation (plain textbook form)."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(dim)
    q /= np.linalg.norm(q)
    Q = [q]
    alphas, betas = [], []
    theta, y = None, None
    for it in range(min(max_iter, dim)):
        wv = matvec(Q[-1])
        a = float(Q[-1] @ wv)
        alphas.append(a)
        wv = wv - a * Q[-1] - (betas[-1] * Q[-2] if betas else 0.0)
        Qm = np.array(Q)
        for _ in range(2):
            wv = wv - Qm.T @ (Qm @ wv)
        b = float(np.linalg.norm(wv))
        T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        ev, evec = np.linalg.eigh(T)
        theta, y = ev[0], evec[:, 0]
        resid = b * abs(y[-1])
        if resid < tol or b < 1e-14 or it + 1 == dim:
            break
        betas.append(b)
        Q.append(wv / b)
    x = np.array(Q[: len(y)]).T @ y
    x /= np.linalg.norm(x)
    return float(theta), x


def fci_ground(h: np.ndarray, v: np.ndarray, n_up: int, n_dn: int, dense_max: int = 6000):
    """Exact ground-state energy in the (n_up, n_dn) sector: dense eigh if small, else Lanczos."""
    H, D = hamiltonian_dets(h, v, n_up, n_dn)
    dim = H.shape[0]
    if dim <= dense_max:
        ev, evec = np.linalg.eigh(H.toarray())
        return float(ev[0]), evec[:, 0], D
    e, x = lanczos_ground(lambda y: H @ y, dim)
    return e, x, D


# --------------------------------------------------------------------------
# orbital reduced density matrices and entropies (post-processing of a state)
# --------------------------------------------------------------------------

def pair_rdm_dets(x: np.ndarray, D: np.ndarray, i: int) -> np.ndarray:
    """Two-orbital reduced density matrix of sites i and i+1 of the state sum_D x_D |D>.

    Indexed by 4 b + c with b, c the site states (0, up, dn, updn) of sites i
    and i+1.  The four modes of the pair are consecutive in the Jordan-Wigner
    order, and elements only connect pair states of equal particle number, so
    the pair factors out of every determinant with a sign that cancels:
    rho[(b c), (b' c')] = sum over the other modes' occupations of
    x(b c, rest) x(b' c', rest).
    """
    local = (D >> (2 * i)) & 0xF
    b = (local & 1) + 2 * ((local >> 1) & 1)
    c = ((local >> 2) & 1) + 2 * ((local >> 3) & 1)
    pair = (4 * b + c).astype(np.int64)
    rest = D & ~(np.int64(0xF) << (2 * i))
    rho = np.zeros((16, 16))
    order = np.argsort(rest, kind="stable")
    rs, ps, xs = rest[order], pair[order], x[order]
    start = 0
    while start < len(rs):
        end = start
        while end < len(rs) and rs[end] == rs[start]:
            end += 1
        v = np.zeros(16)
        v[ps[start:end]] = xs[start:end]
        rho += np.outer(v, v)
        start = end
    return rho


def pair_rdm_dets_ij(x: np.ndarray, D: np.ndarray, i: int, j: int) -> np.ndarray:
    """Two-orbital reduced density matrix of orbitals i < j (not necessarily
    adjacent) of the state sum_D x_D |D>, indexed by 4 b + c with b, c the site
    states of orbitals i and j (the matrix behind the mutual information the
    paper uses for the orbital ordering, Sec. 3).

    Moving the two modes of orbital j (in front of every mode between the two
    orbitals) next to those of orbital i reorders the Jordan-Wigner string:
    each determinant picks up (-1)^(n_j * n_between), n_j the electrons on
    orbital j and n_between those on the orbitals strictly between.  In that
    order the pair is adjacent, and rho[(b c), (b' c')] = sum over the other
    modes' occupations of the two reordered amplitudes (as pair_rdm_dets).
    """
    if not (0 <= i < j):
        raise ValueError("pair_rdm_dets_ij needs 0 <= i < j")
    li = (D >> (2 * i)) & 3
    lj = (D >> (2 * j)) & 3
    b = (li & 1) + 2 * ((li >> 1) & 1)
    c = (lj & 1) + 2 * ((lj >> 1) & 1)
    between = ((np.int64(1) << (2 * j)) - 1) & ~((np.int64(1) << (2 * i + 2)) - 1)
    n_between = popcount(D & between)
    n_j = popcount(lj)
    sign = np.where((n_j * n_between) % 2 == 1, -1.0, 1.0)
    pair = (4 * b + c).astype(np.int64)
    rest = D & ~(np.int64(3) << (2 * i)) & ~(np.int64(3) << (2 * j))
    rho = np.zeros((16, 16))
    order = np.argsort(rest, kind="stable")
    rs, ps, xs = rest[order], pair[order], (sign * x)[order]
    start = 0
    while start < len(rs):
        end = start
        while end < len(rs) and rs[end] == rs[start]:
            end += 1
        v = np.zeros(16)
        v[ps[start:end]] = xs[start:end]
        rho += np.outer(v, v)
        start = end
    return rho


def orbital_entropies(rho: np.ndarray):
    """(s_i, s_{i+1}, s_{i,i+1}): von Neumann entropies -tr(r ln r) of the
    trace-normalised one-orbital matrices (partial traces of the pair matrix)
    and of the pair matrix itself."""
    r = rho / np.trace(rho)
    h = lambda p: float(-sum(q * np.log(q) for q in p if q > 0.0))
    R = r.reshape(4, 4, 4, 4)
    wl = np.einsum("bcbc->b", R)
    wr = np.einsum("bcbc->c", R)
    return h(wl), h(wr), h(np.linalg.eigvalsh(r))
