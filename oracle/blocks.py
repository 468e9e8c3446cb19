"""FP64 CPU oracle, part 2: explicit block bases, projected Hamiltonian, RDM truncation.

TEST INFRASTRUCTURE ONLY (see oracle/fock.py).

Everything here is the plain definition written out on explicit Fock-space
vectors, so it needs no operator algebra:
  * a block basis state is a vector in the block's own Fock space, grown one
    site at a time by the renormalization matrix of Eq. renorm,
        |l_p> = sum_{l_{p-1}, s} O_{l_{p-1} s, l_p} |l_{p-1}> (x) |s>;
  * the superblock basis |l>|s_l>|s_r>|r> of Eq. wf / wf_sec is the Kronecker
    product of those vectors, restricted to the (N_up, N_dn) sector;
  * H.psi of Eqs. h_mat / dgemm is V^T H V psi with H the full-CI Hamiltonian;
  * a renormalized operator (Eq. renorm_mat) is V^T A V with A the operator
    on the block's Fock space;
  * the density matrices of Sec. 2.1 are rho^L = psi psi^T and rho^R = psi^T psi,
    and the kept basis is the M eigenvectors with the largest eigenvalues.

Layout conventions (shared with the C ABI, implemented independently there):
  * block sectors (n_up, n_dn) sorted ascending;
  * enlarged left block l (x) s: sub-blocks (a, b) ordered by (a, b) inside
    each enlarged sector; enlarged right block s (x) r: sub-blocks (c, d)
    ordered by (c, d);
  * psi blocks (a, b, c, d) ordered lexicographically, each m_a x m_d row-major.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fock

TRUNC_DROP = 1e-13
TRUNC_CLUSTER = 1e-10  # eigenvalues closer than this are one near-degenerate cluster


class Block:
    """A block of consecutive sites with an explicit basis.

    sites: global site indices, ascending.  sectors: sorted list of (n_up, n_dn).
    V[sector]: (4^k, m) array, the basis vectors in the block's own Fock space.
    """

    def __init__(self, sites, V):
        self.sites = list(sites)
        self.V = {key: np.asarray(val) for key, val in V.items() if val.shape[1] > 0}
        self.sectors = sorted(self.V)

    @property
    def dims(self):
        return [self.V[s].shape[1] for s in self.sectors]

    def sector_index(self, key):
        return self.sectors.index(key)


def empty_block():
    return Block([], {(0, 0): np.ones((1, 1))})


def enlarged_left(block: Block):
    """Enlarged sectors of block (x) site: {E: [(a_idx, b, row_offset, m_a), ...]}, sorted by E."""
    groups = {}
    for ai, a in enumerate(block.sectors):
        for b in range(4):
            E = (a[0] + int(fock.SITE_NUP[b]), a[1] + int(fock.SITE_NDN[b]))
            groups.setdefault(E, []).append((ai, b))
    out = {}
    for E in sorted(groups):
        off = 0
        subs = []
        for ai, b in sorted(groups[E]):
            m = block.dims[ai]
            subs.append((ai, b, off, m))
            off += m
        out[E] = subs
    return out


def enlarged_right(block: Block):
    """Enlarged sectors of site (x) block: {E: [(c, d_idx, row_offset, m_d), ...]}, sorted by E."""
    groups = {}
    for di, d in enumerate(block.sectors):
        for c in range(4):
            E = (d[0] + int(fock.SITE_NUP[c]), d[1] + int(fock.SITE_NDN[c]))
            groups.setdefault(E, []).append((c, di))
    out = {}
    for E in sorted(groups):
        off = 0
        subs = []
        for c, di in sorted(groups[E]):
            m = block.dims[di]
            subs.append((c, di, off, m))
            off += m
        out[E] = subs
    return out


def enlarged_dims(layout):
    return {E: sum(s[3] for s in subs) for E, subs in layout.items()}


def split_O(layout, kept, O_flat):
    """Cut a flat renormalization matrix (concatenated row-major per enlarged sector) into blocks."""
    out = {}
    pos = 0
    dims = enlarged_dims(layout)
    for ei, E in enumerate(layout):
        n, m = dims[E], int(kept[ei])
        out[E] = np.asarray(O_flat[pos:pos + n * m]).reshape(n, m)
        pos += n * m
    assert pos == len(O_flat)
    return out


def grow_left(block: Block, site: int, O: dict):
    """New left block block + site with basis (Eq. renorm) given per-enlarged-sector O blocks."""
    layout = enlarged_left(block)
    V = {}
    for E, subs in layout.items():
        OE = O.get(E)
        if OE is None or OE.shape[1] == 0:
            continue
        cols = []
        for ai, b, off, m in subs:
            e = np.zeros((4, 1))
            e[b, 0] = 1.0
            cols.append((np.kron(block.V[block.sectors[ai]], e), off, m))
        dimF = 4 ** (len(block.sites) + 1)
        VE = np.zeros((dimF, OE.shape[1]))
        for Vab, off, m in cols:
            VE += Vab @ OE[off:off + m]
        V[E] = VE
    return Block(block.sites + [site], V)


def grow_right(block: Block, site: int, O: dict):
    """New right block site + block with basis given per-enlarged-sector O blocks."""
    layout = enlarged_right(block)
    V = {}
    for E, subs in layout.items():
        OE = O.get(E)
        if OE is None or OE.shape[1] == 0:
            continue
        dimF = 4 ** (len(block.sites) + 1)
        VE = np.zeros((dimF, OE.shape[1]))
        for c, di, off, m in subs:
            e = np.zeros((4, 1))
            e[c, 0] = 1.0
            VE += np.kron(e, block.V[block.sectors[di]]) @ OE[off:off + m]
        V[E] = VE
    return Block([site] + block.sites, V)


def psi_layout(lb: Block, rb: Block, n_up: int, n_dn: int):
    """Allowed psi blocks (a, b, c, d, m_a, m_d, offset) of Eq. wf_sec, lexicographic order."""
    out = []
    off = 0
    for ai, a in enumerate(lb.sectors):
        for b in range(4):
            for c in range(4):
                for di, d in enumerate(rb.sectors):
                    nu = a[0] + fock.SITE_NUP[b] + fock.SITE_NUP[c] + d[0]
                    nd = a[1] + fock.SITE_NDN[b] + fock.SITE_NDN[c] + d[1]
                    if nu == n_up and nd == n_dn:
                        ma, md = lb.dims[ai], rb.dims[di]
                        out.append((ai, b, c, di, ma, md, off))
                        off += ma * md
    return out, off


def superblock_V(lb: Block, rb: Block, L: int, n_up: int, n_dn: int, D: np.ndarray):
    """Columns = superblock basis states (psi layout order) in the determinant basis D."""
    layout, dim = psi_layout(lb, rb, n_up, n_dn)
    kl, kr = len(lb.sites), len(rb.sites)
    assert kl + kr + 2 == L
    mask_l = fock.fock_to_mask(kl)
    mask_r = fock.fock_to_mask(kr)
    nul, ndl = fock.fock_numbers(kl)
    nur, ndr = fock.fock_numbers(kr)
    V = np.zeros((D.shape[0], dim))
    for ai, b, c, di, ma, md, off in layout:
        a, d = lb.sectors[ai], rb.sectors[di]
        Sa = np.nonzero((nul == a[0]) & (ndl == a[1]))[0]
        Sd = np.nonzero((nur == d[0]) & (ndr == d[1]))[0]
        Vl = lb.V[a][Sa]
        Vr = rb.V[d][Sd]
        mid = (np.int64(fock.SITE_NUP[b]) << (2 * kl)) | (np.int64(fock.SITE_NDN[b]) << (2 * kl + 1)) \
            | (np.int64(fock.SITE_NUP[c]) << (2 * kl + 2)) | (np.int64(fock.SITE_NDN[c]) << (2 * kl + 3))
        masks = (mask_l[Sa][:, None] | mid | (mask_r[Sd][None, :] << (2 * (kl + 2)))).ravel()
        rows = np.searchsorted(D, masks)
        assert np.all(D[rows] == masks)
        vals = np.einsum("xi,yj->xyij", Vl, Vr).reshape(Sa.size * Sd.size, ma * md)
        V[rows, off:off + ma * md] = vals
    return V, layout


class Projected:
    """H_eff = V^T H V for one two-site position (Eqs. h_mat, wf_sec, dgemm)."""

    def __init__(self, h, v, lb: Block, rb: Block, n_up: int, n_dn: int, H=None, D=None):
        L = h.shape[0]
        if H is None:
            H, D = fock.hamiltonian_dets(h, v, n_up, n_dn)
        self.H, self.D = H, D
        self.V, self.layout = superblock_V(lb, rb, L, n_up, n_dn, D)
        self.dim = self.V.shape[1]

    def apply(self, psi):
        return self.V.T @ (self.H @ (self.V @ psi))

    def dense(self):
        return self.V.T @ (self.H @ self.V)

    def ground(self):
        ev, evec = np.linalg.eigh(self.dense())
        return float(ev[0]), evec[:, 0]


# --------------------------------------------------------------------------
# exact renormalized block operators (Eq. renorm_mat on explicit bases)
# --------------------------------------------------------------------------

def fock_op(kind: str, idx, subset_sites, space_sites, h, v, cache=None):
    """Sparse operator on the Fock space of space_sites whose index sums run over subset_sites.

    Global spin-orbital indices throughout; space_sites must be consecutive.
    Kinds and definitions (spin-orbital form of Eq. H2q, w = <pq|rs>):
      'H'          sum_pq t c+_p c_q + 1/2 sum w c+_p c+_q c_s c_r     (all in X)
      'C'  (p,)    c+_p
      'T'  (j,)    sum_{i in X} t_ij c+_i - sum_{pqr in X} w_pqrj c+_p c+_q c_r
      'V'  (i,)    sum_{qrs in X} w_iqrs c+_q c_s c_r
      'A'  (p,q)   c+_p c+_q
      'B'  (p,s)   c+_p c_s
      'Pc' (r,s)   sum_{p<q in X} (w_pqrs - w_pqsr) c+_p c+_q
      'Pa' (p,q)   sum_{r<s in X} (w_pqrs - w_pqsr) c_s c_r
      'Q'  (p,s)   sum_{q,r in X} (w_pqsr - w_pqrs) c+_q c_r
    where X is subset_sites.
    """
    k = len(space_sites)
    if cache is None:
        cache = {}
    key = ("cdag", k)
    if key not in cache:
        cache[key] = fock.fock_creation(k) if k > 0 else []
    cdag = cache[key]
    if ("c", k) not in cache:
        cache[("c", k)] = [m.T.tocsr() for m in cdag]
    c = cache[("c", k)]
    if ("tw", id(h), id(v)) not in cache:
        cache[("tw", id(h), id(v))] = fock.spin_orbital_integrals(h, v)
    t, w = cache[("tw", id(h), id(v))]
    base = 2 * space_sites[0] if space_sites else 0
    loc = lambda p: p - base
    modes = [2 * s + sg for s in subset_sites for sg in range(2)]
    dim = 4 ** k
    Z = sp.csr_matrix((dim, dim))
    if kind == "H":
        for p in modes:
            for q in modes:
                if t[p, q] != 0.0:
                    Z = Z + t[p, q] * (cdag[loc(p)] @ c[loc(q)])
        for p in modes:
            for q in modes:
                if p == q:
                    continue
                cc = cdag[loc(p)] @ cdag[loc(q)]
                for r in modes:
                    for s in modes:
                        if r != s and w[p, q, r, s] != 0.0:
                            Z = Z + 0.5 * w[p, q, r, s] * (cc @ (c[loc(s)] @ c[loc(r)]))
        return Z.tocsr()
    if kind == "C":
        return cdag[loc(idx[0])]
    if kind == "A":
        return (cdag[loc(idx[0])] @ cdag[loc(idx[1])]).tocsr()
    if kind == "B":
        return (cdag[loc(idx[0])] @ c[loc(idx[1])]).tocsr()
    if kind == "T":
        j = idx[0]
        for i in modes:
            if t[i, j] != 0.0:
                Z = Z + t[i, j] * cdag[loc(i)]
        for p in modes:
            for q in modes:
                if p == q:
                    continue
                for r in modes:
                    if w[p, q, r, j] != 0.0:
                        Z = Z - w[p, q, r, j] * (cdag[loc(p)] @ cdag[loc(q)] @ c[loc(r)])
        return Z.tocsr()
    if kind == "V":
        i = idx[0]
        for q in modes:
            for r in modes:
                for s in modes:
                    if r != s and w[i, q, r, s] != 0.0:
                        Z = Z + w[i, q, r, s] * (cdag[loc(q)] @ c[loc(s)] @ c[loc(r)])
        return Z.tocsr()
    if kind == "Pc":
        r, s = idx
        for p in modes:
            for q in modes:
                if p < q:
                    W = w[p, q, r, s] - w[p, q, s, r]
                    if W != 0.0:
                        Z = Z + W * (cdag[loc(p)] @ cdag[loc(q)])
        return Z.tocsr()
    if kind == "Pa":
        p, q = idx
        for r in modes:
            for s in modes:
                if r < s:
                    W = w[p, q, r, s] - w[p, q, s, r]
                    if W != 0.0:
                        Z = Z + W * (c[loc(s)] @ c[loc(r)])
        return Z.tocsr()
    if kind == "Q":
        p, s = idx
        for q in modes:
            for r in modes:
                coef = w[p, q, s, r] - w[p, q, r, s]
                if coef != 0.0:
                    Z = Z + coef * (cdag[loc(q)] @ c[loc(r)])
        return Z.tocsr()
    raise ValueError(kind)


def block_fock_operator(block: Block, kind: str, idx, h, v, cache=None):
    """fock_op on the block's own Fock space (sums over the block's sites)."""
    if not block.sites:
        return sp.csr_matrix((1, 1))
    return fock_op(kind, idx, block.sites, block.sites, h, v, cache)


def renormalized(block: Block, A):
    """Sector blocks {(bra sector, ket sector): V_bra^T A V_ket} of a Fock-space operator."""
    out = {}
    A = sp.csr_matrix(A)
    for ka in block.sectors:
        AV = A @ block.V[ka]
        for kb in block.sectors:
            blk = block.V[kb].T @ AV
            if np.any(np.abs(blk) > 0.0):
                out[(kb, ka)] = blk
    return out


# --------------------------------------------------------------------------
# reduced density matrices and truncation (Sec. 2.1, after Eq. wf)
# --------------------------------------------------------------------------

def rdm_blocks(psi, lb: Block, rb: Block, n_up: int, n_dn: int, direction: int):
    """rho_E per enlarged sector: direction +1 -> rho^L = psi psi^T, -1 -> rho^R = psi^T psi."""
    layout, dim = psi_layout(lb, rb, n_up, n_dn)
    blocks = {}
    for ai, b, c, di, ma, md, off in layout:
        blocks[(ai, b, c, di)] = np.asarray(psi[off:off + ma * md]).reshape(ma, md)
    if direction > 0:
        enl = enlarged_left(lb)
        rho = {}
        for E, subs in enl.items():
            n = sum(s[3] for s in subs)
            R = np.zeros((n, n))
            for ai, b, o1, m1 in subs:
                for ai2, b2, o2, m2 in subs:
                    for (x, y, c, di), blk in blocks.items():
                        if x == ai and y == b and (ai2, b2, c, di) in blocks:
                            R[o1:o1 + m1, o2:o2 + m2] += blk @ blocks[(ai2, b2, c, di)].T
            rho[E] = R
        return rho, enl
    enr = enlarged_right(rb)
    rho = {}
    for E, subs in enr.items():
        n = sum(s[3] for s in subs)
        R = np.zeros((n, n))
        for c, di, o1, m1 in subs:
            for c2, di2, o2, m2 in subs:
                for (ai, b, x, y), blk in blocks.items():
                    if x == c and y == di and (ai, b, c2, di2) in blocks:
                        R[o1:o1 + m1, o2:o2 + m2] += blk.T @ blocks[(ai, b, c2, di2)]
        rho[E] = R
    return rho, enr


def truncate(rho: dict, M: int, drop: float = TRUNC_DROP):
    """Keep the M eigenvectors with the largest eigenvalues over all sectors.

    Order: descending eigenvalue, ties by (sector order, in-sector order);
    eigenvalues <= drop are never kept.  "The M largest" is not defined when
    the M-th and the next eigenvalue above drop are (near-)equal: the cut then
    moves down past that whole cluster (consecutive eigenvalues closer than
    TRUNC_CLUSTER), so that the kept space does not depend on how a
    degenerate cluster is split; only if that would keep nothing does the
    cut stay at M (ties then by the order above).  Returns (O per sector,
    kept per sector in sector order, discarded weight = trace - sum of kept
    eigenvalues, all eigenvalues).
    """
    cand = []
    eig = {}
    for si, E in enumerate(rho):
        ev, U = np.linalg.eigh(rho[E])
        ev, U = ev[::-1], U[:, ::-1]
        eig[E] = (ev, U)
        for j, x in enumerate(ev):
            cand.append((-x, si, j, E))
    cand.sort(key=lambda z: (z[0], z[1], z[2]))
    total = sum(float(np.trace(R)) for R in rho.values())
    above = [c for c in cand if -c[0] > drop]
    n = min(M, len(above))
    cut = n
    while 0 < cut < len(above) and (-above[cut - 1][0]) - (-above[cut][0]) < TRUNC_CLUSTER:
        cut -= 1
    if cut == 0:
        cut = n
    keep = {E: [] for E in rho}
    kept_w = 0.0
    for negx, si, j, E in above[:cut]:
        keep[E].append(j)
        kept_w += -negx
    O, kept = {}, []
    for E in rho:
        js = sorted(keep[E])
        O[E] = eig[E][1][:, js]
        kept.append(len(js))
    return O, kept, total - kept_w, eig
