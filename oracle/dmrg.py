"""FP64 CPU oracle, part 3: operator-based two-site DMRG (dense sector blocks, NumPy).

TEST INFRASTRUCTURE ONLY (see oracle/fock.py).  Independent of the CUDA
library: no shared code, tables or helpers.

This is the block algorithm of Sec. 2.1 written plainly, for sizes where
explicit Fock-space bases (oracle/blocks.py) no longer fit:
  * each block stores the renormalized operators needed by the Hamiltonian
    of Eq. H2q (Sec. 2.1 "all operator intermediates"): H, a+_p, the normal
    pairs a+_p a+_q and a+_p a_s, and the one-index pre-summed operators
    T_j (left blocks) / V_i (right blocks);
  * the two-index pre-summed (complementary) operators of Sec. 2.1 are formed
    on the fly as linear combinations of the normal pairs, on the larger half
    (footnote to the pre-summed operators);
  * an enlarged block l (x) s (or s (x) r) has its operators formed
    EXPLICITLY as matrices in the 4M basis (Sec. 2.2.2 "the complete sector
    matrix ... formed according to the blocking tables"), then renormalized
    with O (Eq. renorm_mat);
  * H.psi (Eq. h_mat) uses the enlarged halves L' = l (x) s_l and
    R' = s_r (x) r: psi is an (L' x R') sector-blocked matrix and every term is
    X psi Y^T with a Jordan-Wigner sign (-1)^{p(Y) n(L' ket)}.
The decomposition of H over two halves and the blocking rules are the
identities pinned in tests/test_operator_scheme.py.
"""
from __future__ import annotations

import numpy as np

from . import blocks as ob
from . import fock

SITE_N = np.array([0, 1, 1, 2])
_CU, _CD, _PAR = fock.site_ops()
I4 = np.eye(4)


def cdag(p):
    return _CU if p % 2 == 0 else _CD


def cann(p):
    return cdag(p).T


def mat_parity(S):
    nz = np.argwhere(S != 0)
    if len(nz) == 0:
        return 0
    r, c = nz[0]
    return int(SITE_N[r] + SITE_N[c]) % 2


KIND_PARITY = {"H": 0, "C": 1, "T": 1, "V": 1, "A": 0, "B": 0}


class Ints:
    def __init__(self, h, v):
        self.L = h.shape[0]
        self.t, self.w = fock.spin_orbital_integrals(h, v)

    def W(self, p, q, r, s):
        return self.w[p, q, r, s] - self.w[p, q, s, r]


# ---------------------------------------------------------------- site operators (4x4)

def site_modes(s):
    return (2 * s, 2 * s + 1)


def site_H(I, s):
    m = np.zeros((4, 4))
    md = site_modes(s)
    for p in md:
        for q in md:
            m += I.t[p, q] * cdag(p) @ cann(q)
    for p in md:
        for q in md:
            for r in md:
                for t in md:
                    if p != q and r != t:
                        m += 0.5 * I.w[p, q, r, t] * cdag(p) @ cdag(q) @ cann(t) @ cann(r)
    return m


def site_T(I, s, j):
    m = np.zeros((4, 4))
    md = site_modes(s)
    for i in md:
        m += I.t[i, j] * cdag(i)
    for p in md:
        for q in md:
            for r in md:
                if p != q:
                    m -= I.w[p, q, r, j] * cdag(p) @ cdag(q) @ cann(r)
    return m


def site_V(I, s, i):
    m = np.zeros((4, 4))
    md = site_modes(s)
    for q in md:
        for r in md:
            for t in md:
                if r != t:
                    m += I.w[i, q, r, t] * cdag(q) @ cann(t) @ cann(r)
    return m


def site_Pc(I, s, r, q):
    a, b = site_modes(s)
    return I.W(a, b, r, q) * cdag(a) @ cdag(b)


def site_Pa(I, s, p, q):
    a, b = site_modes(s)
    return I.W(p, q, a, b) * cann(b) @ cann(a)


def site_Q(I, s, p, q):
    m = np.zeros((4, 4))
    for a in site_modes(s):
        for b in site_modes(s):
            m += (I.w[p, a, q, b] - I.w[p, a, b, q]) * cdag(a) @ cann(b)
    return m


# ---------------------------------------------------------------- blocks and sector-blocked operators

class OBlock:
    """A renormalized block: sectors, dims and operators {key: {(bra, ket): matrix}}."""

    def __init__(self, side, sites, sectors, dims):
        self.side = side
        self.sites = list(sites)
        self.sectors = list(sectors)
        self.dims = list(dims)
        self.sidx = {s: i for i, s in enumerate(self.sectors)}
        self.ops = {}

    def modes(self):
        return [2 * s + g for s in self.sites for g in range(2)]

    def op(self, key):
        return self.ops.get(key, {})


def empty_oblock(side):
    return OBlock(side, [], [(0, 0)], [1])


def op_T(X):
    return {(a, b): M.T for (b, a), M in X.items()}


def op_add(X, Y, c=1.0):
    out = {k: v.copy() for k, v in X.items()}
    for k, v in Y.items():
        if k in out:
            out[k] = out[k] + c * v
        else:
            out[k] = c * v
    return out


def lincomb(blk, terms, tr=False):
    """sum coef * op(key) over (key, coef) terms; transposed if tr."""
    out = {}
    for key, c in terms:
        if c == 0.0:
            continue
        for k, M in blk.op(key).items():
            out[k] = out[k] + c * M if k in out else c * M
    return op_T(out) if tr else out


class Enl:
    """Enlarged basis block (x) site (side 0) or site (x) block (side 1)."""

    def __init__(self, blk, side):
        self.blk, self.side = blk, side
        lay = ob.enlarged_left(blk) if side == 0 else ob.enlarged_right(blk)
        self.E = list(lay)
        self.eidx = {E: i for i, E in enumerate(self.E)}
        self.dim = [sum(s[3] for s in lay[E]) for E in self.E]
        self.where = {}
        self.subs = []
        for ei, E in enumerate(self.E):
            subs = []
            for x, y, off, m in lay[E]:
                self.where[(x, y)] = (ei, off, m)
                subs.append((x, y, off, m))
            self.subs.append(subs)
        self.n = [SITE_N_of(E) for E in self.E]

    def embed(self, X, S, coef=1.0, xpar=0):
        """Enlarged matrix of the operator product (X on the block)(S on the site), left;
        (S on the site)(X on the block), right.  X None means identity."""
        out = {}
        if coef == 0.0 or not np.any(S):
            return out
        spar = mat_parity(S)
        blk = self.blk
        if X is not None:
            byket = {}
            for (b2, a1), M in X.items():
                byket.setdefault(a1, []).append((b2, M))
        for ei, subs in enumerate(self.subs):
            for x, y, off, m in subs:
                a, st = (x, y) if self.side == 0 else (y, x)
                for st2 in range(4):
                    sv = S[st2, st]
                    if sv == 0.0:
                        continue
                    cands = [(a, None)] if X is None else byket.get(a, [])
                    for a2, M in cands:
                        key2 = (a2, st2) if self.side == 0 else (st2, a2)
                        if key2 not in self.where:
                            continue
                        ej, off2, m2 = self.where[key2]
                        if self.side == 0:
                            sgn = -1.0 if (spar * (blk.sectors[a][0] + blk.sectors[a][1])) % 2 else 1.0
                        else:
                            sgn = -1.0 if (xpar * SITE_N[st]) % 2 else 1.0
                        blkm = np.eye(m) if M is None else M
                        Z = out.get((ej, ei))
                        if Z is None:
                            Z = np.zeros((self.dim[ej], self.dim[ei]))
                            out[(ej, ei)] = Z
                        Z[off2:off2 + m2, off:off + m] += coef * sv * sgn * blkm
        return out


def SITE_N_of(E):
    return E[0] + E[1]


def eadd(acc, Z):
    for k, M in Z.items():
        if k in acc:
            acc[k] = acc[k] + M
        else:
            acc[k] = M.copy()
    return acc


def eT(Z):
    return {(b, a): M.T for (a, b), M in Z.items()}


# ---------------------------------------------------------------- enlarged operators

class Halves:
    """Enlarged-operator definitions at position k (sl = site k, sr = site k+1)."""

    def __init__(self, I, k, lblk, rblk):
        self.I, self.k = I, k
        self.l, self.r = lblk, rblk
        self.EL = Enl(lblk, 0)
        self.ER = Enl(rblk, 1)
        self.sl, self.sr = k, k + 1
        self.lm = lblk.modes()
        self.rm = rblk.modes()

    # ---- left half L' = l (x) sl: pieces (block op)(site op)
    def L_C(self, p):
        if p in self.lm:
            return self.EL.embed(self.l.op(("C", p)), I4, 1.0, 1)
        return self.EL.embed(None, cdag(p))

    def L_A(self, p, q):
        if p in self.lm and q in self.lm:
            return self.EL.embed(self.l.op(("A", p, q)), I4)
        if p in self.lm:
            return self.EL.embed(self.l.op(("C", p)), cdag(q), 1.0, 1)
        return self.EL.embed(None, cdag(p) @ cdag(q))

    def L_B(self, p, s):
        if p in self.lm and s in self.lm:
            return self.EL.embed(self.l.op(("B", p, s)), I4)
        if p in self.lm:
            return self.EL.embed(self.l.op(("C", p)), cann(s), 1.0, 1)
        if s in self.lm:
            return self.EL.embed(op_T(self.l.op(("C", s))), cdag(p), -1.0, 1)
        return self.EL.embed(None, cdag(p) @ cann(s))

    def _Pc_l(self, r, s):
        return lincomb(self.l, [(("A", p, q), self.I.W(p, q, r, s)) for p in self.lm for q in self.lm if p < q])

    def _Q_l(self, a, b):
        return lincomb(self.l, [(("B", q, r), self.I.w[a, q, b, r] - self.I.w[a, q, r, b])
                                for q in self.lm for r in self.lm])

    def L_H(self):
        I, E, l, k = self.I, self.EL, self.l, self.k
        Z = {}
        eadd(Z, E.embed(l.op(("H",)), I4))
        eadd(Z, E.embed(None, site_H(I, k)))
        for j in site_modes(k):
            X = E.embed(l.op(("T", j)), cann(j), 1.0, 1)
            eadd(Z, X)
            eadd(Z, eT(X))
        for i in self.lm:
            X = E.embed(l.op(("C", i)), site_V(I, k, i), 1.0, 1)
            eadd(Z, X)
            eadd(Z, eT(X))
        r, s = site_modes(k)
        X = E.embed(self._Pc_l(r, s), cann(s) @ cann(r))
        eadd(Z, X)
        eadd(Z, eT(X))
        for a in site_modes(k):
            for b in site_modes(k):
                eadd(Z, E.embed(self._Q_l(a, b), cdag(a) @ cann(b)))
        return Z

    def L_T(self, j):
        I, E, l, k = self.I, self.EL, self.l, self.k
        Z = {}
        eadd(Z, E.embed(l.op(("T", j)), I4, 1.0, 1))
        eadd(Z, E.embed(None, site_T(I, k, j)))
        for r in site_modes(k):
            eadd(Z, E.embed(self._Pc_l(r, j), cann(r), -1.0))
        for q in site_modes(k):
            eadd(Z, E.embed(self._Q_l(q, j), cdag(q)))
        for p in self.lm:
            eadd(Z, E.embed(l.op(("C", p)), site_Q(I, k, p, j), 1.0, 1))
            eadd(Z, E.embed(op_T(l.op(("C", p))), site_Pc(I, k, p, j), -1.0, 1))
        return Z

    def L_Pc(self, r, s):
        I, E, l, k = self.I, self.EL, self.l, self.k
        Z = {}
        eadd(Z, E.embed(self._Pc_l(r, s), I4))
        eadd(Z, E.embed(None, site_Pc(I, k, r, s)))
        for q in site_modes(k):
            X = lincomb(l, [(("C", p), I.W(p, q, r, s)) for p in self.lm])
            eadd(Z, E.embed(X, cdag(q), 1.0, 1))
        return Z

    def L_Q(self, a, b):
        I, E, l, k = self.I, self.EL, self.l, self.k
        coef = lambda q, r: I.w[a, q, b, r] - I.w[a, q, r, b]
        Z = {}
        eadd(Z, E.embed(self._Q_l(a, b), I4))
        eadd(Z, E.embed(None, site_Q(I, k, a, b)))
        for r in site_modes(k):
            X = lincomb(l, [(("C", q), coef(q, r)) for q in self.lm])
            eadd(Z, E.embed(X, cann(r), 1.0, 1))
        for q in site_modes(k):
            X = lincomb(l, [(("C", r), coef(q, r)) for r in self.lm], tr=True)
            eadd(Z, E.embed(X, cdag(q), -1.0, 1))
        return Z

    # ---- right half R' = sr (x) r: pieces (site op)(block op)
    def R_C(self, p):
        if p in self.rm:
            return self.ER.embed(self.r.op(("C", p)), I4, 1.0, 1)
        return self.ER.embed(None, cdag(p))

    def R_A(self, p, q):
        if p in self.rm and q in self.rm:
            return self.ER.embed(self.r.op(("A", p, q)), I4)
        if q in self.rm:
            return self.ER.embed(self.r.op(("C", q)), cdag(p), 1.0, 1)
        return self.ER.embed(None, cdag(p) @ cdag(q))

    def R_B(self, p, s):
        if p in self.rm and s in self.rm:
            return self.ER.embed(self.r.op(("B", p, s)), I4)
        if s in self.rm:
            return self.ER.embed(op_T(self.r.op(("C", s))), cdag(p), 1.0, 1)
        if p in self.rm:
            return self.ER.embed(self.r.op(("C", p)), cann(s), -1.0, 1)
        return self.ER.embed(None, cdag(p) @ cann(s))

    def _Pa_r(self, p, q):
        return lincomb(self.r, [(("A", a, b), self.I.W(p, q, a, b)) for a in self.rm for b in self.rm if a < b],
                       tr=True)

    def _Q_r(self, a, b):
        return lincomb(self.r, [(("B", q, r), self.I.w[a, q, b, r] - self.I.w[a, q, r, b])
                                for q in self.rm for r in self.rm])

    def R_H(self):
        I, E, r, s1 = self.I, self.ER, self.r, self.k + 1
        Z = {}
        eadd(Z, E.embed(r.op(("H",)), I4))
        eadd(Z, E.embed(None, site_H(I, s1)))
        for j in self.rm:
            X = E.embed(op_T(r.op(("C", j))), site_T(I, s1, j), 1.0, 1)
            eadd(Z, X)
            eadd(Z, eT(X))
        for i in site_modes(s1):
            X = E.embed(r.op(("V", i)), cdag(i), 1.0, 1)
            eadd(Z, X)
            eadd(Z, eT(X))
        p, q = site_modes(s1)
        X = E.embed(self._Pa_r(p, q), cdag(p) @ cdag(q))
        eadd(Z, X)
        eadd(Z, eT(X))
        for p in site_modes(s1):
            for s in site_modes(s1):
                eadd(Z, E.embed(self._Q_r(p, s), cdag(p) @ cann(s)))
        return Z

    def R_V(self, i):
        I, E, r, s1 = self.I, self.ER, self.r, self.k + 1
        Z = {}
        eadd(Z, E.embed(None, site_V(I, s1, i)))
        eadd(Z, E.embed(r.op(("V", i)), I4, 1.0, 1))
        for q in site_modes(s1):
            eadd(Z, E.embed(self._Pa_r(i, q), cdag(q)))
        for q in self.rm:
            eadd(Z, E.embed(r.op(("C", q)), site_Pa(I, s1, i, q), 1.0, 1))
        for q in site_modes(s1):
            for s in site_modes(s1):
                X = lincomb(r, [(("C", rr), I.w[i, q, rr, s] - I.w[i, q, s, rr]) for rr in self.rm], tr=True)
                eadd(Z, E.embed(X, cdag(q) @ cann(s), 1.0, 1))
        for s in site_modes(s1):
            eadd(Z, E.embed(self._Q_r(i, s), cann(s)))
        return Z

    def R_Pa(self, p, q):
        I, E, r, s1 = self.I, self.ER, self.r, self.k + 1
        Z = {}
        eadd(Z, E.embed(None, site_Pa(I, s1, p, q)))
        eadd(Z, E.embed(self._Pa_r(p, q), I4))
        for rr in site_modes(s1):
            X = lincomb(r, [(("C", s), I.W(p, q, rr, s)) for s in self.rm], tr=True)
            eadd(Z, E.embed(X, cann(rr), -1.0, 1))
        return Z

    def R_Q(self, a, b):
        I, E, r, s1 = self.I, self.ER, self.r, self.k + 1
        coef = lambda q, rr: I.w[a, q, b, rr] - I.w[a, q, rr, b]
        Z = {}
        eadd(Z, E.embed(None, site_Q(I, s1, a, b)))
        eadd(Z, E.embed(self._Q_r(a, b), I4))
        for q in site_modes(s1):
            X = lincomb(r, [(("C", rr), coef(q, rr)) for rr in self.rm], tr=True)
            eadd(Z, E.embed(X, cdag(q), 1.0, 1))
        for rr in site_modes(s1):
            X = lincomb(r, [(("C", q), coef(q, rr)) for q in self.rm])
            eadd(Z, E.embed(X, cann(rr), -1.0, 1))
        return Z


# ---------------------------------------------------------------- H.psi on the two halves

class HPsi:
    """sigma = H psi at position k with explicit enlarged operators (Eq. h_mat)."""

    def __init__(self, I, k, lblk, rblk, n_up, n_dn):
        self.I, self.k = I, k
        self.Hv = Halves(I, k, lblk, rblk)
        self.layout, self.dim = ob.psi_layout(lblk, rblk, n_up, n_dn)
        EL, ER = self.Hv.EL, self.Hv.ER
        self.EF = {}  # (ei, fi) -> allowed pair
        for ai, b, c, di, ma, md, off in self.layout:
            ei, ro, _ = EL.where[(ai, b)]
            fi, co, _ = ER.where[(c, di)]
            self.EF.setdefault((ei, fi), []).append((off, ma, md, ro, co))
        L = I.L
        lp = list(range(2 * (k + 1)))
        rp = list(range(2 * (k + 1), 2 * L))
        H = self.Hv
        self.terms = []  # (X enlarged dict, Y enlarged dict, parity of Y, hc)
        self.terms.append((H.L_H(), None, 0, False))
        self.terms.append((None, H.R_H(), 0, False))
        for j in rp:
            self.terms.append((H.L_T(j), eT(H.R_C(j)), 1, True))
        for i in lp:
            self.terms.append((H.L_C(i), H.R_V(i), 1, True))
        if (k + 1) <= (L - k - 1):
            for p in lp:
                for q in lp:
                    if p < q:
                        self.terms.append((H.L_A(p, q), H.R_Pa(p, q), 0, True))
            for p in lp:
                for s in lp:
                    self.terms.append((H.L_B(p, s), H.R_Q(p, s), 0, False))
        else:
            for r in rp:
                for s in rp:
                    if r < s:
                        self.terms.append((H.L_Pc(r, s), eT(H.R_A(r, s)), 0, True))
            for q in rp:
                for r in rp:
                    self.terms.append((H.L_Q(q, r), H.R_B(q, r), 0, False))
        self.terms = [t for t in self.terms if (t[0] is None or t[0]) and (t[1] is None or t[1])]

    def to_ef(self, psi):
        EL, ER = self.Hv.EL, self.Hv.ER
        out = {}
        for (ei, fi), parts in self.EF.items():
            Mx = np.zeros((EL.dim[ei], ER.dim[fi]))
            for off, ma, md, ro, co in parts:
                Mx[ro:ro + ma, co:co + md] = psi[off:off + ma * md].reshape(ma, md)
            out[(ei, fi)] = Mx
        return out

    def from_ef(self, ef):
        psi = np.zeros(self.dim)
        for (ei, fi), parts in self.EF.items():
            Mx = ef.get((ei, fi))
            if Mx is None:
                continue
            for off, ma, md, ro, co in parts:
                psi[off:off + ma * md] = Mx[ro:ro + ma, co:co + md].ravel()
        return psi

    def apply(self, psi):
        EL = self.Hv.EL
        x = self.to_ef(psi)
        out = {}

        def acc(key, M):
            if key in self.EF:
                out[key] = out[key] + M if key in out else M

        for X, Y, ypar, hc in self.terms:
            Xk = {}
            if X is not None:
                for (e2, e1), M in X.items():
                    Xk.setdefault(e1, []).append((e2, M))
            Yk = {}
            if Y is not None:
                for (f2, f1), M in Y.items():
                    Yk.setdefault(f1, []).append((f2, M))
            for (ei, fi), P in x.items():
                sgn = -1.0 if (ypar * EL.n[ei]) % 2 else 1.0
                xs = [(ei, None)] if X is None else Xk.get(ei, [])
                ys = [(fi, None)] if Y is None else Yk.get(fi, [])
                for e2, Mx in xs:
                    XP = P if Mx is None else Mx @ P
                    for f2, My in ys:
                        R = XP if My is None else XP @ My.T
                        acc((e2, f2), sgn * R)
            if hc:
                # transpose of the full term: sigma[E,F] += sgn(E) X[E'<-E]^T psi[E',F'] Y[F'<-F]
                for (e2, e1), Mx in (X.items() if X is not None else []):
                    sgn = -1.0 if (ypar * EL.n[e1]) % 2 else 1.0
                    for (f2, f1), My in (Y.items() if Y is not None else []):
                        P = x.get((e2, f2))
                        if P is None or (e1, f1) not in self.EF:
                            continue
                        acc((e1, f1), sgn * (Mx.T @ P @ My))
        return self.from_ef(out)

    def dense(self):
        n = self.dim
        Hm = np.zeros((n, n))
        for i in range(n):
            e = np.zeros(n)
            e[i] = 1.0
            Hm[:, i] = self.apply(e)
        return Hm


# ---------------------------------------------------------------- renormalization

def renormalize(I, k, lblk, rblk, direction, O, kept):
    """New block from O per enlarged sector (Eq. renorm_mat) with all its stored operators."""
    Hv = Halves(I, k, lblk, rblk)
    E = Hv.EL if direction > 0 else Hv.ER
    secs, dims, eidx = [], [], []
    for ei, Ek in enumerate(E.E):
        if kept[ei] > 0:
            secs.append(Ek)
            dims.append(int(kept[ei]))
            eidx.append(ei)
    L = I.L
    if direction > 0:
        sites = list(range(k + 1))
        nb = OBlock(0, sites, secs, dims)
        modes = [2 * s + g for s in sites for g in range(2)]
        keys = [("H",)] + [("C", p) for p in modes] + [("T", j) for j in range(2 * (k + 1), 2 * L)]
        keys += [("A", p, q) for p in modes for q in modes if p < q] + [("B", p, s) for p in modes for s in modes]
        make = {"H": lambda key: Hv.L_H(), "C": lambda key: Hv.L_C(key[1]), "T": lambda key: Hv.L_T(key[1]),
                "A": lambda key: Hv.L_A(key[1], key[2]), "B": lambda key: Hv.L_B(key[1], key[2])}
    else:
        sites = list(range(k + 1, L))
        nb = OBlock(1, sites, secs, dims)
        modes = [2 * s + g for s in sites for g in range(2)]
        keys = [("H",)] + [("C", p) for p in modes] + [("V", i) for i in range(0, 2 * (k + 1))]
        keys += [("A", p, q) for p in modes for q in modes if p < q] + [("B", p, s) for p in modes for s in modes]
        make = {"H": lambda key: Hv.R_H(), "C": lambda key: Hv.R_C(key[1]), "V": lambda key: Hv.R_V(key[1]),
                "A": lambda key: Hv.R_A(key[1], key[2]), "B": lambda key: Hv.R_B(key[1], key[2])}
    new_of = {ei: n for n, ei in enumerate(eidx)}
    for key in keys:
        Z = make[key[0]](key)
        out = {}
        for (e2, e1), M in Z.items():
            if e1 in new_of and e2 in new_of:
                blk = O[e2].T @ M @ O[e1]
                if np.any(blk):
                    out[(new_of[e2], new_of[e1])] = blk
        nb.ops[key] = out
    return nb


def rho_blocks(hp: HPsi, psi, direction):
    """rho^L = psi psi^T (direction +1) or rho^R = psi^T psi per enlarged sector."""
    x = hp.to_ef(psi)
    E = hp.Hv.EL if direction > 0 else hp.Hv.ER
    rho = {Ek: np.zeros((E.dim[i], E.dim[i])) for i, Ek in enumerate(E.E)}
    for (ei, fi), P in x.items():
        if direction > 0:
            rho[E.E[ei]] += P @ P.T
        else:
            rho[E.E[fi]] += P.T @ P
    return rho


def lowest(hp: HPsi, tol=1e-10, dense_max=2500):
    if hp.dim <= dense_max:
        ev, U = np.linalg.eigh(hp.dense())
        return float(ev[0]), U[:, 0]
    return fock.lanczos_ground(hp.apply, hp.dim, tol=tol)


class OracleDMRG:
    """Two-site sweeps (Sec. 2.1) from the Aufbau product state, same schedule as the C ABI."""

    def __init__(self, h, v, N, two_sz, M):
        self.I = Ints(h, v)
        self.L = h.shape[0]
        self.nu, self.nd = (N + two_sz) // 2, (N - two_sz) // 2
        self.M = M
        L = self.L
        self.left = {0: empty_oblock(0)}
        self.right = {0: empty_oblock(1)}
        for k in range(L - 2, 0, -1):
            r = self.right[L - k - 2]
            E = Enl(r, 1)
            st = (1 if k + 1 < self.nu else 0) + (2 if k + 1 < self.nd else 0)
            kept, O = [], []
            for ei, subs in enumerate(E.subs):
                col = np.zeros((E.dim[ei], 0))
                for x, y, off, m in subs:
                    if x == st:
                        col = np.zeros((E.dim[ei], 1))
                        col[off, 0] = 1.0
                kept.append(col.shape[1])
                O.append(col)
            self.right[L - k - 1] = renormalize(self.I, k, self.left.get(k, empty_oblock(0)), r, -1, O, kept)

    def step(self, k, direction, tol):
        L = self.L
        hp = HPsi(self.I, k, self.left[k], self.right[L - k - 2], self.nu, self.nd)
        e, psi = lowest(hp, tol)
        rho = rho_blocks(hp, psi, direction)
        Eobj = hp.Hv.EL if direction > 0 else hp.Hv.ER
        rho_ord = {Ek: rho[Ek] for Ek in Eobj.E}
        O, kept, dw, _ = ob.truncate(rho_ord, self.M)
        Ol = [O[Ek] for Ek in Eobj.E]
        nb = renormalize(self.I, k, self.left[k], self.right[L - k - 2], direction, Ol, kept)
        if direction > 0:
            self.left[k + 1] = nb
        else:
            self.right[L - k - 1] = nb
        return e, dw

    def sweep(self, nsweeps, tol=1e-10):
        L = self.L
        E = []
        for _ in range(nsweeps):
            for k in range(0, L - 2):
                E.append(self.step(k, +1, tol)[0])
            for k in range(L - 2, 0, -1):
                E.append(self.step(k, -1, tol)[0])
        return np.array(E)
