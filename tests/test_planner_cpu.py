"""CPU checks of the library's host planner (no GPU): its operator pieces rebuild H exactly.

The planner's dump lists every product l-op (x) s_l (x) s_r (x) r-op of the
four-part H.psi (Sec. 2.2.1, Eq. dgemm) and the blocking definition of every
operator of a new block (Sec. 2.2.2).  Here each piece is rebuilt as a
genuine fermionic operator on the Fock space of the whole (small) system, with
the oracle's Jordan-Wigner operators, and the sum is compared with the
literal Hamiltonian of Eq. H2q / the literal block operators.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fock
from oracle.blocks import fock_op
from paper_2001_04890_gb300 import binding, workloads

KINDS = {0: "H", 1: "C", 2: "T", 3: "V", 4: "A", 5: "B"}


def _parse_op(tok):
    if tok[0] == "I":
        return ("I",)
    if tok[0] == "S":
        return ("S", int(tok[1]), int(tok[2]), int(tok[3]), bool(int(tok[4])))
    kind, tr, n = int(tok[1]), bool(int(tok[2])), int(tok[3])
    lc = [(int(tok[4 + 3 * m]), int(tok[5 + 3 * m]), float(tok[6 + 3 * m])) for m in range(n)]
    return ("C", kind, tr, lc)


def parse_pieces(text):
    out = []
    for line in text.strip().splitlines():
        head, lop, sl, sr, rop = [x.split() for x in line.split("|")]
        out.append(dict(coef=float(head[0]), hc=bool(int(head[1])), l=_parse_op(lop),
                        sl=np.array(sl, float).reshape(4, 4), sr=np.array(sr, float).reshape(4, 4),
                        r=_parse_op(rop)))
    return out


def parse_newops(text):
    ops = []
    for line in text.strip().splitlines():
        if line.startswith("OP"):
            _, kind, i, j = line.split()
            ops.append(dict(kind=int(kind), i=int(i), j=int(j), pieces=[]))
        else:
            head, blk, site = [x.split() for x in line.split("|")]
            ops[-1]["pieces"].append(dict(coef=float(head[0]), blk=_parse_op(blk),
                                          site=np.array(site, float).reshape(4, 4)))
    return ops


def _idx(kind, i, j):
    if kind == 0:
        return None
    if kind in (1, 2, 3):
        return (i,)
    return (i, j)


class Space:
    def __init__(self, h, v, sites):
        self.h, self.v, self.sites = h, v, list(sites)
        self.cache = {}
        self.dim = 4 ** len(sites)

    def block(self, op, subset):
        if op[0] == "I":
            return sp.identity(self.dim, format="csr")
        if op[0] == "S":
            _, kind, i, j, tr = op
            A = fock_op(KINDS[kind], _idx(kind, i, j), subset, self.sites, self.h, self.v, self.cache)
            return A.T.tocsr() if tr else A
        _, kind, tr, lc = op
        A = sp.csr_matrix((self.dim, self.dim))
        for i, j, c in lc:
            A = A + c * fock_op(KINDS[kind], _idx(kind, i, j), subset, self.sites, self.h, self.v, self.cache)
        return A.T.tocsr() if tr else A

    def site(self, S, s):
        """4x4 site matrix of global site s as an operator (JW string if odd)."""
        nz = np.argwhere(S != 0)
        par = 0
        if len(nz):
            r, c = nz[0]
            par = int(fock.SITE_NUP[r] + fock.SITE_NDN[r] + fock.SITE_NUP[c] + fock.SITE_NDN[c]) % 2
        _, _, P = fock.site_ops()
        m = sp.identity(1, format="csr")
        for t in self.sites:
            if t < s:
                f = sp.csr_matrix(P) if par else sp.identity(4)
            elif t == s:
                f = sp.csr_matrix(S)
            else:
                f = sp.identity(4)
            m = sp.kron(m, f, format="csr")
        return m


def _maxdiff(A, B):
    d = (A - B).toarray()
    return np.max(np.abs(d))


@pytest.mark.parametrize("L,k", [(5, 0), (5, 1), (5, 2), (5, 3), (4, 1)])
@pytest.mark.parametrize("compress", [False, True])
def test_hpsi_pieces_rebuild_hamiltonian(L, k, compress):
    h, v = workloads.integrals(L, seed=30 + L + k)
    text = binding.debug_pieces(h, v, k, l_empty=(k == 0), r_empty=(k == L - 2), compress=compress)
    pieces = parse_pieces(text)
    S = Space(h, v, range(L))
    lsub, rsub = list(range(k)), list(range(k + 2, L))
    Z = sp.csr_matrix((S.dim, S.dim))
    for p in pieces:
        T = S.block(p["l"], lsub) @ S.site(p["sl"], k) @ S.site(p["sr"], k + 1) @ S.block(p["r"], rsub)
        T = p["coef"] * T
        Z = Z + T + (T.T if p["hc"] else 0)
    H = fock.hamiltonian_fock(h, v, fock.fock_creation(L))
    assert _maxdiff(H, Z) < 1e-12


@pytest.mark.parametrize("L,k,side", [(5, 0, 0), (5, 1, 0), (5, 2, 0), (5, 3, 1), (5, 2, 1), (5, 0, 1), (4, 1, 1)])
def test_new_block_operators_blocking(L, k, side):
    h, v = workloads.integrals(L, seed=40 + L + k + side)
    old_empty = (k == 0) if side == 0 else (k == L - 2)
    ops = parse_newops(binding.debug_newops(h, v, k, side, old_empty))
    if side == 0:
        sites, sub_old, s = list(range(k + 1)), list(range(k)), k
    else:
        sites, sub_old, s = list(range(k + 1, L)), list(range(k + 2, L)), k + 1
    S = Space(h, v, sites)
    kinds_seen = set()
    for op in ops:
        Z = sp.csr_matrix((S.dim, S.dim))
        for p in op["pieces"]:
            B = S.block(p["blk"], sub_old)
            E = S.site(p["site"], s)
            Z = Z + p["coef"] * (B @ E if side == 0 else E @ B)
        ref = fock_op(KINDS[op["kind"]], _idx(op["kind"], op["i"], op["j"]), sites, sites, h, v, S.cache)
        assert _maxdiff(ref, Z) < 1e-12, (op["kind"], op["i"], op["j"])
        kinds_seen.add(op["kind"])
    assert {0, 1}.issubset(kinds_seen)


def test_task_dump_reproduces_the_flop_count():
    """The algorithmic FLOPs the bench reports are the sum over the task list of
    2 min(m n p + m p q, n p q + m n q) (identity sides cost nothing)."""
    import numpy as np
    from paper_2001_04890_gb300 import binding, workloads
    L, N, k = 10, 10, 4
    h, v = workloads.integrals(L, seed=3)
    sec = [(a, b, 1 + (3 * a + b) % 5) for a in range(0, 5) for b in range(0, 5)]
    sec_r = [(a, b, 1 + (a + 2 * b) % 4) for a in range(0, 5) for b in range(0, 5)]
    flops, tasks = binding.plan_hpsi_flops(h, v, N, 0, k, sec, sec_r)
    T = binding.debug_tasks(h, v, N, 0, k, sec, sec_r)
    assert T.shape == (tasks, 7)
    g, m, n, p, q, idf, yo = T.T.astype(np.float64)
    xid, zid = (T[:, 5] & 1) > 0, (T[:, 5] & 2) > 0
    f = np.where(xid & zid, 0.0, np.where(xid, 2 * n * p * q, np.where(zid, 2 * m * n * p,
                 2 * np.minimum(m * n * p + m * p * q, n * p * q + m * n * q))))
    assert abs(f.sum() - flops) <= 1e-9 * flops
    # an identity side is square, and every task maps an input block to an output block of the layout
    assert np.all(n[xid] == m[xid]) and np.all(p[zid] == q[zid])
    assert np.all(T[:, 1:5] >= 1)


@pytest.mark.parametrize("layout", ["mixed", "profile_sz1", "profile_large"])
def test_grouped_task_list_is_a_stable_sort_by_output_block(layout):
    """The GPU task list (built in two counting passes straight into grouped order)
    is the build-order list grouped by output psi block, tasks of one block in
    build order (the ordered sigma accumulation relies on it)."""
    import numpy as np
    from paper_2001_04890_gb300 import binding, workloads
    if layout == "mixed":
        L, N, tsz, k = 10, 10, 0, 4
        sec = [(a, b, 1 + (3 * a + b) % 5) for a in range(0, 5) for b in range(0, 5)]
        sec_r = [(a, b, 1 + (a + 2 * b) % 4) for a in range(0, 5) for b in range(0, 5)]
    else:
        L, N, tsz, M, k = (13, 13, 1, 90, 5) if layout == "profile_sz1" else (16, 16, 0, 300, 7)
        nu, nd = (N + tsz) // 2, (N - tsz) // 2
        left, right = workloads.middle_bond_sectors(L, nu, nd, M, k)
        sec = [(a, b, d) for (a, b), d in sorted(left.items())]
        sec_r = [(a, b, d) for (a, b), d in sorted(right.items())]
    h, v = workloads.integrals(L, seed=3)
    T0 = binding.debug_tasks(h, v, N, tsz, k, sec, sec_r)
    T1 = binding.debug_tasks(h, v, N, tsz, k, sec, sec_r, grouped=True)
    assert T1.shape == T0.shape
    order = np.argsort(T0[:, 0], kind="stable")
    assert np.array_equal(T1, T0[order])
    assert np.all(np.diff(T1[:, 0]) >= 0)


@pytest.mark.parametrize("seed", range(12))
def test_grouped_task_list_on_random_layouts(seed):
    """Random sector tables (dims 1..6, random fillings and spins): the two-pass grouped
    expansion the GPU path uses equals the stable grouping of the build-order list, and
    its FLOP count equals the dump's."""
    import numpy as np
    from paper_2001_04890_gb300 import binding, workloads
    rng = np.random.default_rng(100 + seed)
    L = int(rng.integers(5, 10))
    k = int(rng.integers(0, L - 1))
    N = int(rng.integers(1, 2 * L))
    tsz = int(rng.choice([x for x in range(-N, N + 1, 2) if abs(x) <= N and (N - x) // 2 <= L and (N + x) // 2 <= L]))

    def table(n_sites):
        if n_sites == 0:
            return [(0, 0, 1)]
        out = []
        for a in range(0, n_sites + 1):
            for b in range(0, n_sites + 1):
                if rng.random() < 0.6:
                    out.append((a, b, int(rng.integers(1, 7))))
        return out or [(0, 0, 1)]
    sec_l, sec_r = table(k), table(L - k - 2)
    h, v = workloads.integrals(L, seed=seed)
    T0 = binding.debug_tasks(h, v, N, tsz, k, sec_l, sec_r)
    T1 = binding.debug_tasks(h, v, N, tsz, k, sec_l, sec_r, grouped=True)
    assert T1.shape == T0.shape
    if len(T0):
        order = np.argsort(T0[:, 0], kind="stable")
        assert np.array_equal(T1, T0[order])
    f, n = binding.plan_hpsi_flops(h, v, N, tsz, k, sec_l, sec_r)
    assert n == len(T0)
