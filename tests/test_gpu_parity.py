"""GPU parity of the C-ABI path (FP64) against the oracle.

H.psi (Sec. 2.2.1, Eq. dgemm), renormalized operators (Eq. renorm_mat),
Davidson energies (Eq. h_mat), RDM truncation (Sec. 2.1) and full sweeps
against full CI.  FP64 tolerance: 1e-12 relative on H.psi and operators (the
two sides sum the same products in a different order), 1e-10 Eh on energies.
"""
import numpy as np
import pytest

from oracle import blocks as ob
from oracle import fock
from paper_2001_04890_gb300 import binding, workloads
from tests.helpers import build_random_position

pytestmark = pytest.mark.gpu

KIND_NAME = {0: "H", 1: "C", 2: "T", 3: "V", 4: "A", 5: "B"}


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("L,N,two_sz,M,k", [(5, 4, 0, 16, 1), (6, 6, 0, 40, 2), (6, 5, 1, 24, 1),
                                            (6, 6, 0, 40, 0), (6, 6, 0, 40, 4), (7, 7, 1, 30, 3)])
def test_hpsi_matches_projected_hamiltonian(L, N, two_sz, M, k):
    h, v = workloads.integrals(L, seed=100 + L + k)
    nu, nd = (N + two_sz) // 2, (N - two_sz) // 2
    ctx = binding.DMRG(h, v, N, two_sz, M)
    lb, rb = build_random_position(ctx, h, v, k, M, seed=k + 7)
    P = ob.Projected(h, v, lb, rb, nu, nd)
    blocks, dim = ctx.psi_layout()
    assert dim == P.dim
    ref_layout = np.array([(a, b, c, d, ma, md, off) for a, b, c, d, ma, md, off in P.layout])
    assert np.array_equal(blocks, ref_layout)
    for seed in range(2):
        psi = workloads.gaussian(dim, seed=seed)
        assert _rel(ctx.hpsi(psi), P.apply(psi)) < 1e-12
    ctx.close()


def test_renormalized_operators_match_exact():
    L, N, M, k = 6, 6, 30, 3
    h, v = workloads.integrals(L, seed=5)
    ctx = binding.DMRG(h, v, N, 0, M)
    lb, rb = build_random_position(ctx, h, v, k, M, seed=3)
    checks = [(0, 0, -1, -1), (0, 1, 1, -1), (0, 2, 8, -1), (0, 2, 11, -1), (0, 4, 0, 3), (0, 5, 2, 5),
              (0, 5, 1, 0), (1, 0, -1, -1), (1, 1, 10, -1), (1, 3, 2, -1), (1, 3, 7, -1), (1, 4, 10, 11),
              (1, 5, 11, 10)]
    for side, kind, i, j in checks:
        blk = lb if side == 0 else rb
        got = ctx.block_op(side, kind, i, j)
        idx = None if kind == 0 else ((i,) if kind in (1, 2, 3) else (i, j))
        A = ob.block_fock_operator(blk, KIND_NAME[kind], idx, h, v)
        ren = ob.renormalized(blk, A)
        du = dd = 0
        if kind in (1, 2):
            du, dd = (1, 0) if i % 2 == 0 else (0, 1)
        elif kind == 3:
            du, dd = (-1, 0) if i % 2 == 0 else (0, -1)
        elif kind == 4:
            du = (i % 2 == 0) + (j % 2 == 0)
            dd = (i % 2 == 1) + (j % 2 == 1)
        elif kind == 5:
            du = (i % 2 == 0) - (j % 2 == 0)
            dd = (i % 2 == 1) - (j % 2 == 1)
        parts = []
        for ka in blk.sectors:
            kb = (ka[0] + du, ka[1] + dd)
            if kb not in blk.V:
                continue
            parts.append(ren.get((kb, ka), np.zeros((blk.V[kb].shape[1], blk.V[ka].shape[1]))).ravel())
        ref = np.concatenate(parts)
        assert got.shape == ref.shape, (side, kind, i, j)
        assert _rel(got, ref) < 1e-12, (side, kind, i, j)
    ctx.close()


def test_davidson_matches_dense_eigh():
    L, N, M, k = 6, 6, 40, 2
    h, v = workloads.integrals(L, seed=8)
    ctx = binding.DMRG(h, v, N, 0, M)
    lb, rb = build_random_position(ctx, h, v, k, M, seed=4)
    P = ob.Projected(h, v, lb, rb, 3, 3)
    e_ref, x_ref = P.ground()
    e, it = ctx.davidson(tol=1e-10, max_iter=300)
    assert abs(e - e_ref) < 1e-10
    x = ctx.get_psi()
    assert abs(abs(x @ x_ref) - 1.0) < 1e-8
    ctx.close()


def test_auto_truncation_matches_oracle():
    L, N, M, k = 6, 6, 40, 2
    h, v = workloads.integrals(L, seed=9)
    for direction in (+1, -1):
        ctx = binding.DMRG(h, v, N, 0, M)
        lb, rb = build_random_position(ctx, h, v, k, M, seed=6)
        ctx.davidson(tol=1e-11, max_iter=300)
        psi = ctx.get_psi()
        rho, _ = ob.rdm_blocks(psi, lb, rb, 3, 3, direction)
        O_ref, kept_ref, dw_ref, _ = ob.truncate(rho, M)
        dw, kept = ctx.renormalize(direction)
        assert list(kept) == list(kept_ref)
        assert abs(dw - dw_ref) < 1e-12
        ctx.close()


def test_hpsi_hermitian_deterministic_and_conserving():
    L, N, M, k = 10, 10, 48, 4
    h, v = workloads.integrals(L, seed=11)
    ctx = binding.DMRG(h, v, N, 0, M)
    build_random_position(ctx, h, v, k, M, seed=2)
    _, dim = ctx.psi_layout()
    x, y = workloads.gaussian(dim, 1), workloads.gaussian(dim, 2)
    Hx, Hy = ctx.hpsi(x), ctx.hpsi(y)
    assert abs(x @ Hy - y @ Hx) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(Hy)
    assert np.array_equal(ctx.hpsi(x), Hx)  # bitwise repeatable
    ctx.close()


def test_sweep_reaches_fci_small():
    L, N, M = 6, 6, 64
    h, v = workloads.integrals(L, seed=12)
    e_fci = fock.fci_ground(h, v, 3, 3)[0]
    ctx = binding.DMRG(h, v, N, 0, M)
    E = ctx.sweep(4, tol=1e-10)
    # M = 64 keeps 3-site blocks complete once the kept ranks have grown (sweep 3)
    steps = 2 * (L - 2)
    assert np.all(E >= e_fci - 1e-10)
    assert abs(np.min(E[2 * steps:]) - e_fci) < 1e-10
    ctx.close()


def test_l8_m256_exact():
    """M=256 keeps every Schmidt rank of L=8: from sweep 3 on every step is the FCI energy."""
    L, N, M, nsw = 8, 8, 256, 5
    h, v = workloads.integrals(L, seed=0)
    e_fci = fock.fci_ground(h, v, 4, 4)[0]
    ctx = binding.DMRG(h, v, N, 0, M)
    E = ctx.sweep(nsw, tol=1e-10).reshape(nsw, 2 * (L - 2))
    ctx.close()
    # ranks grow 4 -> 16 -> 64 -> 256 per half sweep from the Aufbau start
    assert np.all(np.abs(E[3, 3:] - e_fci) < 1e-10), E[3] - e_fci
    assert np.all(np.abs(E[4] - e_fci) < 1e-10), E[4] - e_fci
    assert np.all(E >= e_fci - 1e-10)
