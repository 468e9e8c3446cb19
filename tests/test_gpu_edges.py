"""Degenerate and edge cases of the GPU path (FP64).

Empty and full filling, fully polarized electrons, the smallest lattices
(L = 2: both blocks empty, L = 3), bond dimension 1, the zero vector and
linearity of H.psi, and argument errors that must come back as status codes
(never a device fault).  Energies against determinant FCI (1e-10 Eh) or the
variational bound.
"""
import numpy as np
import pytest

from oracle import fock
from paper_2001_04890_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,N,two_sz", [(4, 0, 0), (4, 8, 0), (5, 3, 3), (3, 1, 1), (5, 9, 1), (4, 4, -2)])
def test_degenerate_fillings_reach_fci(L, N, two_sz):
    h, v = workloads.integrals(L, seed=40 + L)
    nu, nd = (N + two_sz) // 2, (N - two_sz) // 2
    e_fci = fock.fci_ground(h, v, nu, nd)[0]
    ctx = binding.DMRG(h, v, N, two_sz, 64)
    E = ctx.sweep(3, tol=1e-11)
    assert np.all(E >= e_fci - 1e-10)
    assert abs(np.min(E) - e_fci) < 1e-10
    ctx.close()


def test_two_sites_without_blocks():
    L, N = 2, 2
    h, v = workloads.integrals(L, seed=7)
    e_fci = fock.fci_ground(h, v, 1, 1)[0]
    ctx = binding.DMRG(h, v, N, 0, 16)
    ctx.set_position(0, 1)
    blocks, dim = ctx.psi_layout()
    assert dim == 4  # C(2,1)^2 determinants
    e, _ = ctx.davidson(tol=1e-12, max_iter=50)
    assert abs(e - e_fci) < 1e-10
    ctx.close()


def test_bond_dimension_one_is_variational():
    L, N = 6, 6
    h, v = workloads.integrals(L, seed=8)
    e_fci = fock.fci_ground(h, v, 3, 3)[0]
    ctx = binding.DMRG(h, v, N, 0, 1)
    E = ctx.sweep(2, tol=1e-10)
    assert np.all(np.isfinite(E)) and np.all(E >= e_fci - 1e-10)
    ctx.close()


def test_hpsi_zero_vector_and_linearity():
    L, N, M, k = 8, 8, 40, 3
    h, v = workloads.integrals(L, seed=9)
    ctx = binding.DMRG(h, v, N, 0, M)
    workloads.grow_middle_bond(ctx, L, 4, 4, M, k, seed=1)
    _, dim = ctx.psi_layout()
    assert np.array_equal(ctx.hpsi(np.zeros(dim)), np.zeros(dim))
    x, y = workloads.gaussian(dim, 1), workloads.gaussian(dim, 2)
    a, b = 0.75, -2.5
    lhs = ctx.hpsi(a * x + b * y)
    rhs = a * ctx.hpsi(x) + b * ctx.hpsi(y)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(rhs))
    ctx.close()


def test_argument_errors_are_status_codes():
    L, N = 6, 6
    h, v = workloads.integrals(L, seed=10)
    ctx = binding.DMRG(h, v, N, 0, 16)
    lib = binding.lib()
    assert lib.dmrg_set_position(ctx.ctx, L - 1, 1) == binding.DMRG_EINVAL
    assert lib.dmrg_set_position(ctx.ctx, -1, 1) == binding.DMRG_EINVAL
    assert lib.dmrg_set_position(ctx.ctx, 0, 0) == binding.DMRG_EINVAL
    assert lib.dmrg_hpsi(ctx.ctx, None, None, 0) == binding.DMRG_EINVAL
    with pytest.raises(binding.DMRGError):
        ctx.set_tune(target_chunks=0.5)
    # the context still works after the rejected calls
    ctx.set_position(0, 1)
    e, _ = ctx.davidson(tol=1e-10, max_iter=100)
    assert np.isfinite(e)
    ctx.close()


def test_release_block_keeps_the_middle_bond():
    L, N, M, k = 10, 10, 60, 4
    h, v = workloads.integrals(L, seed=13)
    ref = binding.DMRG(h, v, N, 0, M)
    workloads.grow_middle_bond(ref, L, 5, 5, M, k, seed=3)
    ctx = binding.DMRG(h, v, N, 0, M)
    workloads.grow_middle_bond(ctx, L, 5, 5, M, k, seed=3, release=True)
    _, dim = ctx.psi_layout()
    x = workloads.gaussian(dim, 4)
    assert np.array_equal(ctx.hpsi(x), ref.hpsi(x))
    with pytest.raises(binding.DMRGError) as err:
        ctx.release_block(0, k)  # used at the current position
    assert err.value.code == binding.DMRG_EINVAL
    ctx.set_position(k - 1, 1)  # its left block was released
    with pytest.raises(binding.DMRGError) as err:
        ctx.hpsi(workloads.gaussian(dim, 5))
    assert err.value.code == binding.DMRG_ESTATE
    ref.close()
    ctx.close()


def test_set_precision_switches_the_matvec_path():
    L, N, M, k = 10, 10, 200, 4
    h, v = workloads.integrals(L, seed=14)
    ctx = binding.DMRG(h, v, N, 0, M)
    workloads.grow_middle_bond(ctx, L, 5, 5, M, k, seed=6)
    _, dim = ctx.psi_layout()
    x = workloads.gaussian(dim, 7)
    y64 = ctx.hpsi(x)
    for prec, tol in ((binding.PREC_FP32, 2e-6), (binding.PREC_BF16X3, 2e-4)):
        ctx.set_precision(prec)
        assert np.max(np.abs(ctx.hpsi(x) - y64)) <= tol * np.max(np.abs(y64))
    ctx.set_precision(binding.PREC_FP64)
    assert np.array_equal(ctx.hpsi(x), y64)
    with pytest.raises(binding.DMRGError):
        ctx.set_precision(9)
    ctx.close()


def test_asymmetric_bond_dimensions():
    """RDM truncation keeps at most M_forward states in a new left block and
    M_backward in a new right block (dmrg_set_bond_dims); energies variational."""
    L, N = 8, 8
    h, v = workloads.integrals(L, seed=15)
    e_fci = fock.fci_ground(h, v, 4, 4)[0]
    ctx = binding.DMRG(h, v, N, 0, 48)
    ctx.set_bond_dims(48, 20)
    E = ctx.sweep(2, tol=1e-10)
    assert np.all(E >= e_fci - 1e-10)
    ctx.set_position(3, 1)
    assert ctx.block_sectors(0)[:, 2].sum() <= 48
    assert ctx.block_sectors(1)[:, 2].sum() <= 20
    ctx.close()
    # a grown middle bond with a smaller right bond dimension, then one truncation each way
    L, N, M, MR, k = 10, 10, 120, 60, 4
    h, v = workloads.integrals(L, seed=16)
    ctx = binding.DMRG(h, v, N, 0, M)
    workloads.grow_middle_bond(ctx, L, 5, 5, M, k, seed=2, M_right=MR)
    assert ctx.block_sectors(0)[:, 2].sum() == M and ctx.block_sectors(1)[:, 2].sum() == MR
    ctx.set_bond_dims(9, 7)
    ctx.davidson(tol=1e-8, max_iter=300, allow_noconv=True)
    dw, kept = ctx.renormalize(-1)  # new right block: 7 states
    assert kept.sum() == 7 and dw > 0
    ctx.davidson(tol=1e-8, max_iter=300, allow_noconv=True)
    dw, kept = ctx.renormalize(+1)  # new left block: 9 states
    assert kept.sum() == 9 and dw > 0
    ctx.close()
