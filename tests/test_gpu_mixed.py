"""Mixed precision (DMRG_PREC_FP32): FP32 operator copies for the Davidson matvecs, FP64 elsewhere.

H.psi with FP32 operators agrees with the FP64 oracle to FP32 accuracy; the
Davidson energy, taken as the FP64 Rayleigh quotient of the mixed Ritz
vector, agrees with the FP64 path to far better than 1e-6 Eh (the error is
second order in the vector error).
"""
import numpy as np
import pytest

from oracle import blocks as ob
from paper_2001_04890_gb300 import binding, workloads
from tests.helpers import build_random_position

pytestmark = pytest.mark.gpu


def test_fp32_hpsi_matches_oracle_to_fp32_accuracy():
    L, N, M, k = 6, 6, 40, 2
    h, v = workloads.integrals(L, seed=301)
    ctx = binding.DMRG(h, v, N, 0, M, precision=binding.PREC_FP32)
    lb, rb = build_random_position(ctx, h, v, k, M, seed=3)
    P = ob.Projected(h, v, lb, rb, 3, 3)
    psi = workloads.gaussian(P.dim, seed=4)
    ref = P.apply(psi)
    err = np.max(np.abs(ctx.hpsi(psi) - ref)) / np.max(np.abs(ref))
    assert err < 2e-6, err
    ctx.close()


@pytest.mark.parametrize("L,N,M,k", [(8, 8, 64, 3), (10, 10, 96, 4)])
def test_mixed_energy_matches_fp64(L, N, M, k):
    h, v = workloads.integrals(L, seed=302)
    res = {}
    for prec in (binding.PREC_FP64, binding.PREC_FP32):
        ctx = binding.DMRG(h, v, N, 0, M, precision=prec)
        workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, k, seed=5)
        e, it = ctx.davidson(tol=1e-8, max_iter=400)
        res[prec] = (e, ctx.get_psi())
        ctx.close()
    e64, x64 = res[binding.PREC_FP64]
    e32, x32 = res[binding.PREC_FP32]
    assert abs(e32 - e64) < 1e-8, (e32, e64)
    assert abs(abs(x32 @ x64) - 1.0) < 1e-6


def test_bf16x3_tensor_core_hpsi_matches_oracle():
    """Blocks of 33..128 states run on tcgen05 (split-BF16 x3): ~2^-16 relative accuracy."""
    from oracle import baseline
    from oracle import dmrg as od
    L, N, M = 10, 10, 300
    k = (L - 2) // 2
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, 0, M, precision=binding.PREC_BF16X3)
    workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, k, seed=0)
    sec = ctx.block_sectors(0)
    assert sec[:, 2].max() > 32  # some output blocks take the tensor-core kernel
    wl = dict(name="l10", L=L, N=N, two_sz=0, M=M)
    I, k2, lb, rb, nu, nd = baseline.middle_bond(wl)
    hp = od.HPsi(I, k, lb, rb, nu, nd)
    psi = workloads.gaussian(hp.dim, seed=7)
    ref = hp.apply(psi)
    got = ctx.hpsi(psi)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < 2e-4, err
    e, it = ctx.davidson(tol=1e-8, max_iter=400)
    st = ctx.stats()
    assert st["davidson_iters_lowp"] > 0
    ctx.close()
    ctx64 = binding.DMRG(h, v, N, 0, M, precision=binding.PREC_FP64)
    workloads.grow_middle_bond(ctx64, L, N // 2, N // 2, M, k, seed=0)
    e64, _ = ctx64.davidson(tol=1e-8, max_iter=400)
    ctx64.close()
    assert abs(e - e64) < 1e-8, (e, e64)


@pytest.mark.parametrize("L,M", [(12, 800), (14, 1100)])
def test_bf16x3_tensor_core_hpsi_large_blocks(L, M):
    """Output blocks up to 128 states (several 32-wide K chunks, ragged tails) on the
    tensor cores: H.psi within split-BF16 accuracy of the FP64 path (itself pinned to
    the oracle), over repeated calls (psi tiles rebuilt per call)."""
    N, k = L, (L - 2) // 2
    h, v = workloads.integrals(L, seed=0)
    out = {}
    for prec in (binding.PREC_FP64, binding.PREC_BF16X3):
        ctx = binding.DMRG(h, v, N, 0, M, precision=prec)
        workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, k, seed=0)
        for side in (0, 1):
            dims = ctx.block_sectors(side)[:, 2]
            assert dims.max() > 64 and ((dims > 32) & (dims <= 128)).any()
        _, dim = ctx.psi_layout()
        ys = [ctx.hpsi(workloads.gaussian(dim, seed=s)) for s in (1, 2)]
        out[prec] = ys
        ctx.close()
    for a, b in zip(out[binding.PREC_FP64], out[binding.PREC_BF16X3]):
        err = np.max(np.abs(a - b)) / np.max(np.abs(a))
        assert err < 2e-4, err
