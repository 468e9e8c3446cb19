"""Full-size parity: the L=24, N=24, M=512 middle-bond H.psi that bench.py times, element by element.

Both sides grow the middle-bond blocks from the same seeded random O (drawn
from each side's own enlarged layouts, which must agree); the operator-based
FP64 oracle then applies H to the same psi.  Tolerance 1e-12 relative (FP64,
different summation order).
"""
import numpy as np
import pytest

from oracle import baseline
from oracle import dmrg as od
from paper_2001_04890_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

WL = dict(name="L24_N24_Sz0_M512_fp64_middle_bond", L=24, N=24, two_sz=0, M=512)


def test_fullsize_middle_bond_hpsi_matches_oracle():
    L, N, M = WL["L"], WL["N"], WL["M"]
    k = (L - 2) // 2
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, 0, M)
    workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, k, seed=0)
    I, k2, lb, rb, nu, nd = baseline.middle_bond(WL)
    assert k2 == k
    tl, tr = baseline.sector_tables(lb, rb)
    assert np.array_equal(ctx.block_sectors(0), np.array(tl))
    assert np.array_equal(ctx.block_sectors(1), np.array(tr))
    hp = od.HPsi(I, k, lb, rb, nu, nd)
    blocks, dim = ctx.psi_layout()
    assert dim == hp.dim
    psi = workloads.gaussian(dim, seed=1)
    ref = hp.apply(psi)
    got = ctx.hpsi(psi)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    # the host-only planner counts the same task list as the context
    assert binding.plan_hpsi_flops(h, v, N, 0, k, tl, tr)[0] == ctx.hpsi_flops()[0]
    ctx.close()


def test_l40_m2000_middle_bond_properties():
    """At the L=40/M=2000 workload (too large for the oracle): H.psi is Hermitian
    in FP64 and the tensor-core and FP32 paths agree with it to their accuracy."""
    from paper_2001_04890_gb300 import binding, workloads
    import numpy as np
    L, N, M = 40, 40, 2000
    k = (L - 2) // 2
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, 0, M)
    workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, k, seed=0, release=True)
    _, dim = ctx.psi_layout()
    x, y = workloads.gaussian(dim, 1), workloads.gaussian(dim, 2)
    hx, hy = ctx.hpsi(x), ctx.hpsi(y)
    assert abs(x @ hy - y @ hx) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(hy)
    for prec, tol in ((binding.PREC_FP32, 2e-6), (binding.PREC_BF16X3, 2e-4)):
        ctx.set_precision(prec)
        ctx.set_tune(tc_min=1)
        assert np.max(np.abs(ctx.hpsi(x) - hx)) <= tol * np.max(np.abs(hx))
    ctx.close()
