"""Batched independent instances: one grouped, graph-replayed H.psi over several contexts.

Each instance's block of the batched sigma must equal that instance's own
dmrg_hpsi (same tasks, chunked differently: 1e-12 relative in FP64, the
working precision's rounding otherwise), on the first (direct) and later
(CUDA-graph replay) calls; and two instances (the smallest, and the one with
blocks above 32 states) must equal the FP64 oracle's H.psi (Eq. dgemm) at
the tolerance of the precision (1e-12 FP64, 5e-6 FP32 operators, 5e-5 split-BF16
x3, relative to the largest element).
"""
import numpy as np
import pytest

from paper_2001_04890_gb300 import binding, workloads
from tests.helpers import oracle_middle_bond

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [binding.PREC_FP64, binding.PREC_FP32, binding.PREC_BF16X3])
def test_batched_hpsi_equals_per_instance(prec):
    ctxs, oracles = [], {}
    for seed, (L, M) in enumerate([(8, 40), (10, 64), (7, 24), (12, 320)]):  # last: blocks > 32
        h, v = workloads.integrals(L, seed=seed)
        tsz = L % 2  # odd N: lowest |Sz|
        c = binding.DMRG(h, v, L, tsz, M, precision=prec)
        nu, nd, k = (L + tsz) // 2, (L - tsz) // 2, (L - 2) // 2
        workloads.grow_middle_bond(c, L, nu, nd, M, k, seed=seed)
        ctxs.append(c)
        if seed in (0, 3):
            oracles[seed] = oracle_middle_bond(h, v, nu, nd, M, k, seed)
    refs, psis = [], []
    for i, c in enumerate(ctxs):
        _, dim = c.psi_layout()
        psi = workloads.gaussian(dim, seed=10 + i)
        psis.append(psi)
        refs.append(c.hpsi(psi))
    batch = binding.Batch(ctxs)
    assert batch.offsets[-1] == sum(len(p) for p in psis)
    x = np.concatenate(psis)
    # FP32 / tensor-core partials are summed in another chunking: FP32 / split-BF16 rounding
    tol = {binding.PREC_FP64: 1e-12, binding.PREC_FP32: 1e-6, binding.PREC_BF16X3: 1e-4}[prec]
    otol = {binding.PREC_FP64: 1e-12, binding.PREC_FP32: 5e-6, binding.PREC_BF16X3: 5e-5}[prec]
    oref = {i: hp.apply(psis[i]) for i, hp in oracles.items()}
    for _ in range(3):  # direct run, then graph replays
        y = batch.hpsi(x)
        for i, r in enumerate(refs):
            got = y[batch.offsets[i]:batch.offsets[i + 1]]
            assert np.max(np.abs(got - r)) <= tol * np.max(np.abs(r)), i
            if i in oref:
                err = np.max(np.abs(got - oref[i])) / np.max(np.abs(oref[i]))
                assert err <= otol, (i, err)
    batch.close()
    for c in ctxs:
        c.close()


def test_batch_refuses_after_a_member_rebuilds_its_task_list():
    """A batch addresses its contexts' operator copies: after one of them switches
    precision (its copies are released), dmrg_batch_hpsi refuses instead of reading them."""
    ctxs = []
    for seed, (L, M) in enumerate([(8, 40), (10, 64)]):
        h, v = workloads.integrals(L, seed=seed)
        c = binding.DMRG(h, v, L, 0, M, precision=binding.PREC_FP32)
        workloads.grow_middle_bond(c, L, L // 2, L // 2, M, (L - 2) // 2, seed=seed)
        ctxs.append(c)
    batch = binding.Batch(ctxs)
    x = workloads.gaussian(batch.offsets[-1], seed=5)
    y = batch.hpsi(x)
    ctxs[1].set_precision(binding.PREC_BF16X3)
    with pytest.raises(binding.DMRGError) as err:
        batch.hpsi(x)
    assert err.value.code == binding.DMRG_ESTATE
    batch.close()
    ctxs[1].set_precision(binding.PREC_FP32)
    batch = binding.Batch(ctxs)  # created again: same result
    assert np.max(np.abs(batch.hpsi(x) - y)) <= 1e-12 * np.max(np.abs(y))
    batch.close()
    for c in ctxs:
        c.close()
