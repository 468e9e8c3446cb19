"""Batched independent instances: one grouped, graph-replayed H.psi over several contexts.

Each instance's block of the batched sigma must equal that instance's own
dmrg_hpsi (same tasks, chunked differently: 1e-12 relative in FP64, the
working precision's rounding otherwise), on the first (direct) and later
(CUDA-graph replay) calls.
"""
import numpy as np
import pytest

from paper_2001_04890_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [binding.PREC_FP64, binding.PREC_FP32, binding.PREC_BF16X3])
def test_batched_hpsi_equals_per_instance(prec):
    ctxs = []
    for seed, (L, M) in enumerate([(8, 40), (10, 64), (7, 24), (12, 320)]):  # last: blocks > 32
        h, v = workloads.integrals(L, seed=seed)
        tsz = L % 2  # odd N: lowest |Sz|
        c = binding.DMRG(h, v, L, tsz, M, precision=prec)
        workloads.grow_middle_bond(c, L, (L + tsz) // 2, (L - tsz) // 2, M, (L - 2) // 2, seed=seed)
        ctxs.append(c)
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
    for _ in range(3):  # direct run, then graph replays
        y = batch.hpsi(x)
        for i, r in enumerate(refs):
            got = y[batch.offsets[i]:batch.offsets[i + 1]]
            assert np.max(np.abs(got - r)) <= tol * np.max(np.abs(r)), i
    batch.close()
    for c in ctxs:
        c.close()
