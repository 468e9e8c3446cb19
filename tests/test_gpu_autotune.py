"""Launch-shape autotuning of H.psi task lists (context and batch).

A different split granularity or tensor-core routing changes only the
floating-point summation order: H.psi after tuning equals H.psi before it to
rounding (1e-12 relative in FP64, split-BF16 accuracy in BF16X3), and the
chosen parameters are one of the candidates and are kept by the context.
"""
import numpy as np
import pytest

from paper_2001_04890_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(binding.PREC_FP64, 1e-12), (binding.PREC_BF16X3, 2e-4)])
def test_autotune_keeps_hpsi(prec, tol):
    L, N, M = 12, 12, 400
    k = (L - 2) // 2
    h, v = workloads.integrals(L, seed=0)
    ref_ctx = binding.DMRG(h, v, N, 0, M, precision=binding.PREC_FP64)
    workloads.grow_middle_bond(ref_ctx, L, N // 2, N // 2, M, k, seed=0)
    _, dim = ref_ctx.psi_layout()
    psi = workloads.gaussian(dim, seed=3)
    ref = ref_ctx.hpsi(psi)
    ref_ctx.close()
    ctx = binding.DMRG(h, v, N, 0, M, precision=prec)
    workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, k, seed=0)
    before = ctx.hpsi(psi)
    ms, par = ctx.autotune(reps=1)
    assert ms > 0
    assert par["target_chunks"] in (2048.0, 8192.0, 32768.0, 131072.0)
    assert par["min_chunk"] in (5.0e4, 2.0e5)
    assert par["tc_min"] in ((1, 9, 17, 33, 49, 65) if prec == binding.PREC_BF16X3 else (33,))
    assert par["by_work"] in (0, 1) and par["flat_wide"] in (0, 1)
    assert par["tc_tiny"] in ((0, 1) if prec == binding.PREC_BF16X3 else (0,))
    assert ctx.get_tune() == par
    after = ctx.hpsi(psi)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(after - ref)) <= tol * scale
    assert np.max(np.abs(before - ref)) <= tol * scale
    # an explicit shape: everything on the tensor cores that fits (BF16X3), fine chunks
    ctx.set_tune(target_chunks=32768, min_chunk=5e4, tc_min=1, by_work=1, flat_wide=0)
    again = ctx.hpsi(psi)
    assert np.max(np.abs(again - ref)) <= tol * scale
    # the same with the small blocks on the 32-column tensor-core shape (a launch of its own)
    ctx.set_tune(target_chunks=32768, min_chunk=5e4, tc_min=1, by_work=1, flat_wide=0, tc_tiny=1)
    assert ctx.get_tune()["tc_tiny"] == 1
    tiny = ctx.hpsi(psi)
    assert np.max(np.abs(tiny - ref)) <= tol * scale
    ctx.close()


def test_batch_autotune_keeps_hpsi():
    ctxs, psis, refs = [], [], []
    for seed, (L, M) in enumerate([(8, 40), (12, 320), (9, 64)]):
        h, v = workloads.integrals(L, seed=seed)
        tsz = L % 2
        c = binding.DMRG(h, v, L, tsz, M, precision=binding.PREC_BF16X3)
        workloads.grow_middle_bond(c, L, (L + tsz) // 2, (L - tsz) // 2, M, (L - 2) // 2, seed=seed)
        _, dim = c.psi_layout()
        psis.append(workloads.gaussian(dim, seed=20 + seed))
        refs.append(c.hpsi(psis[-1]))
        ctxs.append(c)
    batch = binding.Batch(ctxs)
    x = np.concatenate(psis)
    y0 = batch.hpsi(x)
    ms, par = batch.autotune(reps=1)
    assert ms > 0 and par["tc_min"] in (1, 9, 17, 33, 49, 65)
    for _ in range(2):  # direct run after tuning, then a graph replay
        y = batch.hpsi(x)
        for i, r in enumerate(refs):
            s = slice(batch.offsets[i], batch.offsets[i + 1])
            assert np.max(np.abs(y[s] - r)) <= 1e-4 * np.max(np.abs(r))
            assert np.max(np.abs(y0[s] - r)) <= 1e-4 * np.max(np.abs(r))
    batch.close()
    for c in ctxs:
        c.close()
