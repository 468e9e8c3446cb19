"""dmrg_hpsi_noalloc: H.psi with its scratch in the library's fixed device array.

For callers that cannot allocate device memory when they need H.psi (a device
memory budget reserved up front, or a latency-critical path that must not
block on the allocator).  Its result must equal dmrg_hpsi's on the same psi,
call after call (the shared array keeps the previous call's contents, which
each call must clear before use), in every working precision: the FP64 and
FP32 chunk kernels and the tensor-core kernel all write their partials into
the array.  A position whose partials do not fit is refused.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2001_04890_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


def _context(prec):
    L, N, M = 10, 10, 96
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, 0, M, precision=prec)
    workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, (L - 2) // 2, seed=0)
    if prec == binding.PREC_BF16X3:
        ctx.set_tune(tc_min=1)  # every block on the tensor cores
    return ctx


@pytest.mark.parametrize("prec", [binding.PREC_FP64, binding.PREC_FP32, binding.PREC_BF16X3])
def test_noalloc_hpsi_matches_hpsi_on_two_calls_in_a_row(prec):
    import torch
    ctx = _context(prec)
    _, dim = ctx.psi_layout()
    psi = torch.from_numpy(workloads.gaussian(dim, seed=3)).cuda()
    # no task list yet at this position: refused without touching the GPU
    with pytest.raises(binding.DMRGError) as err:
        ctx.hpsi_noalloc(psi, torch.empty_like(psi))
    assert err.value.code == binding.DMRG_ESTATE
    ref = ctx.hpsi(psi).cpu().numpy()  # the existing entry point builds the task list
    for _ in range(2):
        sigma = torch.full_like(psi, float("nan"))
        ctx.hpsi_noalloc(psi, sigma)
        ctx.check_status()
        got = sigma.cpu().numpy()
        # same task list and chunking as dmrg_hpsi, only the partials live elsewhere
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert binding.lib().dmrg_hpsi_noalloc_capacity() == 1 << 21
    ctx.close()


def test_noalloc_refuses_a_position_beyond_its_capacity():
    import torch
    ctx = _context(binding.PREC_FP64)
    ctx.set_tune(target_chunks=1e7, min_chunk=0.0)  # one chunk per task: far more partials
    _, dim = ctx.psi_layout()
    psi = torch.from_numpy(workloads.gaussian(dim, seed=4)).cuda()
    ctx.hpsi(psi)
    sigma = torch.full_like(psi, float("nan"))
    with pytest.raises(binding.DMRGError) as err:
        ctx.hpsi_noalloc(psi, sigma)
    assert err.value.code == binding.DMRG_EINVAL
    assert "no-allocation scratch holds" in str(err.value)
    assert torch.isnan(sigma).all()  # untouched
    with pytest.raises(ValueError):  # wrong length: refused before any launch
        ctx.hpsi_noalloc(psi[:-1], sigma[:-1])
    ctx.close()
