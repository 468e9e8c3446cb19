"""dmrg_hpsi_noalloc: H.psi with its scratch in the library's fixed device array.

For callers that cannot allocate device memory when they need H.psi (a device
memory budget reserved up front, or a latency-critical path that must not
block on the allocator).  Its result must equal dmrg_hpsi's on the same psi,
call after call (the shared array keeps the previous call's contents, which
each call must clear before use).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2001_04890_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


def test_noalloc_hpsi_matches_hpsi_on_two_calls_in_a_row():
    import torch
    L, N, M = 10, 10, 96
    k = (L - 2) // 2
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, 0, M)
    workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, k, seed=0)
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
        got = sigma.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert binding.lib().dmrg_hpsi_noalloc_capacity() == 1 << 21
    ctx.close()
