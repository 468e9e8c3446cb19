"""Failure detection without a GPU fault: bounded device waits and allocation failures.

* The tensor-core kernel's pipeline waits are bounded; a wait that runs out
  makes the kernel record the time-out, finish what it has in flight, release
  its tensor memory and return.  dmrg_debug_set_wait_limit(0) makes every such
  wait give up at once (before any copy or MMA is issued), so the report path
  runs deterministically: the call returns DMRG_ETIMEOUT, and with the default
  limit restored the same context computes the right H.psi again.
* A device allocation that fails is injected on the host
  (dmrg_debug_fail_alloc): the call returns DMRG_ENOMEM and the context stays
  usable.
"""
import numpy as np
import pytest

from paper_2001_04890_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


def _tc_context():
    L, N, M = 10, 10, 96
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, 0, M, precision=binding.PREC_BF16X3)
    workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, (L - 2) // 2, seed=0)
    ctx.set_tune(tc_min=1)  # every block on the tensor cores
    return ctx


def test_tensor_core_wait_timeout_is_reported_and_the_context_recovers():
    ctx = _tc_context()
    _, dim = ctx.psi_layout()
    psi = workloads.gaussian(dim, seed=1)
    ref = ctx.hpsi(psi)
    try:
        binding.debug_set_wait_limit(0)
        with pytest.raises(binding.DMRGError) as err:
            ctx.hpsi(psi)
        assert err.value.code == binding.DMRG_ETIMEOUT
        assert "wait ran out" in str(err.value)
    finally:
        binding.debug_set_wait_limit(-1)
    got = ctx.hpsi(psi)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    ctx.close()


def test_noalloc_timeout_is_reported_by_check_status():
    import torch
    ctx = _tc_context()
    _, dim = ctx.psi_layout()
    psi = torch.from_numpy(workloads.gaussian(dim, seed=2)).cuda()
    ref = ctx.hpsi(psi)
    sigma = torch.empty_like(psi)
    try:
        binding.debug_set_wait_limit(0)
        ctx.hpsi_noalloc(psi, sigma)  # returns before the GPU has run it
        with pytest.raises(binding.DMRGError) as err:
            ctx.check_status()
        assert err.value.code == binding.DMRG_ETIMEOUT
    finally:
        binding.debug_set_wait_limit(-1)
    ctx.check_status()  # the report was cleared when read
    ctx.hpsi_noalloc(psi, sigma)
    ctx.check_status()
    assert torch.equal(sigma, ref)
    ctx.close()


def test_injected_allocation_failure_returns_enomem():
    L, N, M = 8, 8, 40
    h, v = workloads.integrals(L, seed=1)
    ctx = binding.DMRG(h, v, N, 0, M)
    workloads.grow_middle_bond(ctx, L, N // 2, N // 2, M, 3, seed=1)
    _, dim = ctx.psi_layout()
    psi = workloads.gaussian(dim, seed=3)
    try:
        binding.debug_fail_alloc(1)  # the first device allocation of the H.psi plan fails
        with pytest.raises(binding.DMRGError) as err:
            ctx.hpsi(psi)
        assert err.value.code == binding.DMRG_ENOMEM
    finally:
        binding.debug_fail_alloc(0)
    sigma = ctx.hpsi(psi)  # the same call succeeds once memory is available
    x = workloads.gaussian(dim, seed=4)
    assert abs(x @ sigma - psi @ ctx.hpsi(x)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(sigma)
    ctx.close()
