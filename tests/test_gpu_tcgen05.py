"""Tensor-core (tcgen05) encodings checked on the device against exact integer products."""
import numpy as np
import pytest

from paper_2001_04890_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,K", [(16, 16), (64, 32), (128, 64), (256, 48), (112, 64)])
def test_tcgen05_gemm_exact_on_small_integers(N, K):
    rng = np.random.default_rng(N + K)
    A = rng.integers(-4, 5, size=(128, K)).astype(np.float32)
    B = rng.integers(-4, 5, size=(N, K)).astype(np.float32)
    C = binding.selftest_tcgen05(A, B)
    assert np.array_equal(C, A @ B.T)
