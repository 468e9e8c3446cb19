"""Element-wise oracle parity where sector blocks exceed 32 states.

Output blocks larger than 32 x 32 take other kernels than the small ones: the
FP64 and FP32 32 x 32 tile kernel, and the tensor-core kernel (split-BF16 x3)
with several K chunks and ragged tails.  Here the middle bond of L=10/M=300
(largest sector 36) and of L=12/M=800 (largest sector 88) is grown from the
same seeded random O on the GPU and in the operator-based FP64 oracle, and the
GPU's H.psi (Eq. dgemm) and renormalized operators (Eq. renorm_mat) are
compared with the oracle's element by element.

Tolerances, relative to the largest element of the oracle's result:
  FP64        1e-12 (same products, another summation order);
  FP32 ops    5e-6  (operators rounded to FP32, ~2^-24 per product over a few
                     hundred terms per element);
  split-BF16  5e-5  (three bf16 passes keep ~2^-16 of each operand; dropping
                     any one pass gives errors near 2^-8 and fails this bound).
"""
import numpy as np
import pytest

from oracle import baseline
from oracle import dmrg as od
from paper_2001_04890_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

_CACHE = {}


def oracle_case(L, M):
    """Oracle middle bond (seeded O) and its H.psi of one seeded psi, computed once."""
    key = (L, M)
    if key not in _CACHE:
        wl = dict(name=f"l{L}", L=L, N=L, two_sz=0, M=M)
        I, k, lb, rb, nu, nd = baseline.middle_bond(wl)
        hp = od.HPsi(I, k, lb, rb, nu, nd)
        psi = workloads.gaussian(hp.dim, seed=1)
        _CACHE[key] = dict(k=k, lb=lb, rb=rb, psi=psi, ref=hp.apply(psi))
    return _CACHE[key]


def gpu_case(L, M, prec):
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, L, 0, M, precision=prec)
    workloads.grow_middle_bond(ctx, L, L // 2, L // 2, M, (L - 2) // 2, seed=0)
    return ctx


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("L,M", [(10, 300), (12, 800)])
def test_fp64_large_blocks_hpsi_matches_oracle(L, M):
    ref = oracle_case(L, M)
    ctx = gpu_case(L, M, binding.PREC_FP64)
    assert ctx.block_sectors(0)[:, 2].max() > 32 and ctx.block_sectors(1)[:, 2].max() > 32
    blocks, dim = ctx.psi_layout()
    assert dim == len(ref["psi"])
    assert max(blocks[:, 4].max(), blocks[:, 5].max()) > 32  # output blocks for the tile kernel
    for scale in (1.0, -0.5):
        assert _rel(ctx.hpsi(scale * ref["psi"]), scale * ref["ref"]) < 1e-12
    ctx.close()


def _oracle_op(blk, kind, i, j):
    key = {0: ("H",), 1: ("C", i), 2: ("T", i), 3: ("V", i), 4: ("A", i, j), 5: ("B", i, j)}[kind]
    return blk.ops[key]


def _family_shift(kind, i, j):
    up = lambda p: 1 if p % 2 == 0 else 0  # noqa: E731
    if kind == 0:
        return 0, 0
    if kind in (1, 2):
        return up(i), 1 - up(i)
    if kind == 3:
        return -up(i), -(1 - up(i))
    if kind == 4:
        return up(i) + up(j), 2 - up(i) - up(j)
    return up(i) - up(j), (1 - up(i)) - (1 - up(j))


def test_fp64_large_blocks_renormalized_operators_match_oracle():
    """Operators of the L=12/M=800 middle-bond blocks (renormalized through sectors of
    up to 88 states) equal the oracle's, sector block by sector block."""
    L, M = 12, 800
    ref = oracle_case(L, M)
    ctx = gpu_case(L, M, binding.PREC_FP64)
    kl = ref["k"]
    lmodes = list(range(2 * kl))
    rmodes = list(range(2 * (kl + 2), 2 * L))
    checks = [(0, 0, -1, -1), (0, 1, 3, -1), (0, 1, lmodes[-1], -1), (0, 2, 2 * L - 1, -1),
              (0, 4, 0, lmodes[-1]), (0, 5, lmodes[-2], 1), (1, 0, -1, -1), (1, 1, rmodes[0], -1),
              (1, 3, 0, -1), (1, 4, rmodes[1], rmodes[-1]), (1, 5, rmodes[-1], rmodes[2])]
    checked = 0
    for side, kind, i, j in checks:
        blk = ref["lb"] if side == 0 else ref["rb"]
        try:
            got = ctx.block_op(side, kind, i, j)
        except binding.DMRGError:
            continue  # not stored on this side (formed on the fly)
        ops = _oracle_op(blk, kind, i, j)
        du, dd = _family_shift(kind, i, j)
        parts = []
        for a, (nu, nd) in enumerate(blk.sectors):
            b = blk.sidx.get((nu + du, nd + dd))
            if b is None:
                continue
            parts.append(ops.get((b, a), np.zeros((blk.dims[b], blk.dims[a]))).ravel())
        want = np.concatenate(parts)
        assert got.shape == want.shape, (side, kind, i, j)
        assert _rel(got, want) < 1e-12, (side, kind, i, j)
        checked += 1
    assert checked >= 8
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(binding.PREC_FP32, 5e-6), (binding.PREC_BF16X3, 5e-5)])
def test_mixed_large_blocks_hpsi_matches_oracle(prec, tol):
    """FP32 tile kernel and tensor-core kernel (blocks of 33..88 states, several K
    chunks, ragged tails) against the oracle, over two calls with different psi
    (the tensor-core psi tiles are rebuilt per call)."""
    L, M = 12, 800
    ref = oracle_case(L, M)
    ctx = gpu_case(L, M, prec)
    for scale in (1.0, -0.5):
        err = _rel(ctx.hpsi(scale * ref["psi"]), scale * ref["ref"])
        assert err < tol, err
    ctx.close()


def test_fp32_renormalization_matches_oracle_to_fp32_accuracy():
    """dmrg_set_renorm_precision(FP32): every renormalization of the L=10/M=300 growth
    runs its products in FP32 (errors compound over the growth steps); the middle-bond
    operators and H.psi stay within 5e-6 of the FP64 oracle's."""
    L, M = 10, 300
    ref = oracle_case(L, M)
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, L, 0, M)
    ctx.set_renorm_precision(binding.PREC_FP32)
    workloads.grow_middle_bond(ctx, L, L // 2, L // 2, M, (L - 2) // 2, seed=0)
    assert _rel(ctx.hpsi(ref["psi"]), ref["ref"]) < 5e-6
    got = ctx.block_op(0, 0)  # the left block's Hamiltonian
    blk = ref["lb"]
    want = np.concatenate([blk.ops[("H",)].get((a, a), np.zeros((d, d))).ravel()
                           for a, d in enumerate(blk.dims)])
    err = _rel(got, want)
    assert 1e-12 < err < 5e-6, err  # FP32 rounding is present, and bounded
    ctx.close()
