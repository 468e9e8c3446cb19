"""Thin ctypes binding of the C ABI in include/dmrg_gb300.h (argument marshalling only).

Every step of the hot path runs inside libdmrg_gb300.so (CUDA kernels for
sm_103a plus its host planner); this module only converts Python / numpy /
torch arguments to pointers and sizes.  There is no fallback: if the shared
library is missing the import of the handle fails with an error that says how
to build it.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdmrg_gb300.so")

DMRG_OK, DMRG_EINVAL, DMRG_ENOMEM, DMRG_ECUDA, DMRG_ENOCONV, DMRG_ESTATE, DMRG_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
PREC_FP64, PREC_FP32, PREC_BF16X3 = 0, 1, 2

_lib = None


class DMRGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dmrg error {code}: {msg}")
        self.code = code


def lib():
    """Load libdmrg_gb300.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not found: run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p
    llp = C.POINTER(C.c_longlong)
    sig = {
        "dmrg_last_error": (C.c_char_p, []),
        "dmrg_init": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, vp, C.POINTER(vp)]),
        "dmrg_free": (C.c_int, [vp]),
        "dmrg_set_position": (C.c_int, [vp, C.c_int, C.c_int]),
        "dmrg_get_position": (C.c_int, [vp, ip, ip]),
        "dmrg_psi_layout": (C.c_int, [vp, ip, ip, llp]),
        "dmrg_block_sectors": (C.c_int, [vp, C.c_int, ip, ip]),
        "dmrg_enlarged_layout": (C.c_int, [vp, C.c_int, ip, ip]),
        "dmrg_hpsi": (C.c_int, [vp, vp, vp, C.c_int]),
        "dmrg_hpsi_flops": (C.c_int, [vp, dp, llp]),
        "dmrg_hpsi_noalloc": (C.c_int, [vp, vp, vp]),
        "dmrg_hpsi_noalloc_capacity": (C.c_longlong, []),
        "dmrg_check_status": (C.c_int, [vp]),
        "dmrg_debug_set_wait_limit": (C.c_int, [C.c_longlong]),
        "dmrg_debug_fail_alloc": (C.c_int, [C.c_longlong]),
        "dmrg_set_psi": (C.c_int, [vp, vp, C.c_int]),
        "dmrg_get_psi": (C.c_int, [vp, vp, C.c_int]),
        "dmrg_davidson": (C.c_int, [vp, C.c_double, C.c_int, dp, ip]),
        "dmrg_davidson_lowp": (C.c_int, [vp, C.c_double, C.c_int, dp, ip]),
        "dmrg_renormalize": (C.c_int, [vp, C.c_int, ip, dp, dp]),
        "dmrg_sweep": (C.c_int, [vp, C.c_int, C.c_double, dp]),
        "dmrg_block_op": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, dp, llp]),
        "dmrg_release_block": (C.c_int, [vp, C.c_int, C.c_int]),
        "dmrg_set_precision": (C.c_int, [vp, C.c_int]),
        "dmrg_set_bond_dims": (C.c_int, [vp, C.c_int, C.c_int]),
        "dmrg_stats": (C.c_int, [vp, C.c_int, dp, llp, dp, llp, llp, llp, dp]),
        "dmrg_plan_hpsi_flops": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, ip,
                                           C.c_int, ip, dp, llp]),
        "dmrg_selftest_tcgen05": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                            C.POINTER(C.c_float)]),
        "dmrg_batch_create": (C.c_int, [C.c_int, C.POINTER(vp), C.POINTER(vp)]),
        "dmrg_batch_layout": (C.c_int, [vp, llp, dp]),
        "dmrg_batch_hpsi": (C.c_int, [vp, vp, vp, C.c_int]),
        "dmrg_batch_free": (C.c_int, [vp]),
        "dmrg_autotune": (C.c_int, [vp, C.c_int, dp, dp]),
        "dmrg_set_tune": (C.c_int, [vp, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int]),
        "dmrg_get_tune": (C.c_int, [vp, dp]),
        "dmrg_truncation_stats": (C.c_int, [vp, dp, dp, llp, llp]),
        "dmrg_orbital_entropies": (C.c_int, [vp, dp, dp]),
        "dmrg_mutual_information": (C.c_int, [vp, dp, dp, dp]),
        "dmrg_block_basis": (C.c_int, [vp, C.c_int, C.c_int, ip, ip, dp, llp]),
        "dmrg_sweep_record": (C.c_int, [vp, C.c_int, C.c_double, dp, dp, dp]),
        "dmrg_set_davidson": (C.c_int, [vp, C.c_int, C.c_int]),
        "dmrg_set_renorm_precision": (C.c_int, [vp, C.c_int]),
        "dmrg_debug_pair_rdm": (C.c_int, [C.c_int, ip, llp, dp, dp, dp]),
        "dmrg_debug_truncation": (C.c_int, [C.c_int, ip, dp, C.c_int, ip, ip, dp]),
        "dmrg_batch_autotune": (C.c_int, [vp, C.c_int, dp, dp]),
        "dmrg_debug_pieces": (C.c_int, [C.c_int, dp, dp, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_char_p, C.c_longlong, llp]),
        "dmrg_debug_tasks": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, ip, C.c_int, ip,
                                       C.c_int, ip, C.c_longlong, llp]),
        "dmrg_debug_exec": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, ip, C.c_int, ip,
                                      C.c_int, dp, llp, llp, llp, llp]),
        "dmrg_debug_validate": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, ip, C.c_int, ip,
                                          C.c_int, dp, llp, llp]),
        "dmrg_debug_tc": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, ip, C.c_int, ip, dp,
                                    llp, llp, llp, llp, llp]),
        "dmrg_debug_newops": (C.c_int, [C.c_int, dp, dp, C.c_int, C.c_int, C.c_int,
                                        C.c_char_p, C.c_longlong, llp]),
    }
    for name, (res, args) in sig.items():
        if not hasattr(L, name):
            continue  # reported by the export test; calling it raises AttributeError
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(code):
    if code != DMRG_OK:
        raise DMRGError(code, lib().dmrg_last_error().decode())
    return code


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dump(fn, *args):
    need = C.c_longlong(0)
    _check(fn(*args, None, 0, C.byref(need)))
    buf = C.create_string_buffer(need.value)
    _check(fn(*args, buf, need.value, C.byref(need)))
    return buf.value.decode()


def debug_tasks(h, v, N, two_sz, k, sec_l, sec_r, grouped=False):
    """Host-only H.psi task list: (ntasks, 7) int array (group, m, n, p, q, identity flags, input offset),
    in build order or grouped by output block (the GPU order)."""
    h, v = _f64(h), _f64(v)
    L = h.shape[0]
    tl = np.ascontiguousarray(np.asarray(sec_l, dtype=np.int32).reshape(-1, 3))
    tr = np.ascontiguousarray(np.asarray(sec_r, dtype=np.int32).reshape(-1, 3))
    n = C.c_longlong()
    args = (L, N, two_sz, _dptr(h), _dptr(v), k, len(tl), _iptr(tl), len(tr), _iptr(tr), int(grouped))
    _check(lib().dmrg_debug_tasks(*args, None, 0, C.byref(n)))
    out = np.zeros((n.value, 7), dtype=np.int32)
    _check(lib().dmrg_debug_tasks(*args, _iptr(out), n.value, C.byref(n)))
    return out


def _debug_tune(tune):
    """Launch shape of the host-only plan dumps: target_chunks, min_chunk, tc_min, by_work and
    optionally tc_tiny (0 when omitted), as the 5 doubles the library reads."""
    if tune is None:
        return None
    t = [float(x) for x in tune]
    if len(t) == 4:
        t.append(0.0)
    if len(t) != 5:
        raise ValueError("tune: target_chunks, min_chunk, tc_min, by_work[, tc_tiny]")
    return np.ascontiguousarray(t, dtype=np.float64)


def debug_exec(h, v, N, two_sz, k, sec_l, sec_r, tensor_cores=False, tune=None):
    """Host-only execution plan of the H.psi task list: dict of counts and the arrays
    xs (n, 8), chunks (n, 8) and reduce (n, 8) described in the header."""
    h, v = _f64(h), _f64(v)
    L = h.shape[0]
    tl = np.ascontiguousarray(np.asarray(sec_l, dtype=np.int32).reshape(-1, 3))
    tr = np.ascontiguousarray(np.asarray(sec_r, dtype=np.int32).reshape(-1, 3))
    tune_arr = _debug_tune(tune)
    tp = None if tune_arr is None else _dptr(tune_arr)
    cnt = np.zeros(8, dtype=np.int64)
    llp = C.POINTER(C.c_longlong)
    args = (L, N, two_sz, _dptr(h), _dptr(v), k, len(tl), _iptr(tl), len(tr), _iptr(tr), int(tensor_cores), tp)
    _check(lib().dmrg_debug_exec(*args, cnt.ctypes.data_as(llp), None, None, None))
    xs = np.zeros((cnt[0], 8), dtype=np.int64)
    ch = np.zeros((cnt[1] + cnt[2] + cnt[3], 8), dtype=np.int64)
    red = np.zeros((cnt[4], 8), dtype=np.int64)
    _check(lib().dmrg_debug_exec(*args, cnt.ctypes.data_as(llp), xs.ctypes.data_as(llp), ch.ctypes.data_as(llp),
                                 red.ctypes.data_as(llp)))
    keys = ("entries", "tile_chunks", "flat_chunks", "tc_chunks", "reduce_groups", "tiles", "scratch", "reduced")
    return dict(zip(keys, (int(x) for x in cnt))), xs, ch, red


def debug_validate(h, v, N, two_sz, k, sec_l, sec_r, tensor_cores=False, tune=None):
    """Host-only bounds check of the execution plan (and, with tensor_cores, of the
    tensor-core tile plan) for the default or a given launch shape (target_chunks, min_chunk,
    tc_min, by_work[, tc_tiny]): (views checked, violations, first violation)."""
    h, v = _f64(h), _f64(v)
    tl = np.ascontiguousarray(np.asarray(sec_l, dtype=np.int32).reshape(-1, 3))
    tr = np.ascontiguousarray(np.asarray(sec_r, dtype=np.int32).reshape(-1, 3))
    tune_arr = _debug_tune(tune)
    chk, bad = C.c_longlong(), C.c_longlong()
    _check(lib().dmrg_debug_validate(h.shape[0], N, two_sz, _dptr(h), _dptr(v), k, len(tl), _iptr(tl), len(tr),
                                     _iptr(tr), int(tensor_cores), None if tune_arr is None else _dptr(tune_arr),
                                     C.byref(chk), C.byref(bad)))
    return chk.value, bad.value, (lib().dmrg_last_error().decode() if bad.value else "")


def debug_tc(h, v, N, two_sz, k, sec_l, sec_r, tune=None):
    """Host-only tensor-core launch plan: dict of counts and the arrays tasks (n, 14),
    blocks (n, 7), op_tiles (n, 6), psi_tiles (n, 4) described in the header."""
    h, v = _f64(h), _f64(v)
    L = h.shape[0]
    tl = np.ascontiguousarray(np.asarray(sec_l, dtype=np.int32).reshape(-1, 3))
    tr = np.ascontiguousarray(np.asarray(sec_r, dtype=np.int32).reshape(-1, 3))
    tune_arr = _debug_tune(tune)
    tp = None if tune_arr is None else _dptr(tune_arr)
    llp = C.POINTER(C.c_longlong)
    cnt = np.zeros(9, dtype=np.int64)
    args = (L, N, two_sz, _dptr(h), _dptr(v), k, len(tl), _iptr(tl), len(tr), _iptr(tr), tp)
    _check(lib().dmrg_debug_tc(*args, cnt.ctypes.data_as(llp), None, None, None, None))
    te = np.zeros((cnt[0], 14), dtype=np.int64)
    tg = np.zeros((cnt[1], 7), dtype=np.int64)
    ts = np.zeros((cnt[2], 6), dtype=np.int64)
    ps = np.zeros((cnt[3], 4), dtype=np.int64)
    _check(lib().dmrg_debug_tc(*args, cnt.ctypes.data_as(llp), te.ctypes.data_as(llp), tg.ctypes.data_as(llp),
                               ts.ctypes.data_as(llp), ps.ctypes.data_as(llp)))
    keys = ("tasks", "blocks", "op_tiles", "psi_tiles", "op_bytes", "psi_bytes", "shape64x32", "shape64x64",
            "shape128")
    return dict(zip(keys, (int(x) for x in cnt))), te, tg, ts, ps


def plan_hpsi_flops(h, v, N, two_sz, k, sec_l, sec_r):
    """Host-only FLOP count of one H.psi for blocks with the given (n_up, n_dn, dim) sector tables."""
    h, v = _f64(h), _f64(v)
    sl = np.ascontiguousarray(np.asarray(sec_l).reshape(-1, 3), dtype=np.int32)
    sr = np.ascontiguousarray(np.asarray(sec_r).reshape(-1, 3), dtype=np.int32)
    f, t = C.c_double(), C.c_longlong()
    _check(lib().dmrg_plan_hpsi_flops(h.shape[0], N, two_sz, _dptr(h), _dptr(v), k, len(sl), _iptr(sl),
                                      len(sr), _iptr(sr), C.byref(f), C.byref(t)))
    return f.value, t.value


def debug_truncation(spectra, mkeep):
    """Host-only truncation rule of the library on per-sector spectra (each in ascending
    order): (kept per sector, kept columns per sector as ascending-order indices with the
    largest eigenvalue first, trace, kept weight, cut gap)."""
    dims = np.array([len(s) for s in spectra], dtype=np.int32)
    ev = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.float64) for s in spectra])
                              if len(spectra) else np.zeros(0))
    kept = np.zeros(max(len(dims), 1), dtype=np.int32)
    cols = np.zeros(max(int(dims.sum()), 1), dtype=np.int32)
    out3 = np.zeros(3)
    _check(lib().dmrg_debug_truncation(len(dims), _iptr(dims), _dptr(ev), int(mkeep), _iptr(kept), _iptr(cols),
                                       _dptr(out3)))
    kept = kept[:len(dims)]
    per, pos = [], 0
    for n in kept:
        per.append(cols[pos:pos + n].copy())
        pos += n
    return kept, per, out3[0], out3[1], out3[2]


def debug_pair_rdm(layout, psi):
    """Host-only two-orbital matrix and entropies of a two-site wave function given as
    blocks (a, b, c, d, m_a, m_d, offset) and values: (rho2 16 x 16, (s_left, s_right, s_pair))."""
    lay = np.asarray(layout, dtype=np.int64).reshape(-1, 7)
    abcd = np.ascontiguousarray(lay[:, :4], dtype=np.int32)
    offsz = np.ascontiguousarray(np.stack([lay[:, 6], lay[:, 4] * lay[:, 5]], axis=1), dtype=np.int64)
    psi = _f64(psi)
    rho = np.zeros(256)
    s3 = np.zeros(3)
    _check(lib().dmrg_debug_pair_rdm(len(lay), _iptr(abcd), offsz.ctypes.data_as(C.POINTER(C.c_longlong)),
                                     _dptr(psi), _dptr(rho), _dptr(s3)))
    return rho.reshape(16, 16), tuple(s3)


def debug_set_wait_limit(tries):
    """Process-wide polls per pipeline wait of the tensor-core kernel (0: give up at once,
    < 0: the default)."""
    _check(lib().dmrg_debug_set_wait_limit(int(tries)))


def debug_fail_alloc(n):
    """Process-wide: the n-th device allocation from now fails (n <= 0 disarms)."""
    _check(lib().dmrg_debug_fail_alloc(int(n)))


def selftest_tcgen05(A, B):
    """C = A B^T on the tensor cores (A: 128 x K, B: N x K, float32)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    N, K = B.shape
    Cm = np.zeros((128, N), dtype=np.float32)
    fp = C.POINTER(C.c_float)
    _check(lib().dmrg_selftest_tcgen05(N, K, A.ctypes.data_as(fp), B.ctypes.data_as(fp), Cm.ctypes.data_as(fp)))
    return Cm


def debug_pieces(h, v, k, l_empty, r_empty, compress=True):
    h, v = _f64(h), _f64(v)
    return _dump(lib().dmrg_debug_pieces, h.shape[0], _dptr(h), _dptr(v), k, int(l_empty),
                 int(r_empty), int(compress))


def debug_newops(h, v, k, side, old_empty):
    h, v = _f64(h), _f64(v)
    return _dump(lib().dmrg_debug_newops, h.shape[0], _dptr(h), _dptr(v), k, side, int(old_empty))


class DMRG:
    """One two-site DMRG problem on the GPU (wraps a dmrg_ctx)."""

    def __init__(self, h, v, N, two_sz, M, precision=PREC_FP64, stream=None):
        self._h, self._v = _f64(h), _f64(v)
        self.L = self._h.shape[0]
        self.N, self.two_sz, self.M = N, two_sz, M
        ctx = C.c_void_p()
        s = C.c_void_p(stream) if stream else None
        _check(lib().dmrg_init(self.L, N, two_sz, _dptr(self._h), _dptr(self._v), M, precision,
                               s, C.byref(ctx)))
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", None):
            lib().dmrg_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_position(self, k, direction=1):
        _check(lib().dmrg_set_position(self.ctx, k, direction))

    def position(self):
        k, d = C.c_int(), C.c_int()
        _check(lib().dmrg_get_position(self.ctx, C.byref(k), C.byref(d)))
        return k.value, d.value

    def psi_layout(self):
        n, dim = C.c_int(), C.c_longlong()
        _check(lib().dmrg_psi_layout(self.ctx, C.byref(n), None, C.byref(dim)))
        blocks = np.zeros(7 * n.value, dtype=np.int32)
        _check(lib().dmrg_psi_layout(self.ctx, C.byref(n), _iptr(blocks), C.byref(dim)))
        return blocks.reshape(n.value, 7), dim.value

    def block_sectors(self, side):
        n = C.c_int()
        _check(lib().dmrg_block_sectors(self.ctx, side, C.byref(n), None))
        out = np.zeros(3 * n.value, dtype=np.int32)
        _check(lib().dmrg_block_sectors(self.ctx, side, C.byref(n), _iptr(out)))
        return out.reshape(n.value, 3)

    def enlarged_layout(self, direction):
        n = C.c_int()
        _check(lib().dmrg_enlarged_layout(self.ctx, direction, C.byref(n), None))
        out = np.zeros(3 * n.value, dtype=np.int32)
        _check(lib().dmrg_enlarged_layout(self.ctx, direction, C.byref(n), _iptr(out)))
        return out.reshape(n.value, 3)

    def hpsi(self, psi):
        """sigma = H psi.  psi: numpy float64 (host path) or a CUDA torch tensor (device path)."""
        if isinstance(psi, np.ndarray):
            psi = _f64(psi)
            sigma = np.empty_like(psi)
            _check(lib().dmrg_hpsi(self.ctx, psi.ctypes.data, sigma.ctypes.data, 0))
            return sigma
        import torch  # device path: torch provides the memory only
        assert psi.is_cuda and psi.dtype == torch.float64 and psi.is_contiguous()
        sigma = torch.empty_like(psi)
        _check(lib().dmrg_hpsi(self.ctx, psi.data_ptr(), sigma.data_ptr(), 1))
        return sigma

    def hpsi_noalloc(self, psi, sigma):
        """sigma = H psi (CUDA torch tensors, float64) without any device allocation in the call.

        The call does not wait for the GPU: check_status() reports a tensor-core
        time-out of the calls made since the last check."""
        import torch
        _, dim = self.psi_layout()
        for name, t in (("psi", psi), ("sigma", sigma)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                    and t.numel() == dim):
                raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of {dim} elements")
        _check(lib().dmrg_hpsi_noalloc(self.ctx, psi.data_ptr(), sigma.data_ptr()))
        return sigma

    def check_status(self):
        """Wait for the context's stream; raise DMRGError (DMRG_ETIMEOUT) if a bounded
        device wait of the work queued since the last check ran out."""
        _check(lib().dmrg_check_status(self.ctx))

    def hpsi_flops(self):
        f, t = C.c_double(), C.c_longlong()
        _check(lib().dmrg_hpsi_flops(self.ctx, C.byref(f), C.byref(t)))
        return f.value, t.value

    def set_psi(self, psi):
        """Set the current wave function from a numpy array or a CUDA torch tensor (float64)."""
        if isinstance(psi, np.ndarray):
            psi = _f64(psi)
            _check(lib().dmrg_set_psi(self.ctx, psi.ctypes.data, 0))
        else:
            _check(lib().dmrg_set_psi(self.ctx, psi.data_ptr(), 1 if psi.is_cuda else 0))

    def get_psi(self, out=None):
        """Copy the current wave function into out (numpy / torch, host or device) or a new numpy array."""
        if out is None:
            _, dim = self.psi_layout()
            out = np.zeros(dim)
        if isinstance(out, np.ndarray):
            _check(lib().dmrg_get_psi(self.ctx, out.ctypes.data, 0))
        else:
            _check(lib().dmrg_get_psi(self.ctx, out.data_ptr(), 1 if out.is_cuda else 0))
        return out

    def davidson(self, tol=1e-9, max_iter=200, allow_noconv=False):
        e, it = C.c_double(), C.c_int()
        code = lib().dmrg_davidson(self.ctx, tol, max_iter, C.byref(e), C.byref(it))
        if code == DMRG_ENOCONV and allow_noconv:
            return e.value, it.value
        _check(code)
        return e.value, it.value

    def davidson_lowp(self, tol=1e-9, max_iter=200, allow_noconv=False):
        """Davidson in the working precision only (no FP64 refinement): (Ritz value, H.psi count)."""
        e, it = C.c_double(), C.c_int()
        code = lib().dmrg_davidson_lowp(self.ctx, tol, max_iter, C.byref(e), C.byref(it))
        if code == DMRG_ENOCONV and allow_noconv:
            return e.value, it.value
        _check(code)
        return e.value, it.value

    def renormalize(self, direction, O=None, kept=None):
        dw = C.c_double()
        if O is None:
            n = len(self.enlarged_layout(direction))
            kept_out = np.zeros(n, dtype=np.int32)
            _check(lib().dmrg_renormalize(self.ctx, direction, _iptr(kept_out), None, C.byref(dw)))
            return dw.value, kept_out
        O = _f64(O)
        kept = np.ascontiguousarray(kept, dtype=np.int32)
        _check(lib().dmrg_renormalize(self.ctx, direction, _iptr(kept), _dptr(O), C.byref(dw)))
        return dw.value, kept

    def sweep(self, nsweeps, tol=1e-9):
        e = np.zeros(nsweeps * 2 * (self.L - 2))
        _check(lib().dmrg_sweep(self.ctx, nsweeps, tol, _dptr(e)))
        return e

    def sweep_record(self, nsweeps, tol=1e-9):
        """Sweeps with per-step records: dict of energies, discarded weights and entropies
        (steps x 3: s_k, s_k+1, s_pair of the step's two sites)."""
        n = nsweeps * 2 * (self.L - 2)
        e, dw, ent = np.zeros(n), np.zeros(n), np.zeros(3 * n)
        _check(lib().dmrg_sweep_record(self.ctx, nsweeps, tol, _dptr(e), _dptr(dw), _dptr(ent)))
        return dict(energies=e, discarded=dw, entropies=ent.reshape(n, 3))

    def stats(self, reset=False):
        ms, calls, fl, launches, dav = C.c_double(), C.c_longlong(), C.c_double(), C.c_longlong(), C.c_longlong()
        dlow, res = C.c_longlong(), C.c_double()
        _check(lib().dmrg_stats(self.ctx, int(reset), C.byref(ms), C.byref(calls), C.byref(fl),
                                C.byref(launches), C.byref(dav), C.byref(dlow), C.byref(res)))
        return dict(hpsi_ms=ms.value, hpsi_calls=calls.value, hpsi_flops=fl.value,
                    kernel_launches=launches.value, davidson_iters=dav.value,
                    davidson_iters_lowp=dlow.value, last_residual=res.value)

    def autotune(self, reps=3):
        """Time candidate launch shapes of this position's H.psi task list; keep the fastest.

        Returns (ms per H.psi with the chosen shape, {target_chunks, min_chunk, tc_min, by_work,
        flat_wide, tc_tiny})."""
        ms = C.c_double()
        par = np.zeros(6)
        _check(lib().dmrg_autotune(self.ctx, reps, C.byref(ms), _dptr(par)))
        return ms.value, _tune_dict(par)

    def set_tune(self, target_chunks=8192.0, min_chunk=2.0e5, tc_min=33, by_work=0, flat_wide=1, tc_tiny=0):
        _check(lib().dmrg_set_tune(self.ctx, float(target_chunks), float(min_chunk), int(tc_min), int(by_work),
                                   int(flat_wide), int(tc_tiny)))

    def get_tune(self):
        par = np.zeros(6)
        _check(lib().dmrg_get_tune(self.ctx, _dptr(par)))
        return _tune_dict(par)

    def block_basis(self, side, sites):
        """(kept per enlarged sector, flat O) of the stored left (0) / right (1) block of `sites`
        sites, in the format dmrg_renormalize takes."""
        n, tot = C.c_int(), C.c_longlong()
        _check(lib().dmrg_block_basis(self.ctx, int(side), int(sites), C.byref(n), None, None, C.byref(tot)))
        kept = np.zeros(max(n.value, 1), dtype=np.int32)
        O = np.zeros(max(tot.value, 1))
        _check(lib().dmrg_block_basis(self.ctx, int(side), int(sites), C.byref(n), _iptr(kept), _dptr(O),
                                      C.byref(tot)))
        return kept[:n.value], O[:tot.value]

    def orbital_entropies(self):
        """Entropies of the two sites of the current wave function (k and k+1): dict with
        s_left, s_right, s_pair and the 16 x 16 two-orbital matrix rho2."""
        s3 = np.zeros(3)
        rho = np.zeros(256)
        _check(lib().dmrg_orbital_entropies(self.ctx, _dptr(s3), _dptr(rho)))
        return dict(s_left=s3[0], s_right=s3[1], s_pair=s3[2], rho2=rho.reshape(16, 16))

    def mutual_information(self, pair_matrices=False):
        """Mutual information of every orbital pair of the wave function at position 0:
        dict with I (L x L), s1 (the L one-orbital entropies) and, if asked, rho (L x L x
        16 x 16 two-orbital matrices, filled for i < j)."""
        L = self.L
        I = np.zeros(L * L)
        s1 = np.zeros(L)
        rho = np.zeros(L * L * 256) if pair_matrices else None
        _check(lib().dmrg_mutual_information(self.ctx, _dptr(I), _dptr(s1),
                                             _dptr(rho) if rho is not None else None))
        out = dict(I=I.reshape(L, L), s1=s1)
        if rho is not None:
            out["rho"] = rho.reshape(L, L, 16, 16)
        return out

    def truncation_stats(self):
        """Record of the density-matrix truncations since init: gap at the cut of the
        last one and the smallest, their count, and how many had a gap below 1e-10."""
        last, low = C.c_double(), C.c_double()
        n, straddled = C.c_longlong(), C.c_longlong()
        _check(lib().dmrg_truncation_stats(self.ctx, C.byref(last), C.byref(low), C.byref(n), C.byref(straddled)))
        return dict(last_gap=last.value, min_gap=low.value, truncations=n.value, straddled=straddled.value)

    def set_davidson(self, refine_keep=0, sweep_max_iter=200):
        """Ritz vectors carried between refinement steps of the mixed-precision Davidson (0: none)
        and the matvec cap of each Davidson step of a sweep."""
        _check(lib().dmrg_set_davidson(self.ctx, int(refine_keep), int(sweep_max_iter)))

    def set_renorm_precision(self, precision):
        """Arithmetic of the renormalization products: PREC_FP64 (default) or PREC_FP32."""
        _check(lib().dmrg_set_renorm_precision(self.ctx, precision))

    def set_bond_dims(self, m_forward, m_backward):
        """Kept states of new left blocks (forward) and new right blocks (backward) in RDM truncations."""
        _check(lib().dmrg_set_bond_dims(self.ctx, int(m_forward), int(m_backward)))

    def set_precision(self, precision):
        """Switch the working precision of the Davidson matvecs (PREC_FP64 / PREC_FP32 / PREC_BF16X3)."""
        _check(lib().dmrg_set_precision(self.ctx, int(precision)))

    def release_block(self, side, sites):
        """Free the stored block of `sites` sites on side 0 (left) / 1 (right)."""
        _check(lib().dmrg_release_block(self.ctx, side, sites))

    def block_op(self, side, kind, i=-1, j=-1):
        n = C.c_longlong()
        _check(lib().dmrg_block_op(self.ctx, side, kind, i, j, None, C.byref(n)))
        out = np.zeros(n.value)
        _check(lib().dmrg_block_op(self.ctx, side, kind, i, j, _dptr(out), C.byref(n)))
        return out


def _tune_dict(par):
    return {"target_chunks": float(par[0]), "min_chunk": float(par[1]), "tc_min": int(par[2]),
            "by_work": int(par[3]), "flat_wide": int(par[4]), "tc_tiny": int(par[5])}


class Batch:
    """Grouped, graph-replayed H.psi over several contexts (each at its current position)."""

    def __init__(self, ctxs):
        arr = (C.c_void_p * len(ctxs))(*[c.ctx.value for c in ctxs])
        h = C.c_void_p()
        _check(lib().dmrg_batch_create(len(ctxs), arr, C.byref(h)))
        self.h, self.n = h, len(ctxs)
        self._ctxs = ctxs
        off = (C.c_longlong * (self.n + 1))()
        fl = C.c_double()
        _check(lib().dmrg_batch_layout(h, off, C.byref(fl)))
        self.offsets = list(off)
        self.flops = fl.value

    def hpsi(self, psi):
        """psi: concatenated float64 vector (numpy, or CUDA torch tensor)."""
        if isinstance(psi, np.ndarray):
            psi = _f64(psi)
            out = np.empty_like(psi)
            _check(lib().dmrg_batch_hpsi(self.h, psi.ctypes.data, out.ctypes.data, 0))
            return out
        import torch
        out = torch.empty_like(psi)
        _check(lib().dmrg_batch_hpsi(self.h, psi.data_ptr(), out.data_ptr(), 1))
        return out

    def autotune(self, reps=3):
        """Time candidate launch shapes of the grouped task list; keep the fastest.

        Returns (ms per batched H.psi with the chosen shape, parameters)."""
        ms = C.c_double()
        par = np.zeros(6)
        _check(lib().dmrg_batch_autotune(self.h, reps, C.byref(ms), _dptr(par)))
        return ms.value, _tune_dict(par)

    def close(self):
        if getattr(self, "h", None):
            lib().dmrg_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
