"""The C-ABI library loads on a machine without a GPU and exports every declared symbol."""
import glob
import os
import re

from paper_2001_04890_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(dmrg_\w+)\s*\(", text))
    return names


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for required in ("dmrg_init", "dmrg_hpsi", "dmrg_renormalize", "dmrg_davidson", "dmrg_sweep",
                     "dmrg_free", "dmrg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = binding.lib()
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_report_errors_without_a_gpu():
    import numpy as np
    L = 3
    h = np.eye(L)
    v = np.zeros((L,) * 4)
    try:
        binding.debug_pieces(h, v, 7, False, False)
    except binding.DMRGError as e:
        assert e.code == binding.DMRG_EINVAL
        assert "bad arguments" in str(e)
    else:
        raise AssertionError("expected an error for an out-of-range position")


def test_tune_calls_reject_bad_arguments_without_a_gpu():
    import ctypes as C
    lib = binding.lib()
    par = (C.c_double * 5)()
    assert lib.dmrg_set_tune(None, 8192.0, 2e5, 33, 0, 1, 0) == binding.DMRG_EINVAL
    assert lib.dmrg_get_tune(None, par) == binding.DMRG_EINVAL
    assert lib.dmrg_autotune(None, 1, None, None) == binding.DMRG_EINVAL
    assert lib.dmrg_batch_autotune(None, 1, None, None) == binding.DMRG_EINVAL
    assert b"dmrg_batch_autotune" in lib.dmrg_last_error()
    assert lib.dmrg_set_bond_dims(None, 10, 10) == binding.DMRG_EINVAL
    assert b"dmrg_set_bond_dims" in lib.dmrg_last_error()
    assert lib.dmrg_truncation_stats(None, None, None, None, None) == binding.DMRG_EINVAL
    assert lib.dmrg_orbital_entropies(None, None, None) == binding.DMRG_EINVAL
    assert lib.dmrg_block_basis(None, 0, 1, None, None, None, None) == binding.DMRG_EINVAL
    assert lib.dmrg_sweep_record(None, 1, 1e-8, None, None, None) == binding.DMRG_EINVAL
    assert lib.dmrg_set_davidson(None, 3, 200) == binding.DMRG_EINVAL


def test_init_rejects_bad_problems_without_a_gpu():
    import ctypes as C
    import numpy as np
    lib = binding.lib()
    L = 4
    h = np.eye(L)
    v = np.zeros((L,) * 4)
    hp = h.ctypes.data_as(C.POINTER(C.c_double))
    vp = v.ctypes.data_as(C.POINTER(C.c_double))
    out = C.c_void_p()
    cases = [(1, 2, 0, 8, 0),      # L < 2
             (L, 9, 1, 8, 0),      # N > 2L
             (L, 4, 1, 8, 0),      # 2Sz parity differs from N
             (L, 4, 6, 8, 0),      # |2Sz| > N
             (L, 6, 4, 8, 0),      # 5 up electrons on 4 orbitals
             (L, 4, 0, 0, 0),      # M < 1
             (L, 4, 0, 8, 7)]      # unknown precision
    for (l, n, sz, m, prec) in cases:
        assert lib.dmrg_init(l, n, sz, hp, vp, m, prec, None, C.byref(out)) == binding.DMRG_EINVAL
        assert not out.value
    hbad = h.copy()
    hbad[1, 2] = np.nan
    assert lib.dmrg_init(L, 4, 0, hbad.ctypes.data_as(C.POINTER(C.c_double)), vp, 8, 0, None,
                         C.byref(out)) == binding.DMRG_EINVAL
    assert b"non-finite" in lib.dmrg_last_error()
