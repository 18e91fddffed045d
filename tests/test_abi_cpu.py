"""Host-side checks of the C ABI that need no GPU: the shared library loads,
exports every entry point declared in include/gn.h, and the host-only sizing
and validation logic behaves."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "gn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gn_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2009_11392_gb300 as gn
    declared = _declared_symbols()
    assert len(declared) >= 15
    assert sorted(gn.ABI_SYMBOLS) == declared
    L = ctypes.CDLL(gn.lib_path())
    for name in declared:
        assert hasattr(L, name), name


def test_status_strings():
    import paper_2009_11392_gb300 as gn
    assert gn.lib.gn_status_string(0) == b"ok"
    assert gn.lib.gn_status_string(7) == b"device-side wait timed out"
    assert gn.lib.gn_status_string(99) == b"unknown status"


def test_workspace_size_validates_shapes():
    import paper_2009_11392_gb300 as gn
    b = ctypes.c_size_t()
    ws = gn.lib.gn_workspace_size
    assert ws(1000, 500, 20, 10, gn.F64, ctypes.byref(b)) == 0 and b.value > 0
    small = b.value
    assert ws(32768, 16384, 1000, 500, gn.BF16, ctypes.byref(b)) == 0 and b.value > small
    assert ws(1000, 500, 0, 10, gn.F64, ctypes.byref(b)) == 2          # r < 1
    assert ws(1000, 500, 501, 10, gn.F64, ctypes.byref(b)) == 2        # r > min(m, n)
    assert ws(1000, 500, 20, 0, gn.F64, ctypes.byref(b)) == 2          # l < 1
    assert ws(1000, 500, 20, 10, gn.F32, ctypes.byref(b)) == 3         # no F32 operand path
    assert ws(1000, 500, 20, 10, gn.F64, None) == 1


def test_null_arguments_rejected_on_host():
    import paper_2009_11392_gb300 as gn
    assert gn.lib.gn_create(None, None) == 1
    assert gn.lib.gn_destroy(None) == 1
    assert gn.lib.gn_sketch(None, None, None, None, None, None, None, 0) == 1
    assert gn.lib.gn_core(None, None, None, 0.0, 0, None, None, 0) == 1
    assert gn.lib.gn_factors(None, None, None, None, None, None, None, 0) == 1
    assert gn.lib.gn_hmt(None, None, None, None, None, None, 0) == 1
    assert gn.lib.gn_sync_status(None) == 1


def test_fp64_tc_workspace_size_is_monotone():
    """Callers size one workspace for their largest product and reuse it for
    smaller ones: the digit-sliced product's workspace must not shrink when M,
    N or K grows (K beyond one pass of 1024 and N beyond one launch's panel
    included)."""
    import paper_2009_11392_gb300 as gn
    b = ctypes.c_size_t()
    f = gn.lib.gn_dgemm_tc_workspace_size
    sizes = [1, 15, 16, 100, 255, 256, 257, 1000, 1024, 1500, 4096, 32768]
    def ws(M, N, K, a32=0):
        assert f(M, N, K, a32, ctypes.byref(b)) == 0
        return b.value
    for M in sizes:
        for N in (1, 32, 128, 256, 1000, 2000):
            last = 0
            for K in (1, 32, 900, 1024, 1025, 3000):
                v = ws(M, N, K)
                assert v >= last and v > 0
                last = v
    for K in (32, 1500):
        for N in (32, 1000):
            vals = [ws(M, N, K) for M in sizes]
            assert vals == sorted(vals)
        for M in (256, 32768):
            vals = [ws(M, N, K) for N in (1, 16, 100, 256, 600, 1000, 5000)]
            assert vals == sorted(vals)
    assert f(10, 10, 0, 0, ctypes.byref(b)) == 1      # K < 1
    assert f(-1, 10, 10, 0, ctypes.byref(b)) == 1
    assert f(10, 10, 10, 0, None) == 1


def test_fp64_tc_arguments_rejected_on_host():
    import paper_2009_11392_gb300 as gn
    L = gn.lib
    assert L.gn_dgemm_tc(None, 4, 4, 4, 1.0, None, 0, 4, 0, None, 4, 0, 0.0, None, 4, None, 0) == 1
    assert L.gn_set_fp64_tc(None, 1) == 1
    assert L.gn_set_fp64_g(None, 1) == 1


def test_apply_and_update_host_validation():
    """gn_apply / gn_update size their scratch and reject bad arguments on the
    host, before any launch."""
    import paper_2009_11392_gb300 as gn
    L = gn.lib
    b = ctypes.c_size_t()
    assert L.gn_apply_workspace_size(1000, 500, 20, 10, 7, 0, ctypes.byref(b)) == 0 and b.value > 0
    small = b.value
    assert L.gn_apply_workspace_size(32768, 16384, 1000, 500, 64, 1, ctypes.byref(b)) == 0 and b.value > small
    assert L.gn_apply_workspace_size(1000, 500, 20, 10, 0, 0, ctypes.byref(b)) == 1     # kw < 1
    assert L.gn_apply_workspace_size(1000, 500, 20, 10, 7, 2, ctypes.byref(b)) == 1     # side not 0 / 1
    assert L.gn_apply_workspace_size(1000, 500, 20, 10, 7, 0, None) == 1
    assert L.gn_apply(None, None, None, None, None, None, 0, None, 0) == 1
    assert L.gn_update_workspace_size(1000, 500, 20, 10, gn.BF16, ctypes.byref(b)) == 0
    upd = b.value
    # the scratch holds E's two sketches in FP32: at least (m r + (r + l) n) floats
    assert upd >= 4 * (1000 * 20 + 30 * 500)
    # blocks of any size are sized: one appended row or column (m or n = 1, r > m)
    assert L.gn_update_workspace_size(1, 500, 20, 10, gn.BF16, ctypes.byref(b)) == 0 and 0 < b.value < upd
    assert L.gn_update_workspace_size(1000, 1, 20, 10, gn.F64, ctypes.byref(b)) == 0 and b.value > 0
    assert L.gn_update_workspace_size(1000, 500, 20, 0, gn.BF16, ctypes.byref(b)) == 0   # l = 0 allowed
    assert L.gn_update_workspace_size(1000, 500, 20, 10, gn.F32, ctypes.byref(b)) == 3  # no F32 operand path
    assert L.gn_update_workspace_size(1000, 500, 0, 10, gn.BF16, ctypes.byref(b)) == 2  # r < 1
    assert L.gn_update_workspace_size(0, 500, 20, 10, gn.BF16, ctypes.byref(b)) == 2   # empty block
    assert L.gn_update(None, None, None, None, None, None, None, 0) == 1


def test_backward_saved_rejects_null_arguments():
    """gn_backward_saved checks its arguments on the host before looking at
    the handle's record of the last front."""
    import paper_2009_11392_gb300 as gn
    L = gn.lib
    assert L.gn_backward_saved(None, None, None, None, None, None, 0) == 1


def test_sketch_state_calls_reject_null_arguments():
    import paper_2009_11392_gb300 as gn
    L = gn.lib
    assert L.gn_resample(None, None, None, None, None, None, None, None, None, 0) == 1
    assert L.gn_append_rows(None, None, None, None, None, None, None, None, 0) == 1
    assert L.gn_append_cols(None, None, None, None, None, None, None, None, 0) == 1


def test_resample_sizing_and_null_workspace():
    """gn_resample_workspace_size accepts dr = 0 or dl = 0 (not both), and
    gn_resample rejects a null workspace on the host even when every matrix
    descriptor is valid (device pointers are never dereferenced on the host)."""
    import paper_2009_11392_gb300 as gn
    L = gn.lib
    b = ctypes.c_size_t()
    f = L.gn_resample_workspace_size
    assert f(1000, 500, 10, 5, gn.F64, ctypes.byref(b)) == 0 and b.value > 0
    assert f(1000, 500, 10, 0, gn.BF16, ctypes.byref(b)) == 0
    assert f(1000, 500, 0, 5, gn.E4M3, ctypes.byref(b)) == 0 and b.value > 0
    assert f(1000, 500, 0, 0, gn.BF16, ctypes.byref(b)) == 2
    assert f(1000, 500, -1, 5, gn.BF16, ctypes.byref(b)) == 2
    assert f(1000, 500, 10, 5, gn.F32, ctypes.byref(b)) == 3
    assert f(1000, 500, 10, 5, gn.F64, None) == 1
    m, n, r, l, dr, dl = 40, 30, 4, 2, 3, 1
    fake = 0x10000   # never dereferenced: the call returns before any launch
    M = lambda rows, cols: gn.GnMat(fake, 0, rows, cols, cols, gn.F64)
    h = ctypes.c_void_p(fake)
    args = [M(m, n), M(n, dr), M(m, dr + dl), M(m, r), M(r + l, n), M(m, r + dr), M(r + l + dr + dl, n)]
    assert L.gn_resample(h, *[ctypes.byref(a) for a in args], None, 1 << 20) == 1
