"""The allocation-free error entry point, through the C ABI.

gn_error_fro2_noalloc serves callers that cannot allocate device memory: it
keeps its partial sums in a fixed device array inside the library instead of
a caller workspace.  It must give the same result as gn_error_fro2 (same
kernels, same summation order) on consecutive calls, whose shared array keeps
the previous call's contents.  This file is collected last on purpose.
"""
import ctypes

import pytest
import torch

import gn_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_11392_gb300 as g
    return g


def test_noalloc_error_matches_workspace_version_twice(gn):
    H = gn.Handle()
    torch.cuda.synchronize()
    cases = [(700, 500, 40), (333, 129, 17)]
    for m, n, k in cases:
        A = gn_synth.gaussian((m, n), 51, 0).cuda()
        F = gn_synth.gaussian((m, k), 52, 0).cuda()
        G = gn_synth.gaussian((k, n), 53, 0).cuda() * 0.1
        ws = H.workspace(m, n, min(k, m, n), 1, gn.F64)
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        H.error_fro2(A, F, G, ref, ws)
        outs = []
        for _ in range(2):   # two calls in a row on the shared array
            o = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            H.error_fro2_noalloc(A, F, G, o)
            outs.append(o)
        torch.cuda.synchronize()
        assert H.sync_status() == 0
        r = ref.item()
        for o in outs:
            assert abs(o.item() - r) <= 1e-12 * r
        # and the value itself: ||A - F G||_F^2 from torch in FP64
        assert abs(outs[-1].item() - torch.sum((A - F @ G) ** 2).item()) <= 1e-10 * r
    # beyond the fixed capacity: rejected on the host, nothing launched
    big = gn.GnMat(1, 0, 8192 + 64, 8192, 8192, gn.F64)
    f = gn.GnMat(1, 0, 8192 + 64, 4, 4, gn.F64)
    g = gn.GnMat(1, 0, 4, 8192, 8192, gn.F64)
    st = gn.lib.gn_error_fro2_noalloc(H.h, ctypes.byref(big), ctypes.byref(f), ctypes.byref(g),
                                      ctypes.c_void_p(1))
    assert st == 2   # GN_ERR_SHAPE
    H.close()
