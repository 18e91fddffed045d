"""Sparse A with CountSketch sketches (Section 2.5's input-sparsity route,
Section 7's sparse experiment) through the C ABI: the O(nnz) sketch kernel
against the oracle's CountSketch products on the seeded sparse stand-in
(bit-exact on integer values, FP64 within the reordering of atomic sums
otherwise), GN on the sketch state against the oracle, and the device-side
index checks (an out-of-range bucket latches GN_ERR_INVALID_ARG and skips that
entry)."""
import numpy as np
import pytest
import torch

import gn_synth
from oracle import gn_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_11392_gb300 as g
    return g


@pytest.fixture(scope="module")
def H(gn):
    return gn.Handle()


def _csr(m, n, k, per_row, seed, integer=False):
    rows, cols, vals = gn_synth.sparse_lowrank_plus_noise(m, n, k, per_row, seed=seed)
    if integer:   # small integers: every sum exact in FP64 and FP32
        g = torch.Generator().manual_seed(seed)
        vals = torch.randint(-3, 4, (vals.numel(),), generator=g).double()
    A = O.sparse_from_coo(m, n, rows.numpy(), cols.numpy(), vals.numpy())
    A.sort_indices()
    return A


def _dev(A, dtype=torch.float64):
    crow = torch.from_numpy(A.indptr.astype(np.int64)).cuda()
    col = torch.from_numpy(A.indices.astype(np.int32)).cuda()
    vals = torch.from_numpy(A.data).to(dtype).cuda()
    return crow, col, vals


def _draws(m, n, r, l, seed):
    bx, sx = gn_synth.countsketch_draws(n, r, seed=seed)
    by, sy = gn_synth.countsketch_draws(m, r + l, seed=seed + 1)
    return bx, sx, by, sy


@pytest.mark.parametrize("integer", [True, False])
def test_countsketch_sketches_against_oracle(gn, H, integer):
    m, n, r, l = 3000, 2500, 40, 20
    A = _csr(m, n, 30, 6, seed=5, integer=integer)
    bx, sx, by, sy = _draws(m, n, r, l, 9)
    AX = torch.full((m, r), float("nan"), dtype=torch.float64, device="cuda")
    YtA = torch.full((r + l, n), float("nan"), dtype=torch.float64, device="cuda")
    H.sketch_csr_countsketch(*_dev(A), (m, n), bx.cuda(), sx.cuda(), by.cuda(), sy.cuda(), AX, YtA)
    assert H.sync_status() == 0
    oAX = O.countsketch_apply_right(A, bx.numpy(), sx.numpy(), r)
    oYtA = O.countsketch_apply_right(A.T.tocsr(), by.numpy(), sy.numpy(), r + l).T
    if integer:
        assert np.array_equal(AX.cpu().numpy(), oAX)
        assert np.array_equal(YtA.cpu().numpy(), oYtA)
    else:
        # the same products summed in another order: a few units of roundoff per entry
        absA = abs(A)
        bAX = O.countsketch_apply_right(absA, bx.numpy(), np.ones(n), r)
        bYtA = O.countsketch_apply_right(absA.T.tocsr(), by.numpy(), np.ones(m), r + l).T
        assert np.all(np.abs(AX.cpu().numpy() - oAX) <= 8 * 2.0 ** -53 * 20 * bAX + 1e-300)
        assert np.all(np.abs(YtA.cpu().numpy() - oYtA) <= 8 * 2.0 ** -53 * 60 * bYtA + 1e-300)


def test_countsketch_fp32_values(gn, H):
    m, n, r, l = 2000, 1800, 32, 16
    A = _csr(m, n, 20, 5, seed=6, integer=True)
    bx, sx, by, sy = _draws(m, n, r, l, 19)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    H.sketch_csr_countsketch(*_dev(A, torch.float32), (m, n), bx.cuda(), sx.cuda(), by.cuda(), sy.cuda(), AX, YtA)
    assert H.sync_status() == 0
    assert np.array_equal(AX.double().cpu().numpy(), O.countsketch_apply_right(A, bx.numpy(), sx.numpy(), r))
    assert np.array_equal(YtA.double().cpu().numpy(),
                          O.countsketch_apply_right(A.T.tocsr(), by.numpy(), sy.numpy(), r + l).T)


def test_gn_on_countsketch_state_matches_oracle(gn, H):
    """The sketch state of the sparse stand-in, then the FP64 core and factors:
    the approximant against the oracle's GN on the dense matrix with the dense
    CountSketch matrices (1e-10), and the dense CountSketch matrix itself."""
    m, n, r, l = 1500, 1200, 30, 15
    A = _csr(m, n, 20, 8, seed=7)
    bx, sx, by, sy = _draws(m, n, r, l, 29)
    X = H.countsketch_matrix(n, r, bx.cuda(), sx.cuda())
    assert np.array_equal(X.cpu().numpy(), O.countsketch(n, r, bx.numpy(), sx.numpy()))
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    H.sketch_csr_countsketch(*_dev(A), (m, n), bx.cuda(), sx.cuda(), by.cuda(), sy.cuda(), AX, YtA)
    ws = H.workspace(m, n, r, l, gn.F64)
    core = gn.Core.empty(r, l, "cuda")
    H.core(YtA, X, 0.0, gn.PLAIN, core, ws)
    F = torch.empty(m, r, dtype=torch.float64, device="cuda")
    G = torch.empty(r, n, dtype=torch.float64, device="cuda")
    H.factors(AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    Ad = A.toarray()
    Xd = O.countsketch(n, r, bx.numpy(), sx.numpy())
    Yd = O.countsketch(m, r + l, by.numpy(), sy.numpy())
    ref, _ = O.gn(Ad, Xd, Yd, 0.0, O.PLAIN)
    Ah = (F @ G).cpu().numpy()
    assert np.linalg.norm(Ah - ref) <= 1e-10 * np.linalg.norm(ref)


def test_countsketch_bad_bucket_latched(gn, H):
    """A bucket outside [0, r) is an input error the kernel's own bounds check
    catches: that entry is skipped and GN_ERR_INVALID_ARG is latched; the next
    call with valid draws is exact."""
    m, n, r, l = 500, 400, 16, 8
    A = _csr(m, n, 10, 4, seed=8, integer=True)
    bx, sx, by, sy = _draws(m, n, r, l, 39)
    bad = bx.clone()
    bad[int(A.indices[0])] = r + 5
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    d = _dev(A)
    H.sketch_csr_countsketch(*d, (m, n), bad.cuda(), sx.cuda(), by.cuda(), sy.cuda(), AX, YtA)
    assert H.sync_status() == 1
    H.sketch_csr_countsketch(*d, (m, n), bx.cuda(), sx.cuda(), by.cuda(), sy.cuda(), AX, YtA)
    assert H.sync_status() == 0
    assert np.array_equal(AX.cpu().numpy(), O.countsketch_apply_right(A, bx.numpy(), sx.numpy(), r))


def test_core_with_countsketch_product_given(gn, H):
    """C = (Y^T A) X formed by gn_countsketch_apply (O((r+l) n) work, no dense X)
    and handed to gn_core (GN_CORE_C_GIVEN): the same R and Q as the core that
    forms C from the dense CountSketch matrix, and C against the oracle's."""
    m, n, r, l = 1200, 1000, 24, 12
    A = _csr(m, n, 15, 6, seed=17)
    bx, sx, by, sy = _draws(m, n, r, l, 49)
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    H.sketch_csr_countsketch(*_dev(A), (m, n), bx.cuda(), sx.cuda(), by.cuda(), sy.cuda(), AX, YtA)
    ws = H.workspace(m, n, r, l, gn.F64)
    X = H.countsketch_matrix(n, r, bx.cuda(), sx.cuda())
    c1 = gn.Core.empty(r, l, "cuda")
    H.core(YtA, X, 0.0, gn.PLAIN, c1, ws)
    c2 = gn.Core.empty(r, l, "cuda")
    H.countsketch_apply(YtA, bx.cuda(), sx.cuda(), c2.C)
    H.core(YtA, X, 0.0, gn.PLAIN | gn.CORE_C_GIVEN, c2, ws)
    assert H.sync_status() == 0
    Co = YtA.cpu().numpy() @ O.countsketch(n, r, bx.numpy(), sx.numpy())
    assert np.linalg.norm(c2.C.cpu().numpy() - Co) <= 1e-14 * np.linalg.norm(Co)
    kappa = np.linalg.cond(c1.R.cpu().numpy())
    assert (c2.R - c1.R).norm().item() <= 1e-14 * kappa * c1.R.norm().item()
    assert (c2.Q - c1.Q).norm().item() <= 1e-14 * kappa * c1.Q.norm().item()
