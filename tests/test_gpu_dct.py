"""Subsampled DCT sketches made on the device (gn_dct_sketch, the sketches of
Section 7's experiments) against the oracle's dct_sketch, and GN with them
through the C ABI against the oracle on the same (quantized) sketches.
Tolerances: the FP64 sketch matrix within 1e-11 absolute (numpy evaluates the
cosine of the unreduced angle, up to pi 2n, which carries an absolute rounding
of about 1e-12); the BF16 one equal to the oracle's entries rounded through
FP32 except where the two FP64 values straddle a rounding boundary; the
FP64 path's approximant within 1e-10 of the oracle's; the BF16 tensor-core
sketches within the FP32 accumulation bound of the oracle's products."""
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


@pytest.mark.parametrize("n,r", [(500, 30), (1000, 1), (4096, 257), (3, 3)])
def test_dct_sketch_matrix_against_oracle(gn, H, n, r):
    signs, cols = gn_synth.dct_sketch_draws(n, r, seed=n + r)
    ref = O.dct_sketch(n, signs.numpy(), cols.numpy())
    X64 = H.dct_sketch(n, signs, cols, dtype=torch.float64)
    assert np.max(np.abs(X64.cpu().numpy() - ref)) <= 1e-11
    Xb = H.dct_sketch(n, signs, cols, dtype=torch.bfloat16)
    got = Xb.double().cpu().numpy()
    want = O.quantize_bf16(ref)
    # where the angle is an odd multiple of pi/2 the cosine is exactly 0: the
    # device reduces the angle exactly and gets 0, numpy's unreduced angle gives
    # about 1e-16; elsewhere a mismatch only where the oracle's FP64 value sits
    # within its 1e-11 of a BF16 rounding boundary (one unit apart)
    exact_zero = np.abs(ref) <= 1e-12
    assert np.all(got[exact_zero] == 0.0)
    diff = (got != want) & ~exact_zero
    assert diff.sum() <= max(1, diff.size // 100000)
    if diff.any():
        assert np.all(np.abs(got[diff] - want[diff]) <= 2.0 ** -7 * np.abs(want[diff]))


def test_gn_fp64_with_dct_sketches_matches_oracle(gn, H):
    """Algorithm 2 with subsampled DCT X, Y (FP64 path) against the oracle's GN
    with its own dct_sketch matrices, and exact recovery of a rank-r input."""
    m, n, r, l = 600, 400, 24, 12
    sx, cx = gn_synth.dct_sketch_draws(n, r, seed=71)
    sy, cy = gn_synth.dct_sketch_draws(m, r + l, seed=72)
    X, Y = H.dct_sketch(n, sx, cx, torch.float64), H.dct_sketch(m, sy, cy, torch.float64)
    p = gn_synth.config2(m=m, n=n, r=r, l=l)
    A = p.a.numpy()
    Xo, Yo = X.cpu().numpy(), Y.cpu().numpy()
    ref, _ = O.gn(A, Xo, Yo, 0.0, O.PLAIN)
    ws = H.workspace(m, n, r, l, gn.F64)
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    F = torch.empty(m, r, dtype=torch.float64, device="cuda")
    G = torch.empty(r, n, dtype=torch.float64, device="cuda")
    core = gn.Core.empty(r, l, "cuda")
    H.approx(torch.from_numpy(A).cuda(), X, Y, 0.0, gn.PLAIN, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    Ah = (F @ G).cpu().numpy()
    assert np.linalg.norm(Ah - ref) <= 1e-10 * np.linalg.norm(ref)
    # exact recovery of a rank-r matrix with DCT sketches (Section 2)
    rng = np.random.default_rng(3)
    B = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    H.approx(torch.from_numpy(B).cuda(), X, Y, 0.0, gn.PLAIN, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    assert np.linalg.norm((F @ G).cpu().numpy() - B) <= 1e-11 * np.linalg.norm(B)


def test_tensor_core_sketch_with_dct_sketches(gn, H):
    """BF16 DCT sketches on the tensor cores: AX and Y^T A within the FP32
    accumulation bound of the oracle's products of the same BF16 operands, over
    several tiles and ragged tails."""
    m, n, r, l = 1100, 900, 100, 50
    sx, cx = gn_synth.dct_sketch_draws(n, r, seed=81)
    sy, cy = gn_synth.dct_sketch_draws(m, r + l, seed=82)
    Xb, Yb = H.dct_sketch(n, sx, cx), H.dct_sketch(m, sy, cy)
    A = gn_synth.gaussian((m, n), 83, 0)
    Ab = H.quantize(A.cuda())
    Aq = Ab.double().cpu().numpy()
    Xq, Yq = Xb.double().cpu().numpy(), Yb.double().cpu().numpy()
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(Aq, Xq, Yq)
    u = 2.0 ** -24
    assert np.all(np.abs(AX.double().cpu().numpy() - oAX) <= 2 * n * u * (np.abs(Aq) @ np.abs(Xq)))
    assert np.all(np.abs(YtA.double().cpu().numpy() - oYtA) <= 2 * m * u * (np.abs(Yq).T @ np.abs(Aq)))
