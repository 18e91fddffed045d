"""e4m3 path on the GPU: per-tile quantization, the block-scaled tensor-core
sketch and GN on e4m3 operands, against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import gn_oracle as O
import gn_synth

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


def npy(t):
    return t.detach().double().cpu().numpy()


def tiled_magnitudes(rows, cols, seed, lo=-8.0, hi=8.0):
    """A factor that is constant on each 128 x 128 tile (exercises the scales)."""
    rng = np.random.default_rng(seed)
    f = np.exp(rng.uniform(lo, hi, (-(-rows // 128), -(-cols // 128))))
    return np.kron(f, np.ones((128, 128)))[:rows, :cols]


@pytest.mark.parametrize("rows,cols", [(300, 260), (256, 384), (97, 1000)])
def test_quantize_e4m3_matches_oracle_bitwise(gn, H, rows, cols):
    rng = np.random.default_rng(rows + cols)
    x = rng.standard_normal((rows, cols)) * tiled_magnitudes(rows, cols, 3)
    x[:128, :128] = 0.0                                  # an all-zero tile
    x[-5:, -7:] *= 1e-30                                  # tiny values (subnormal codes)
    q = H.quantize_e4m3(torch.from_numpy(x).cuda())
    assert H.sync_status() == 0
    vals, exps = O.quantize_e4m3_tiles(x)
    assert np.array_equal(q.scale.cpu().numpy().astype(np.int64) - 127, exps)
    assert np.array_equal(npy(q.values()), vals)
    qt = gn.E4M3Mat(rows, cols, q.scale, None, q.data_t)
    assert np.array_equal(npy(qt.values()), vals)
    # FP32 sources round the same way
    q32 = H.quantize_e4m3(torch.from_numpy(x).float().cuda())
    assert np.array_equal(npy(q32.values()), vals)


def integer_tiled(rows, cols, seed):
    """Integers in [-4, 4] times 1 or 2 per 128 x 128 tile: exact in e4m3 under
    the tile scale (each tile's scale differs with its maximum), and every sum
    of products is an integer far below 2^24, so accumulation is exact."""
    g = torch.Generator().manual_seed(seed)
    v = torch.randint(-4, 5, (rows, cols), generator=g).double()
    t = torch.randint(0, 2, (-(-rows // 128), -(-cols // 128)), generator=g).double()
    return v * torch.kron(1.0 + t, torch.ones(128, 128))[:rows, :cols]   # t in {0, 1}: 2^t = 1 + t


def e4m3_operands(H, A, X, Y):
    return (H.quantize_e4m3(A.cuda(), data=True, transposed=True),
            H.quantize_e4m3(X.cuda(), data=False, transposed=True),
            H.quantize_e4m3(Y.cuda(), data=False, transposed=True))


@pytest.mark.parametrize("m,n,r,l", [(300, 200, 70, 35), (520, 390, 130, 65), (256, 128, 16, 8), (1100, 300, 70, 35)])
def test_e4m3_sketch_exact_on_integer_inputs(gn, H, m, n, r, l):
    A, X, Y = integer_tiled(m, n, 1), integer_tiled(n, r, 2), integer_tiled(m, r + l, 3)
    for t in (A, X, Y):   # the quantization is exact on these inputs
        assert np.array_equal(O.quantize_e4m3_tiles(t.numpy())[0], t.numpy())
    A8, X8, Y8 = e4m3_operands(H, A, X, Y)
    AX = torch.full((m, r), float("nan"), dtype=torch.float32, device="cuda")
    YtA = torch.full((r + l, n), float("nan"), dtype=torch.float32, device="cuda")
    ws = H.workspace(m, n, r, l, gn.E4M3)
    H.sketch(A8, X8, Y8, AX, YtA, ws)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(A.numpy(), X.numpy(), Y.numpy())
    assert np.array_equal(npy(AX), oAX)
    assert np.array_equal(npy(YtA), oYtA)


@pytest.mark.parametrize("r", [1000, 780])
def test_e4m3_sketch_large_sampled(gn, H, r):
    """16384 x 8192, l = r / 2: enough tiles for the 256-row tile shape (r = 780:
    an odd number of AX column tiles, the last one ragged); 64 sampled rows of
    AX and 64 sampled columns of Y^T A against the oracle, bitwise
    (integer-valued inputs as above, drawn on the device)."""
    m, n, l = 16384, 8192, r // 2
    g = torch.Generator(device="cuda").manual_seed(77)
    def draw(rows, cols):
        v = torch.randint(-3, 4, (rows, cols), generator=g, device="cuda", dtype=torch.int8).double()
        t = torch.randint(0, 2, (-(-rows // 128), -(-cols // 128)), generator=g, device="cuda").double()
        return v.mul_((1.0 + t).repeat_interleave(128, 0).repeat_interleave(128, 1)[:rows, :cols])
    A, X, Y = draw(m, n), draw(n, r), draw(m, r + l)
    A8, X8, Y8 = (H.quantize_e4m3(A), H.quantize_e4m3(X, data=False), H.quantize_e4m3(Y, data=False))
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    ws = H.workspace(m, n, r, l, gn.E4M3)
    H.sketch(A8, X8, Y8, AX, YtA, ws)
    assert H.sync_status() == 0
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(m, 64, replace=False))
    cols = np.sort(rng.choice(n, 64, replace=False))
    Xh, Yh = X.cpu().numpy(), Y.cpu().numpy()
    oAX = A[torch.from_numpy(rows).cuda()].cpu().numpy() @ Xh
    oYtA = Yh.T @ A[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    assert np.array_equal(npy(AX)[rows], oAX)
    assert np.array_equal(npy(YtA)[:, cols], oYtA)
    del A, X, Y, AX, YtA, ws
    torch.cuda.empty_cache()


def test_e4m3_sketch_fp32_accumulation_bound(gn, H):
    m, n, r, l = 700, 450, 100, 50
    A = gn_synth.gaussian((m, n), 11, 0) * torch.from_numpy(tiled_magnitudes(m, n, 4, -3, 3))
    X, Y = gn_synth.sketches(m, n, r, l, 12)
    A8, X8, Y8 = e4m3_operands(H, A, X, Y)
    Aq, Xq, Yq = (O.quantize_e4m3_tiles(t.numpy())[0] for t in (A, X, Y))
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    ws = H.workspace(m, n, r, l, gn.E4M3)
    H.sketch(A8, X8, Y8, AX, YtA, ws)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(Aq, Xq, Yq)
    bAX = 2 * n * O.U32 * (np.abs(Aq) @ np.abs(Xq))
    bYA = 2 * m * O.U32 * (np.abs(Yq).T @ np.abs(Aq))
    assert np.all(np.abs(npy(AX) - oAX) <= bAX)
    assert np.all(np.abs(npy(YtA) - oYtA) <= bYA)


def test_e4m3_gn_error_parity(gn, H):
    """GN on e4m3 operands (block-scaled sketch, split-BF16 core product, FP64
    core): against the oracle's GN on the same quantized inputs, ||A_q - A_hat||_F
    within 1.05x; the floor against the unquantized A is the e4m3 storage error."""
    m, n, r, l = 1200, 900, 40, 20
    W1 = gn_synth.gaussian((m, 200), 31, 0) / math.sqrt(200)
    W2 = gn_synth.gaussian((n, 200), 32, 0) / math.sqrt(200)
    s = torch.pow(torch.arange(1, 201, dtype=torch.float64), -2.0)
    A = (W1 * s) @ W2.T + 1e-8 * gn_synth.gaussian((m, n), 33, 0)
    X, Y = gn_synth.sketches(m, n, r, l, 34)
    Aq, Xq, Yq = (O.quantize_e4m3_tiles(t.numpy())[0] for t in (A, X, Y))
    eps = 10 * O.U32
    Ahat_o, parts = O.gn(Aq, Xq, Yq, eps, O.AUTO, eps_relative=True, diag_iters=6)
    err_o = np.linalg.norm(Aq - Ahat_o)
    A8, X8, Y8 = e4m3_operands(H, A, X, Y)
    ws = H.workspace(m, n, r, l, gn.E4M3)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    core = gn.Core.empty(r, l, "cuda")
    F = torch.zeros(m, r, dtype=torch.float64, device="cuda")
    G = torch.zeros(r, n, dtype=torch.float64, device="cuda")
    H.approx(A8, X8, Y8, eps, gn.AUTO | gn.EPS_RELATIVE, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    k = core.k
    Ah = npy(F)[:, :k] @ npy(G)[:k]
    err_g = np.linalg.norm(Aq - Ah)
    assert err_g <= 1.05 * err_o
    floor = np.linalg.norm(A.numpy() - Aq)
    assert np.linalg.norm(A.numpy() - Ah) <= floor + 1.05 * err_o
