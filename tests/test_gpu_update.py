"""A <- A + E on the sketch state (gn_update, Section 6): the updated sketches
against the sketches of A + E, and the core of the updated state against the
core of a fresh sketch."""
import numpy as np
import pytest
import torch

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


def npy(t):
    return t.detach().double().cpu().numpy()


def test_update_bf16_exact_on_integer_inputs(gn, H):
    """Integers in [-3, 3] are exact in BF16 and every sum stays an integer below
    2^24: the updated AX, Y^T A equal (A + E) X and Y^T (A + E) bit for bit,
    and the core of the updated state is the core of a fresh sketch of A + E."""
    m, n, r, l = 700, 520, 60, 30
    g = torch.Generator().manual_seed(5)
    draw = lambda a, b: torch.randint(-3, 4, (a, b), generator=g).double()
    A, E, X, Y = draw(m, n), draw(m, n), draw(n, r), draw(m, r + l)
    Ab, Eb, Xb, Yb, ABb = (H.quantize(t.cuda()) for t in (A, E, X, Y, A + E))
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    H.update(Eb, Xb, Yb, AX, YtA)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch((A + E).numpy(), X.numpy(), Y.numpy())
    assert np.array_equal(npy(AX), oAX)
    assert np.array_equal(npy(YtA), oYtA)
    AX2 = torch.empty_like(AX)
    YtA2 = torch.empty_like(YtA)
    H.sketch(ABb, Xb, Yb, AX2, YtA2, ws)
    c1, c2 = gn.Core.empty(r, l, "cuda"), gn.Core.empty(r, l, "cuda")
    H.core(YtA, Xb, 0.0, gn.PLAIN, c1, ws)
    H.core(YtA2, Xb, 0.0, gn.PLAIN, c2, ws)
    assert H.sync_status() == 0
    assert torch.equal(c1.R, c2.R) and torch.equal(c1.Q, c2.Q)


def test_update_fp64_against_oracle(gn, H):
    m, n, r, l = 400, 300, 25, 12
    rng = np.random.default_rng(6)
    A, E = rng.standard_normal((m, n)), 1e-3 * rng.standard_normal((m, n))
    X, Y = rng.standard_normal((n, r)), rng.standard_normal((m, r + l))
    cu = lambda t: torch.from_numpy(t).cuda()
    ws = H.workspace(m, n, r, l, gn.F64)
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    H.sketch(cu(A), cu(X), cu(Y), AX, YtA, ws)
    H.update(cu(E), cu(X), cu(Y), AX, YtA)
    assert H.sync_status() == 0
    AXn, YtAn, _, _ = O.update(*O.sketch(A, X, Y), X, Y, E)
    assert np.linalg.norm(npy(AX) - AXn) <= 1e-13 * np.linalg.norm(AXn)
    assert np.linalg.norm(npy(YtA) - YtAn) <= 1e-13 * np.linalg.norm(YtAn)


def _ints(g, a, b):
    return torch.randint(-3, 4, (a, b), generator=g).double()


def test_resample_bf16_exact_on_integer_inputs(gn, H):
    """Rank r -> r + dr (Section 6): the old sketches copied, A Xd and Yd^T A
    written in place; equal to the sketches with [X, Xd], [Y, Yd] bit for bit."""
    m, n, r, l, dr, dl = 500, 420, 40, 20, 12, 6
    g = torch.Generator().manual_seed(11)
    A, X, Y, Xd, Yd = _ints(g, m, n), _ints(g, n, r), _ints(g, m, r + l), _ints(g, n, dr), _ints(g, m, dr + dl)
    Ab, Xb, Yb, Xdb, Ydb = (H.quantize(t.cuda()) for t in (A, X, Y, Xd, Yd))
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    AXn = torch.full((m, r + dr), float("nan"), dtype=torch.float32, device="cuda")
    YtAn = torch.full((r + l + dr + dl, n), float("nan"), dtype=torch.float32, device="cuda")
    H.resample(Ab, Xdb, Ydb, AX, YtA, AXn, YtAn)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(A.numpy(), torch.cat([X, Xd], 1).numpy(), torch.cat([Y, Yd], 1).numpy())
    assert np.array_equal(npy(AXn), oAX)
    assert np.array_equal(npy(YtAn), oYtA)


def test_append_rows_and_cols_bf16_exact_on_integer_inputs(gn, H):
    """[A; B] and [A, B] (Section 6): the updated sketches equal the sketches of
    the enlarged matrix with the enlarged sketch matrix, bit for bit."""
    m, n, r, l, mb, nb = 460, 380, 36, 18, 70, 54
    g = torch.Generator().manual_seed(12)
    A, X, Y = _ints(g, m, n), _ints(g, n, r), _ints(g, m, r + l)
    Br, Yr = _ints(g, mb, n), _ints(g, mb, r + l)
    Bc, Xc = _ints(g, m, nb), _ints(g, nb, r)
    Ab, Xb, Yb, Brb, Yrb, Bcb, Xcb = (H.quantize(t.cuda()) for t in (A, X, Y, Br, Yr, Bc, Xc))
    ws = H.workspace(m, n, r, l, gn.BF16)

    def fresh():
        AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
        YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
        H.sketch(Ab, Xb, Yb, AX, YtA, ws)
        return AX, YtA

    AX, YtA = fresh()
    AXn = torch.full((m + mb, r), float("nan"), dtype=torch.float32, device="cuda")
    H.append_rows(Brb, Xb, Yrb, AX, YtA, AXn)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(torch.cat([A, Br], 0).numpy(), X.numpy(), torch.cat([Y, Yr], 0).numpy())
    assert np.array_equal(npy(AXn), oAX)
    assert np.array_equal(npy(YtA), oYtA)

    AX, YtA = fresh()
    YtAn = torch.full((r + l, n + nb), float("nan"), dtype=torch.float32, device="cuda")
    H.append_cols(Bcb, Xcb, Yb, AX, YtA, YtAn)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(torch.cat([A, Bc], 1).numpy(), torch.cat([X, Xc], 0).numpy(), Y.numpy())
    assert np.array_equal(npy(AX), oAX)
    assert np.array_equal(npy(YtAn), oYtA)


def _resample_case(gn, H, m, n, r, l, dr, dl, seed):
    """Resample on integer inputs (exact in BF16, sums below 2^24) and compare
    with the sketches of [X, Xd], [Y, Yd] bit for bit."""
    g = torch.Generator().manual_seed(seed)
    A, X, Y = _ints(g, m, n), _ints(g, n, r), _ints(g, m, r + l)
    Xd, Yd = _ints(g, n, dr), _ints(g, m, dr + dl)
    Ab, Xb, Yb, Ydb = (H.quantize(t.cuda()) for t in (A, X, Y, Yd))
    Xdb = H.quantize(Xd.cuda()) if dr > 0 else torch.empty(n, 0, dtype=torch.bfloat16, device="cuda")
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    AXn = torch.full((m, r + dr), float("nan"), dtype=torch.float32, device="cuda")
    YtAn = torch.full((r + l + dr + dl, n), float("nan"), dtype=torch.float32, device="cuda")
    H.resample(Ab, Xdb, Ydb, AX, YtA, AXn, YtAn)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(A.numpy(), torch.cat([X, Xd], 1).numpy(), torch.cat([Y, Yd], 1).numpy())
    assert np.array_equal(npy(AXn), oAX)
    assert np.array_equal(npy(YtAn), oYtA)


@pytest.mark.parametrize("r,dr,dl", [(41, 7, 3), (40, 12, 0), (40, 0, 9)])
def test_resample_odd_r_and_single_sided(gn, H, r, dr, dl):
    """r odd (the new columns of AX start off a 16-byte boundary: scalar
    epilogue), dl = 0 (r raised, l kept) and dr = 0 (l raised alone, Xd has no
    columns and only Yd^T A is formed)."""
    _resample_case(gn, H, 430, 390, r, 20, dr, dl, seed=31 + r + dr + dl)


def test_resample_fp64_against_oracle(gn, H):
    m, n, r, l, dr, dl = 300, 260, 23, 11, 5, 2
    rng = np.random.default_rng(8)
    A, X, Y = rng.standard_normal((m, n)), rng.standard_normal((n, r)), rng.standard_normal((m, r + l))
    Xd, Yd = rng.standard_normal((n, dr)), rng.standard_normal((m, dr + dl))
    cu = lambda t: torch.from_numpy(t).cuda()
    ws = H.workspace(m, n, r, l, gn.F64)
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    H.sketch(cu(A), cu(X), cu(Y), AX, YtA, ws)
    AXn = torch.full((m, r + dr), float("nan"), dtype=torch.float64, device="cuda")
    YtAn = torch.full((r + l + dr + dl, n), float("nan"), dtype=torch.float64, device="cuda")
    H.resample(cu(A), cu(Xd), cu(Yd), AX, YtA, AXn, YtAn)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(A, np.hstack([X, Xd]), np.hstack([Y, Yd]))
    assert np.linalg.norm(npy(AXn) - oAX) <= 1e-13 * np.linalg.norm(oAX)
    assert np.linalg.norm(npy(YtAn) - oYtA) <= 1e-13 * np.linalg.norm(oYtA)


@pytest.mark.parametrize("mb,nb", [(1, 1), (3, 5)])
def test_append_single_rows_and_cols(gn, H, mb, nb):
    """Appending fewer rows than r + l or fewer columns than r (one at a time,
    the usual case of Section 6's appended data): bit for bit against the
    sketches of the enlarged inputs."""
    m, n, r, l = 300, 280, 30, 15
    g = torch.Generator().manual_seed(40 + mb)
    A, X, Y = _ints(g, m, n), _ints(g, n, r), _ints(g, m, r + l)
    Br, Yr = _ints(g, mb, n), _ints(g, mb, r + l)
    Bc, Xc = _ints(g, m, nb), _ints(g, nb, r)
    Ab, Xb, Yb, Brb, Yrb, Bcb, Xcb = (H.quantize(t.cuda()) for t in (A, X, Y, Br, Yr, Bc, Xc))
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    AXn = torch.full((m + mb, r), float("nan"), dtype=torch.float32, device="cuda")
    H.append_rows(Brb, Xb, Yrb, AX, YtA, AXn)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(torch.cat([A, Br], 0).numpy(), X.numpy(), torch.cat([Y, Yr], 0).numpy())
    assert np.array_equal(npy(AXn), oAX)
    assert np.array_equal(npy(YtA), oYtA)

    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    YtAn = torch.full((r + l, n + nb), float("nan"), dtype=torch.float32, device="cuda")
    H.append_cols(Bcb, Xcb, Yb, AX, YtA, YtAn)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(torch.cat([A, Bc], 1).numpy(), torch.cat([X, Xc], 0).numpy(), Y.numpy())
    assert np.array_equal(npy(AX), oAX)
    assert np.array_equal(npy(YtAn), oYtA)
