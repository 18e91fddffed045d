"""The bench's own shape, 32768 x 16384 with r = 1000, l = 500, in the launch
configuration bench.py times (256-row sketch tiles in CTA pairs with half-K
Y^T A items; the core's Q formed in 256-reflector blocks on the tensor cores;
the factors' solve with its updates on the tensor cores): sampled outputs
against the oracle's products, the core against the oracle's Householder QR of
the same C, and the factors against the same solve on the FP64 units."""
import numpy as np
import pytest
import torch

from oracle import gn_oracle as O

pytestmark = pytest.mark.gpu

M, N, R, L = 32768, 16384, 1000, 500
U32 = 2.0 ** -24


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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def run(gn, H):
    """Integer inputs in [-3, 3] (exact in BF16; every AX and Y^T A sum stays an
    integer below 2^24), drawn on the device; sketch, core (AUTO, relative eps)
    and factors through the C ABI."""
    g = torch.Generator(device="cuda").manual_seed(2009)

    def draw(rows, cols):
        return torch.randint(-3, 4, (rows, cols), generator=g, device="cuda", dtype=torch.int8)

    A8, X8, Y8 = draw(M, N), draw(N, R), draw(M, R + L)
    Ab, Xb, Yb = H.quantize(A8.double()), H.quantize(X8.double()), H.quantize(Y8.double())
    ws = H.workspace(M, N, R, L, gn.BF16)
    AX = torch.empty(M, R, dtype=torch.float32, device="cuda")
    YtA = torch.empty(R + L, N, dtype=torch.float32, device="cuda")
    core = gn.Core.empty(R, L, "cuda")
    F = torch.zeros(M, R, dtype=torch.float64, device="cuda")
    G = torch.zeros(R, N, dtype=torch.float64, device="cuda")
    eps = 10 * U32
    H.approx(Ab, Xb, Yb, eps, gn.AUTO | gn.EPS_RELATIVE, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    out = dict(A8=A8, X8=X8, Y8=Y8, AX=AX, YtA=YtA, core=core, F=F, G=G, eps=eps, ws=ws, Ab=Ab, Xb=Xb, Yb=Yb)
    yield out
    del out
    torch.cuda.empty_cache()


def test_full_size_sketch_sampled_bitwise(gn, H, run):
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(M, 64, replace=False))
    cols = np.sort(rng.choice(N, 64, replace=False))
    A8, X = run["A8"], run["X8"].double().cpu().numpy()
    Y = run["Y8"].double().cpu().numpy()
    oAX = A8[torch.from_numpy(rows).cuda()].double().cpu().numpy() @ X
    oYtA = Y.T @ A8[:, torch.from_numpy(cols).cuda()].double().cpu().numpy()
    assert np.array_equal(npy(run["AX"])[rows], oAX)
    assert np.array_equal(npy(run["YtA"])[:, cols], oYtA)


def test_full_size_core_against_oracle_qr(gn, H, run):
    """C from the split-BF16 core product within its FP32 accumulation bound of
    the exact (Y^T A) X; Q and R against the oracle's Householder QR of the
    GPU's C; the detector's estimates against the oracle's power iterations."""
    core = run["core"]
    YtA, X = npy(run["YtA"]), run["X8"].double().cpu().numpy()
    C = npy(core.C)
    bound = 6 * N * U32 * (np.abs(YtA) @ np.abs(X))
    assert np.all(np.abs(C - YtA @ X) <= bound)
    Qo, Ro = O.householder_qr(C)
    kappa = np.linalg.cond(Ro)
    tol = max(1e-11, 50 * kappa * 1.1e-16)
    assert rel(npy(core.R), Ro) <= tol
    assert rel(npy(core.Q), Qo) <= max(tol, 1e-11)
    Rg = npy(core.R)
    assert abs(core.rinv_est - O.rinv_norm_estimate(Rg, iters=6)) <= 1e-8 * core.rinv_est
    assert abs(core.c_norm_est - O.norm2_estimate(Rg, iters=6)) <= 1e-10 * core.c_norm_est
    assert core.k == R and core.sgn == 0


def test_full_size_factors_tensor_core_vs_fp64_units(gn, H, run):
    """F R = AX solved with its updates on the tensor cores (the bench's path)
    against the same solve on the FP64 units; G (three BF16 slices per operand,
    FP32 accumulation) against the FP64 product of Q_1^T and Y^T A within the
    FP32 accumulation bound (r + l) u32 (|Q_1|^T |Y^T A|) per element."""
    core, ws = run["core"], run["ws"]
    F1, G1 = run["F"], run["G"]
    F0 = torch.zeros_like(F1)
    G0 = torch.zeros_like(G1)
    H.set_fp64_tc(False)
    H.set_fp64_g(True)
    try:
        H.factors(run["AX"], run["YtA"], core, F0, G0, ws)
        assert H.sync_status() == 0
    finally:
        H.set_fp64_tc(True)
        H.set_fp64_g(False)
    d = torch.linalg.norm(F1 - F0).item()
    assert d <= 1e-11 * torch.linalg.norm(F0).item()
    bound = 4 * (R + L) * U32 * (core.Q.abs().T @ run["YtA"].double().abs())
    assert torch.all((G1 - G0).abs() <= bound)


def test_full_size_factors_sampled_rows_against_oracle(gn, H, run):
    """The tensor-core triangular solve F R = AX (the bench's path) against the
    oracle's column-oriented back substitution on 64 sampled rows of the same
    AX with the GPU's R (rows of F are independent solves), and G against
    Q_1^T (Y^T A) on 64 sampled columns within the FP32 accumulation bound."""
    core, F, G = run["core"], run["F"], run["G"]
    rng = np.random.default_rng(17)
    rows = np.sort(rng.choice(M, 64, replace=False))
    cols = np.sort(rng.choice(N, 64, replace=False))
    Rg = npy(core.R)
    AXs = npy(run["AX"])[rows]
    Fo = O.right_solve_upper(AXs, Rg)
    Fs = npy(F)[rows]
    assert rel(Fs, Fo) <= 1e-10
    Q1 = npy(core.Q)
    YtAs = npy(run["YtA"])[:, cols]
    Go = Q1.T @ YtAs
    bound = 4 * (R + L) * U32 * (np.abs(Q1).T @ np.abs(YtAs))
    assert np.all(np.abs(npy(G)[:, cols] - Go) <= bound)


@pytest.fixture(scope="module")
def run2000(gn, H, run):
    """r = 2000, l = 1000 on the bench's shape with integer inputs (every AX and
    Y^T A sum an integer below 2^24), through the C ABI: sketch, core (AUTO,
    relative eps), factors."""
    r, l = 2000, 1000
    g = torch.Generator(device="cuda").manual_seed(4001)

    def draw(rows, cols):
        return torch.randint(-3, 4, (rows, cols), generator=g, device="cuda", dtype=torch.int8)

    A8 = run["A8"]
    X8, Y8 = draw(N, r), draw(M, r + l)
    Xb, Yb = H.quantize(X8.double()), H.quantize(Y8.double())
    ws = H.workspace(M, N, r, l, gn.BF16)
    AX = torch.empty(M, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, N, dtype=torch.float32, device="cuda")
    core = gn.Core.empty(r, l, "cuda")
    F = torch.zeros(M, r, dtype=torch.float64, device="cuda")
    G = torch.zeros(r, N, dtype=torch.float64, device="cuda")
    H.sketch(run["Ab"], Xb, Yb, AX, YtA, ws)
    H.core(YtA, Xb, 10 * U32, gn.AUTO | gn.EPS_RELATIVE, core, ws)
    H.factors(AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    out = dict(X8=X8, Y8=Y8, AX=AX, YtA=YtA, core=core, F=F, G=G, ws=ws, r=r, l=l)
    yield out
    del out
    torch.cuda.empty_cache()


def test_r2000_sketch_factors_and_error(gn, H, run, run2000):
    """r = 2000: sampled sketch rows / columns bit for bit, sampled rows of F
    against the oracle's back substitution with the GPU's R, sampled columns of
    G within the FP32 bound, and the fused error kernel against numpy on a
    64-row block (the full n and k = r width)."""
    d = run2000
    r, l, core = d["r"], d["l"], d["core"]
    assert core.k == r and core.sgn == 0
    rng = np.random.default_rng(23)
    rows = np.sort(rng.choice(M, 64, replace=False))
    cols = np.sort(rng.choice(N, 64, replace=False))
    rows_t = torch.from_numpy(rows).cuda()
    A8 = run["A8"]
    Ar = A8[rows_t].double().cpu().numpy()
    X = d["X8"].double().cpu().numpy()
    assert np.array_equal(npy(d["AX"])[rows], Ar @ X)
    Ac = A8[:, torch.from_numpy(cols).cuda()].double()
    assert np.array_equal(npy(d["YtA"])[:, cols], (d["Y8"].double().T @ Ac).cpu().numpy())
    Rg = npy(core.R)
    assert np.all(np.diag(Rg) >= 0) and np.allclose(Rg, np.triu(Rg))
    Fo = O.right_solve_upper(npy(d["AX"])[rows], Rg)
    assert rel(npy(d["F"])[rows], Fo) <= 1e-10
    Q1 = npy(core.Q)
    YtAs = npy(d["YtA"])[:, cols]
    bound = 4 * (r + l) * U32 * (np.abs(Q1).T @ np.abs(YtAs))
    assert np.all(np.abs(npy(d["G"])[:, cols] - Q1.T @ YtAs) <= bound)
    # fused error on a 64-row block: ||A_s - F_s G||_F^2 against numpy
    As = A8[rows_t].double().contiguous()
    Fs = d["F"][rows_t].contiguous()
    e2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    H.error_fro2(As, Fs, d["G"], e2, d["ws"])
    assert H.sync_status() == 0
    ref = np.linalg.norm(As.cpu().numpy() - npy(Fs) @ npy(d["G"])) ** 2
    assert abs(e2.item() - ref) <= 1e-9 * ref
