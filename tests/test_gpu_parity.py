"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Inputs come from gn_synth (seeded); the same arrays go to both sides.  Sizes
span several tiles of every kernel and end in ragged tails.  Tolerances:
  * FP64 path: <= 1e-10 relative Frobenius for sketches, factors and A_hat;
  * tensor-core sketches on bf16 operands: exact when every product and
    partial sum is an integer below 2^24, otherwise within the FP32
    accumulation bound |err_ij| <= 2 K u32 (|A||X|)_ij;
  * quantisation: bit-exact against the oracle's rounding.
"""
import math

import numpy as np
import pytest
import torch

import gn_synth
from oracle import gn_oracle as O

pytestmark = pytest.mark.gpu

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


def cu(t):
    return torch.as_tensor(t).cuda()


def npy(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def bf16_operand(gn, t):
    """bf16 copy with an 8-aligned leading dimension (exact when t is bf16-representable)."""
    p = gn.padded(t.shape[0], t.shape[1], torch.bfloat16, "cuda")
    p.copy_(t.to(torch.bfloat16))
    return p


# ------------------------------------------------------------------ quantisation
@pytest.mark.parametrize("shape", [(257, 131), (64, 8)])
def test_quantize_matches_oracle_bitwise(gn, H, shape):
    x = gn_synth.gaussian(shape, 5, 0) * 3.0
    hi = H.quantize(cu(x))
    hi2, lo2 = H.quantize(cu(x), split=True)
    torch.cuda.synchronize()
    q = O.quantize_bf16(x.numpy())
    oh, ol = O.split_bf16(x.numpy())
    assert np.array_equal(npy(hi), q)
    assert np.array_equal(npy(hi2), oh)
    assert np.array_equal(npy(lo2), ol)


# ---------------------------------------------------------------- FP64 sketches
@pytest.mark.parametrize("m,n,r,l", [(1000, 500, 20, 10), (333, 200, 37, 19)])
def test_fp64_sketch_parity(gn, H, m, n, r, l):
    A = gn_synth.gaussian((m, n), 1, 0)
    X, Y = gn_synth.sketches(m, n, r, l, 2)
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    ws = H.workspace(m, n, r, l, gn.F64)
    H.sketch(cu(A), cu(X), cu(Y), AX, YtA, ws)
    oAX, oYtA = O.sketch(A.numpy(), X.numpy(), Y.numpy())
    assert rel(npy(AX), oAX) <= 1e-13
    assert rel(npy(YtA), oYtA) <= 1e-13
    assert H.sync_status() == 0


# --------------------------------------------------------- tensor-core sketches
@pytest.mark.parametrize("m,n,r,l", [(300, 200, 70, 35), (128, 64, 16, 8), (520, 390, 130, 65), (1100, 300, 70, 35)])
def test_tc_sketch_exact_on_integer_inputs(gn, H, m, n, r, l):
    """Small integers are exact in bf16, and every partial sum stays an
    integer below 2^24, so FP32 accumulation is exact: bitwise parity."""
    g = torch.Generator().manual_seed(m * 7 + n)
    A = torch.randint(-3, 4, (m, n), generator=g).double()
    X = torch.randint(-3, 4, (n, r), generator=g).double()
    Y = torch.randint(-3, 4, (m, r + l), generator=g).double()
    AX = torch.full((m, r), float("nan"), dtype=torch.float32, device="cuda")
    YtA = torch.full((r + l, n), float("nan"), dtype=torch.float32, device="cuda")
    ws = H.workspace(m, n, r, l, gn.BF16)
    H.sketch(bf16_operand(gn, A), bf16_operand(gn, X), bf16_operand(gn, Y), AX, YtA, ws)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(A.numpy(), X.numpy(), Y.numpy())
    assert np.array_equal(npy(AX), oAX)
    assert np.array_equal(npy(YtA), oYtA)


def test_tc_sketch_large_sampled(gn, H):
    """16384 x 8192, r = 1000, l = 500: enough tiles for the 256-row tile shape
    (two MMAs sharing each B stage).  Integer inputs drawn on the
    device; 64 sampled rows of AX and 64 sampled columns of Y^T A against the
    oracle's products, bitwise."""
    m, n, r, l = 16384, 8192, 1000, 500
    g = torch.Generator(device="cuda").manual_seed(78)
    def draw(rows, cols):
        return torch.randint(-3, 4, (rows, cols), generator=g, device="cuda", dtype=torch.int8).double()
    A, X, Y = draw(m, n), draw(n, r), draw(m, r + l)
    Ab, Xb, Yb = H.quantize(A), H.quantize(X), H.quantize(Y)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    ws = H.workspace(m, n, r, l, gn.BF16)
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    assert H.sync_status() == 0
    rng = np.random.default_rng(6)
    rows = np.sort(rng.choice(m, 64, replace=False))
    cols = np.sort(rng.choice(n, 64, replace=False))
    oAX = A[torch.from_numpy(rows).cuda()].cpu().numpy() @ X.cpu().numpy()
    oYtA = Y.cpu().numpy().T @ A[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    assert np.array_equal(npy(AX)[rows], oAX)
    assert np.array_equal(npy(YtA)[:, cols], oYtA)
    del A, X, Y, Ab, Xb, Yb, AX, YtA, ws
    torch.cuda.empty_cache()


@pytest.mark.parametrize("split", [False, True])
def test_tc_sketch_fp32_accumulation_bound(gn, H, split):
    m, n, r, l = 700, 450, 100, 50
    A = gn_synth.gaussian((m, n), 11, 0)
    X, Y = gn_synth.sketches(m, n, r, l, 12)
    Aq, Xq, Yq = (torch.from_numpy(O.quantize_bf16(t.numpy())) for t in (A, X, Y))
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    ws = H.workspace(m, n, r, l, gn.BF16X2 if split else gn.BF16)
    if split:
        hi, lo = O.split_bf16(A.numpy())
        Ah, Al = bf16_operand(gn, torch.from_numpy(hi)), bf16_operand(gn, torch.from_numpy(lo))
        H.sketch(Ah, bf16_operand(gn, Xq), bf16_operand(gn, Yq), AX, YtA, ws, A_lo=Al)
        Aref = hi + lo
    else:
        H.sketch(bf16_operand(gn, Aq), bf16_operand(gn, Xq), bf16_operand(gn, Yq), AX, YtA, ws)
        Aref = Aq.numpy()
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(Aref, Xq.numpy(), Yq.numpy())
    bAX = 2 * n * U32 * (np.abs(Aref) @ np.abs(Xq.numpy())) * (2 if split else 1)
    bYA = 2 * m * U32 * (np.abs(Yq.numpy()).T @ np.abs(Aref)) * (2 if split else 1)
    assert np.all(np.abs(npy(AX) - oAX) <= bAX)
    assert np.all(np.abs(npy(YtA) - oYtA) <= bYA)


# ------------------------------------------------------------------- core + factors
def _core_tensors(gn, r, l):
    return gn.Core.empty(r, l, "cuda")


def test_fp64_core_qr_parity(gn, H):
    m, n, r, l = 400, 300, 48, 24
    A = gn_synth.gaussian((m, n), 21, 0) * torch.pow(0.9, torch.arange(n, dtype=torch.float64))
    X, Y = gn_synth.sketches(m, n, r, l, 22)
    oAX, oYtA = O.sketch(A.numpy(), X.numpy(), Y.numpy())
    c = O.core(oYtA, X.numpy(), 0.0, O.PLAIN)
    ws = H.workspace(m, n, r, l, gn.F64)
    core = _core_tensors(gn, r, l)
    H.core(cu(oYtA), cu(X), 0.0, gn.PLAIN, core, ws)
    assert H.sync_status() == 0
    assert rel(npy(core.C), c["C"]) <= 1e-13
    kappa = np.linalg.cond(c["R"])
    tol = max(1e-11, 50 * kappa * 1.1e-16)
    assert rel(npy(core.R), c["R"]) <= tol
    assert rel(npy(core.Q), c["Q"]) <= tol
    assert core.k == r and core.sgn == 0


def test_fp64_core_full_size(gn, H):
    """The bench's core shape, (r+l) x r = 1500 x 1000 in FP64, mode AUTO with
    relative eps: Q, R against the oracle's Householder QR (31 panels with
    look-ahead, WY updates of every width); the detector's ||R^{-1}|| and ||C||
    estimates against the oracle's power iterations on the same R (two 32-row
    blocks per CTA in the clustered detector)."""
    r, l, n = 1000, 500, 1100
    rng = np.random.default_rng(11)
    YtA = rng.standard_normal((r + l, n))
    X = rng.standard_normal((n, r)) * (0.996 ** np.arange(r))[None, :]
    c = O.core(YtA, X, 10 * O.U64, O.AUTO, eps_relative=True, diag_iters=6)
    ws = H.workspace(r + l, n, r, l, gn.F64)
    core = _core_tensors(gn, r, l)
    H.core(cu(YtA), cu(X), 10 * O.U64, gn.AUTO | gn.EPS_RELATIVE, core, ws)
    assert H.sync_status() == 0
    assert rel(npy(core.C), c["C"]) <= 1e-13
    kappa = np.linalg.cond(c["R"])
    tol = max(1e-11, 50 * kappa * 1.1e-16)
    assert rel(npy(core.R), c["R"]) <= tol
    assert rel(npy(core.Q), c["Q"]) <= tol
    Rg = npy(core.R)
    assert abs(core.rinv_est - O.rinv_norm_estimate(Rg, iters=6)) <= 1e-8 * core.rinv_est
    assert abs(core.c_norm_est - O.norm2_estimate(Rg, iters=6)) <= 1e-10 * core.c_norm_est
    assert core.k == c["k"] == r and core.sgn == int(c["sgn"]) == 0


def test_fp64_core_r2000_properties(gn, H):
    """r = 2000, l = 1000 (the larger core of the bench shape, 3000 x 2000, 63
    panels): properties that hold at any size -- Householder backward error
    ||C - QR|| and orthogonality ||Q^T Q - I|| at the FP64 rounding level,
    R upper triangular with a non-negative diagonal -- and the detector's
    estimates against the oracle's power iterations on the same R."""
    r, l, n = 2000, 1000, 2200
    rng = np.random.default_rng(12)
    YtA = rng.standard_normal((r + l, n))
    X = rng.standard_normal((n, r)) * (0.998 ** np.arange(r))[None, :]
    ws = H.workspace(r + l, n, r, l, gn.F64)
    core = _core_tensors(gn, r, l)
    H.core(cu(YtA), cu(X), 10 * O.U64, gn.AUTO | gn.EPS_RELATIVE, core, ws)
    assert H.sync_status() == 0
    C, Q, R = npy(core.C), npy(core.Q), npy(core.R)
    assert rel(C, YtA @ X) <= 1e-13
    u = O.U64
    assert np.linalg.norm(C - Q @ R) <= 50 * r * u * np.linalg.norm(C)
    assert np.linalg.norm(Q.T @ Q - np.eye(r)) <= 50 * r * u
    assert np.array_equal(np.triu(R), R) and np.all(np.diag(R) >= 0)
    assert abs(core.rinv_est - O.rinv_norm_estimate(R, iters=6)) <= 1e-8 * core.rinv_est
    assert abs(core.c_norm_est - O.norm2_estimate(R, iters=6)) <= 1e-10 * core.c_norm_est
    assert core.k == r and core.sgn == 0


def test_factor_g_tensor_core_vs_fp64(gn, H):
    """For FP32 Y^T A the factor G = Q_1^T (Y^T A) is formed on the tensor cores
    from three BF16 slices of each operand; against the FP64 product (the
    gn_set_fp64_g path) it agrees to FP32 accumulation accuracy, and F (the
    FP64 triangular solve) is identical."""
    m, n, r, l = 900, 700, 60, 30
    A = gn_synth.gaussian((m, n), 41, 0) * torch.pow(0.97, torch.arange(n, dtype=torch.float64))
    X, Y = gn_synth.sketches(m, n, r, l, 42)
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    H.sketch(bf16_operand(gn, A), bf16_operand(gn, X), bf16_operand(gn, Y), AX, YtA, ws)
    core = _core_tensors(gn, r, l)
    H.core(YtA, bf16_operand(gn, X), 10 * O.U32, gn.PLAIN, core, ws)
    F1 = torch.empty(m, r, dtype=torch.float64, device="cuda")
    G1 = torch.empty(r, n, dtype=torch.float64, device="cuda")
    F2, G2 = torch.empty_like(F1), torch.empty_like(G1)
    H.factors(AX, YtA, core, F1, G1, ws)
    H.set_fp64_g(True)
    try:
        H.factors(AX, YtA, core, F2, G2, ws)
    finally:
        H.set_fp64_g(False)
    assert H.sync_status() == 0
    assert torch.equal(F1, F2)
    Q, S = npy(core.Q), npy(YtA)
    bound = 4 * (r + l) * O.U32 * (np.abs(Q).T @ np.abs(S))
    assert np.all(np.abs(npy(G1) - npy(G2)) <= bound)
    assert rel(npy(G2), Q.T @ S) <= 1e-12


@pytest.mark.parametrize("mode", ["plain", "auto"])
def test_fp64_gn_config1(gn, H, mode):
    """The 1000 x 500 geometric case: factors and A_hat at 1e-10."""
    p = gn_synth.config1()
    A, X, Y = p.a.numpy(), p.x.numpy(), p.y.numpy()
    md = O.PLAIN if mode == "plain" else O.AUTO
    Ahat, o = O.gn(A, X, Y, p.eps, md)
    m, n = A.shape
    r, l = p.r, p.l
    ws = H.workspace(m, n, r, l, gn.F64)
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    F = torch.empty(m, r, dtype=torch.float64, device="cuda")
    G = torch.empty(r, n, dtype=torch.float64, device="cuda")
    core = _core_tensors(gn, r, l)
    H.approx(cu(A), cu(X), cu(Y), p.eps, gn.PLAIN if mode == "plain" else gn.AUTO, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    assert core.k == o["k"] == r
    assert rel(npy(F), o["F"]) <= 1e-10
    assert rel(npy(G), o["G"]) <= 1e-10
    Ah = npy(F) @ npy(G)
    assert rel(Ah, Ahat) <= 1e-10
    # fused error kernel
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    H.error_fro2(cu(A), F, G, out, ws)
    torch.cuda.synchronize()
    assert abs(math.sqrt(out.item()) - np.linalg.norm(A - Ahat)) <= 1e-9 * np.linalg.norm(A)
    if mode == "auto":
        est = O.rinv_norm_estimate(o["R"], iters=6)
        assert abs(core.rinv_est - est) <= 1e-8 * est


def test_fp64_sgn_truncation_parity(gn, H):
    """Exactly rank-k0 input with k0 < r: the truncated branch (Section 5.1.1)."""
    m, n, k0, r, l = 300, 220, 9, 24, 12
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((m, k0)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k0)))
    A = (U * np.linspace(2.0, 1.0, k0)) @ V.T
    X, Y = gn_synth.sketches(m, n, r, l, 6)
    X, Y = X.numpy(), Y.numpy()
    eps = O.scale_eps(2.0, np.linalg.norm(X, 2), np.linalg.norm(Y, 2), O.U64)
    Ahat, o = O.gn(A, X, Y, eps, O.SGN)
    assert o["k"] == k0
    ws = H.workspace(m, n, r, l, gn.F64)
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    F = torch.zeros(m, r, dtype=torch.float64, device="cuda")
    G = torch.zeros(r, n, dtype=torch.float64, device="cuda")
    core = _core_tensors(gn, r, l)
    H.approx(cu(A), cu(X), cu(Y), eps, gn.SGN, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    assert core.k == k0 and core.sgn == 1
    Fk, Gk = npy(F)[:, :k0], npy(G)[:k0]
    assert rel(Fk @ Gk, Ahat) <= 1e-10
    assert rel(Fk @ Gk, A) <= 1e-11
    assert rel(Fk, o["F"]) <= 1e-9 and rel(Gk, o["G"]) <= 1e-9


def test_hmt_parity(gn, H):
    m, n, r = 900, 400, 40
    A = (gn_synth.gaussian((m, n), 31, 0) * torch.pow(0.95, torch.arange(n, dtype=torch.float64))).numpy()
    X = gn_synth.gaussian((n, r), 32, 0).numpy()
    Qo, Bo = O.hmt(A, X)
    ws = H.workspace(m, n, r, 1, gn.F64)
    Q = torch.empty(m, r, dtype=torch.float64, device="cuda")
    B = torch.empty(r, n, dtype=torch.float64, device="cuda")
    H.hmt(cu(A), cu(X), Q, B, ws)
    assert H.sync_status() == 0
    assert rel(npy(Q), Qo) <= 1e-10
    assert rel(npy(B), Bo) <= 1e-10


# -------------------------------------------------------------- mixed-precision path
def test_mixed_path_matches_oracle_on_quantized_inputs(gn, H):
    """bf16 sketches + split-bf16 core product: C within FP32 accuracy, and the
    approximation error within 1.05x of the oracle's on the same quantised A."""
    m, n, r, l = 1200, 640, 64, 32
    p = gn_synth.config2(m=m, n=n, r=r, l=l)
    A = p.a.numpy()
    Aq = O.quantize_bf16(A)
    Xq, Yq = O.quantize_bf16(p.x.numpy()), O.quantize_bf16(p.y.numpy())
    Ahat, o = O.gn(Aq, Xq, Yq, 0.0, O.PLAIN)
    err_o = np.linalg.norm(Aq - Ahat)
    ws = H.workspace(m, n, r, l, gn.BF16)
    Ab = bf16_operand(gn, torch.from_numpy(Aq))
    Xb = bf16_operand(gn, torch.from_numpy(Xq))
    Yb = bf16_operand(gn, torch.from_numpy(Yq))
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    F = torch.empty(m, r, dtype=torch.float64, device="cuda")
    G = torch.empty(r, n, dtype=torch.float64, device="cuda")
    core = _core_tensors(gn, r, l)
    H.approx(Ab, Xb, Yb, 0.0, gn.PLAIN, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    # C from the FP32 sketch, exact bf16 X: compare with the oracle's C of the GPU's Y^T A
    Cref = O.core_matrix(npy(YtA), Xq)
    bound = 4 * n * U32 * (np.abs(npy(YtA)) @ np.abs(Xq))
    assert np.all(np.abs(npy(core.C) - Cref) <= bound)
    Ah = npy(F) @ npy(G)
    err_g = np.linalg.norm(Aq - Ah)
    assert err_g <= 1.05 * err_o
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    H.error_fro2(Ab, F, G, out, ws)
    torch.cuda.synchronize()
    assert abs(math.sqrt(out.item()) - err_g) <= 1e-6 * err_g


def test_relative_eps_and_auto_switch(gn, H):
    """GN_EPS_RELATIVE: eps scales with the 6-iteration power estimate of
    ||C||_2, as in the oracle.  An exactly zero column of C (zero column of X)
    gives R_jj = 0, est = inf, and AUTO takes the truncated branch at k = j."""
    m, n, r, l = 260, 180, 20, 10
    A = gn_synth.gaussian((m, n), 41, 0).numpy()
    X, Y = gn_synth.sketches(m, n, r, l, 42)
    X, Y = X.numpy().copy(), Y.numpy()
    eps = 10 * O.U64
    mode = gn.AUTO | gn.EPS_RELATIVE
    ws = H.workspace(m, n, r, l, gn.F64)
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    F = torch.zeros(m, r, dtype=torch.float64, device="cuda")
    G = torch.zeros(r, n, dtype=torch.float64, device="cuda")
    core = _core_tensors(gn, r, l)
    H.approx(cu(A), cu(X), cu(Y), eps, mode, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    _, o = O.gn(A, X, Y, eps, O.AUTO, eps_relative=True, diag_iters=6)
    assert core.sgn == 0 and core.k == r and not o["sgn"]
    assert abs(core.eps_abs - o["eps_abs"]) <= 1e-10 * o["eps_abs"]
    assert abs(core.rinv_est - o["rinv_est"]) <= 1e-8 * o["rinv_est"]
    X[:, 7] = 0.0
    Ahat, o = O.gn(A, X, Y, eps, O.AUTO, eps_relative=True, diag_iters=6)
    assert o["sgn"] and o["k"] == 7
    core = _core_tensors(gn, r, l)
    H.approx(cu(A), cu(X), cu(Y), eps, mode, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    assert core.sgn == 1 and core.k == 7 and math.isinf(core.rinv_est)
    Ah = npy(F)[:, :7] @ npy(G)[:7]
    assert rel(Ah, Ahat) <= 1e-10


@pytest.mark.parametrize("kind", ["wellcond", "rankdef"])
def test_core_diagnostics_cluster_path(gn, H, kind):
    """r >= 64 takes the clustered diagnostics kernel: est ||R^{-1}||, est ||C||
    (relative eps) and the truncation rank against the oracle (6 iterations)."""
    m, n, r, l = 700, 420, 100, 50
    rng = np.random.default_rng(77)
    if kind == "wellcond":
        A = rng.standard_normal((m, n)) * (0.97 ** np.arange(n))[None, :]
    else:
        k0 = 70
        U, _ = np.linalg.qr(rng.standard_normal((m, k0)))
        V, _ = np.linalg.qr(rng.standard_normal((n, k0)))
        A = (U * np.linspace(3.0, 1.0, k0)) @ V.T
    X, Y = gn_synth.sketches(m, n, r, l, 78)
    X, Y = X.numpy(), Y.numpy()
    eps = 10 * O.U64 if kind == "wellcond" else 1e-9
    md = gn.AUTO if kind == "wellcond" else gn.SGN
    omd = O.AUTO if kind == "wellcond" else O.SGN
    Ahat, o = O.gn(A, X, Y, eps, omd, eps_relative=True, diag_iters=6)
    ws = H.workspace(m, n, r, l, gn.F64)
    AX = torch.empty(m, r, dtype=torch.float64, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float64, device="cuda")
    F = torch.zeros(m, r, dtype=torch.float64, device="cuda")
    G = torch.zeros(r, n, dtype=torch.float64, device="cuda")
    core = _core_tensors(gn, r, l)
    H.approx(cu(A), cu(X), cu(Y), eps, md | gn.EPS_RELATIVE, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    assert abs(core.eps_abs - o["eps_abs"]) <= 1e-10 * o["eps_abs"]
    assert core.k == o["k"] and core.sgn == int(o["sgn"])
    if kind == "wellcond":
        assert abs(core.rinv_est - o["rinv_est"]) <= 1e-8 * o["rinv_est"]
    else:
        assert core.k == 70
    k = core.k
    assert rel(npy(F)[:, :k] @ npy(G)[:k], Ahat) <= 1e-9


@pytest.mark.parametrize("part_k", [4096, 8192])
def test_split_sketch_fp64_accumulation_parts(gn, H, part_k):
    """Split-BF16 sketches with FP64-level accumulation (gn_set_fp64_accum): the K
    range runs as stored parts summed in FP64.  Integer inputs (every part sum
    exact): AX and Y^T A equal the oracle's products bit for bit with several
    parts on both products and ragged tails; the core's C then equals the exact
    (Y^T A) X (digit-sliced product, FP64-accurate)."""
    m, n, r, l = 2500, 9000, 100, 50
    g = torch.Generator().manual_seed(91)
    draw = lambda a, b: torch.randint(-3, 4, (a, b), generator=g).double()
    A, X, Y = draw(m, n), draw(n, r), draw(m, r + l)
    Ahi, Alo = H.quantize(A.cuda(), split=True)
    Xb, Yb = H.quantize(X.cuda()), H.quantize(Y.cuda())
    ws = H.workspace(m, n, r, l, gn.BF16X2)
    AX = torch.full((m, r), float("nan"), dtype=torch.float32, device="cuda")
    YtA = torch.full((r + l, n), float("nan"), dtype=torch.float32, device="cuda")
    H.set_fp64_accum(part_k)
    try:
        H.sketch(Ahi, Xb, Yb, AX, YtA, ws, A_lo=Alo)
        core = gn.Core.empty(r, l, "cuda")
        H.core(YtA, Xb, 0.0, gn.PLAIN, core, ws)
        assert H.sync_status() == 0
    finally:
        H.set_fp64_accum(0)
    oAX, oYtA = O.sketch(A.numpy(), X.numpy(), Y.numpy())
    assert np.array_equal(npy(AX), oAX)
    assert np.array_equal(npy(YtA), oYtA)
    C = npy(core.C)
    oC = oYtA @ X.numpy()
    assert np.max(np.abs(C - oC)) <= 1e-13 * np.max(np.abs(oC))
