"""FP64 products on the tensor cores by exact digit slicing (gn_dgemm_tc) and
their use in the factors' triangular solve, against exact integer products,
an extended-precision reference and the FP64-unit path."""
import numpy as np
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


@pytest.fixture(scope="module")
def H(gn):
    return gn.Handle()


def npy(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("M,N,K,ta,tb", [(300, 130, 270, False, False), (257, 300, 333, True, False),
                                         (129, 77, 200, False, True), (1000, 260, 1500, False, False)])
def test_dgemm_tc_exact_on_scaled_integers(gn, H, M, N, K, ta, tb):
    """Integers below 2^20 times per-row / per-column powers of two: every digit
    product and partial sum is exact (K <= 1500 keeps the FP32 sums below 2^24
    units in each pass, the FP64 combination below 2^53), so the result equals
    the exact product bit for bit."""
    rng = np.random.default_rng(M + N + K)
    Ai = rng.integers(-(1 << 20), 1 << 20, (M, K), dtype=np.int64)
    Bi = rng.integers(-(1 << 20), 1 << 20, (K, N), dtype=np.int64)
    Ai[3] = 0                                                    # an all-zero row
    ps = rng.integers(-30, 31, M)
    qs = rng.integers(-30, 31, N)
    # exact reference: integer products per pass of at most 1024 of K, scaled
    exact = np.zeros((M, N))
    for k0 in range(0, K, 1024):
        exact += (Ai[:, k0:k0 + 1024] @ Bi[k0:k0 + 1024]).astype(np.float64)
    exact = np.ldexp(exact, ps[:, None] + qs[None, :])
    A = np.ldexp(Ai.astype(np.float64), ps[:, None])
    B = np.ldexp(Bi.astype(np.float64), qs[None, :])
    At = torch.from_numpy(np.ascontiguousarray(A.T if ta else A)).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(B.T if tb else B)).cuda()
    C = H.dgemm_tc(At, Bt, ta=ta, tb=tb)
    assert H.sync_status() == 0
    if K <= 1024:
        assert np.array_equal(npy(C), exact)
    else:   # two passes: the FP64 sum of two exact partial products rounds once
        assert np.all(np.abs(npy(C) - exact) <= 2.0 ** -52 * np.abs(exact))


@pytest.mark.parametrize("M,N,K,ta,tb,a32", [(1, 1, 1, False, False, False), (33, 31, 1025, True, True, False),
                                             (65, 40, 7, True, False, True), (40, 65, 2049, False, True, True),
                                             (31, 97, 9, True, True, True)])
def test_dgemm_tc_exact_slicing_edges(gn, H, M, N, K, ta, tb, a32):
    """The slicing's edge cases on exact integer products: operands strided or
    contiguous along K, FP32 or FP64 A, K = 1, odd K, a last pass of one
    element, three passes, and row counts off the 32-row grain of the slicing
    launch.  Each pass of at most 1024 of K is exact; the FP64 sum of the
    passes rounds once per pass."""
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    Ai = rng.integers(-(1 << 20), 1 << 20, (M, K), dtype=np.int64)
    Bi = rng.integers(-(1 << 20), 1 << 20, (K, N), dtype=np.int64)
    ps = rng.integers(-20, 21, M)
    qs = rng.integers(-20, 21, N)
    parts = [(Ai[:, k0:k0 + 1024] @ Bi[k0:k0 + 1024]).astype(np.float64) for k0 in range(0, K, 1024)]
    exact = np.ldexp(sum(parts), ps[:, None] + qs[None, :])
    A = np.ldexp(Ai.astype(np.float64), ps[:, None])
    B = np.ldexp(Bi.astype(np.float64), qs[None, :])
    An = np.ascontiguousarray(A.T if ta else A)
    At = torch.from_numpy(An.astype(np.float32) if a32 else An).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(B.T if tb else B)).cuda()
    C = npy(H.dgemm_tc(At, Bt, ta=ta, tb=tb))
    assert H.sync_status() == 0
    if len(parts) == 1:
        assert np.array_equal(C, exact)
    else:
        assert np.all(np.abs(C - exact) <= (len(parts) - 1) * 2.0 ** -52 * np.abs(exact))


def test_dgemm_tc_alpha_beta_and_fp32_operand(gn, H):
    M, N, K = 200, 90, 150
    rng = np.random.default_rng(7)
    A32 = rng.integers(-1000, 1000, (M, K)).astype(np.float32) / 8
    B = rng.integers(-1000, 1000, (K, N)).astype(np.float64) / 4
    C0 = rng.integers(-1000, 1000, (M, N)).astype(np.float64)
    exact = -2.0 * (A32.astype(np.float64) @ B) + 0.5 * C0
    C = torch.from_numpy(C0.copy()).cuda()
    H.dgemm_tc(torch.from_numpy(A32).cuda(), torch.from_numpy(B).cuda(), C, alpha=-2.0, beta=0.5)
    assert H.sync_status() == 0
    assert np.array_equal(npy(C), exact)


def test_dgemm_tc_accuracy_general(gn, H):
    """Gaussian entries with row and column magnitudes over 2^+-15: error per
    element within 2^-44 K max|a_i.| max|b_.j| of an extended-precision
    reference, and relative Frobenius error <= 1e-13."""
    M, N, K = 160, 96, 1100
    rng = np.random.default_rng(11)
    A = rng.standard_normal((M, K)) * np.exp2(rng.uniform(-15, 15, M))[:, None]
    B = rng.standard_normal((K, N)) * np.exp2(rng.uniform(-15, 15, N))[None, :]
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble))
    C = npy(H.dgemm_tc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()))
    assert H.sync_status() == 0
    bound = 2.0 ** -44 * K * np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :]
    err = np.abs(C - ref).astype(np.float64)
    assert np.all(err <= bound)
    # relative to the size of each row-column product, not dominated by the largest rows
    scale = np.abs(A) @ np.abs(B)
    assert np.max(err / scale) <= 1e-13


@pytest.mark.parametrize("K,ta,a32", [(9000, False, False), (5000, True, True)])
def test_dgemm_tc_groups_of_passes(gn, H, K, ta, a32):
    """K beyond one group of four 1024-element passes: the groups run one after
    another, beta applies to the first only and alpha to every pass.  Against an
    extended-precision reference of alpha op(A) B + beta C0, within 2^-44 K
    max|a_i.| max|b_.j| |alpha| plus one rounding per pass of the partial sums."""
    M, N = 96, 70
    alpha, beta = -1.5, 0.75
    rng = np.random.default_rng(K)
    A = rng.standard_normal((M, K)) * np.exp2(rng.uniform(-8, 8, M))[:, None]
    if a32:
        A = A.astype(np.float32).astype(np.float64)
    B = rng.standard_normal((K, N)) * np.exp2(rng.uniform(-8, 8, N))[None, :]
    C0 = rng.standard_normal((M, N))
    ref = alpha * (A.astype(np.longdouble) @ B.astype(np.longdouble)) + beta * C0.astype(np.longdouble)
    An = np.ascontiguousarray(A.T if ta else A)
    At = torch.from_numpy(An.astype(np.float32) if a32 else An).cuda()
    C = torch.from_numpy(C0.copy()).cuda()
    H.dgemm_tc(At, torch.from_numpy(B).cuda(), C, alpha=alpha, beta=beta, ta=ta)
    assert H.sync_status() == 0
    err = np.abs(npy(C) - ref).astype(np.float64)
    # the passes' FP64 additions round against their partial sums (at most one per pass)
    passes = -(-K // 1024)
    scale = np.abs(beta * C0) + abs(alpha) * (np.abs(A) @ np.abs(B))
    bound = (2.0 ** -44 * K * abs(alpha) * np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :]
             + (passes + 1) * 2.0 ** -53 * scale)
    assert np.all(err <= bound)


def _mixed_factors(gn, H, A, X, Y, eps, mode, tc):
    m, n = A.shape
    r, l = X.shape[1], Y.shape[1] - X.shape[1]
    Ab, Xb, Yb = H.quantize(A.cuda()), H.quantize(X.cuda()), H.quantize(Y.cuda())
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    F = torch.zeros(m, r, dtype=torch.float64, device="cuda")
    G = torch.zeros(r, n, dtype=torch.float64, device="cuda")
    core = gn.Core.empty(r, l, "cuda")
    H.set_fp64_tc(tc)
    try:
        H.approx(Ab, Xb, Yb, eps, mode, AX, YtA, core, F, G, ws)
        assert H.sync_status() == 0
    finally:
        H.set_fp64_tc(True)
    return npy(F)[:, :core.k], core


def test_factors_tensor_core_solve_matches_fp64_units(gn, H):
    """m = 4096, r = 300: the solve F R = AX with its outer-block updates on the
    tensor cores against the same solve on the FP64 units (cond(R) ~ 10^2 on a
    flat-spectrum A)."""
    m, n, r, l = 4096, 1500, 300, 150
    A = gn_synth.gaussian((m, n), 61, 0)
    X, Y = gn_synth.sketches(m, n, r, l, 62)
    F1, c1 = _mixed_factors(gn, H, A, X, Y, 0.0, gn.PLAIN, True)
    F0, c0 = _mixed_factors(gn, H, A, X, Y, 0.0, gn.PLAIN, False)
    assert c1.k == c0.k == r
    assert np.linalg.norm(F1 - F0) <= 1e-11 * np.linalg.norm(F0)


def test_factors_tensor_core_truncated_branch(gn, H):
    """A truncation (zero columns of X give R_jj = 0): F = (AX Q_2) R_2^{-T} with
    AX Q_2 and the transposed solve's updates on the tensor cores."""
    m, n, r, l = 3000, 1200, 260, 130
    A = gn_synth.gaussian((m, n), 71, 0)
    X, Y = gn_synth.sketches(m, n, r, l, 72)
    X = X.clone()
    X[:, 200:] = 0.0
    mode = gn.AUTO | gn.EPS_RELATIVE
    eps = 10 * 2.0 ** -24
    F1, c1 = _mixed_factors(gn, H, A, X, Y, eps, mode, True)
    F0, c0 = _mixed_factors(gn, H, A, X, Y, eps, mode, False)
    assert c1.sgn == c0.sgn == 1 and c1.k == c0.k == 200
    assert np.linalg.norm(F1 - F0) <= 1e-11 * np.linalg.norm(F0)


@pytest.mark.parametrize("n,r,l", [(2048, 600, 300), (700, 96, 48)])
def test_core_q_tensor_core_vs_fp64_units(gn, H, n, r, l):
    """The core's Householder QR with its block updates (256-column blocks,
    r = 600) and the formation of Q as digit-sliced products on the tensor
    cores, against the same QR on the FP64 units: R and Q equal to a
    few 1e-11 (each digit-sliced product errs by ~1e-13 of |A||B| per
    element), Q orthonormal to 1e-12 r and C = QR to 1e-11 relative (the
    trailing products' error, far below the 2^-24 of the FP32 sketches that
    such a core comes from)."""
    g = torch.Generator(device="cuda").manual_seed(n + r)
    YtA = torch.randn(r + l, n, generator=g, device="cuda", dtype=torch.float32)
    X = H.quantize(torch.randn(n, r, generator=g, device="cuda", dtype=torch.float64))
    ws = H.workspace(4096, n, r, l, gn.BF16)
    out = []
    for tc in (True, False):
        core = gn.Core.empty(r, l, "cuda")
        H.set_fp64_tc(tc)
        try:
            H.core(YtA, X, 0.0, gn.PLAIN, core, ws)
            assert H.sync_status() == 0
        finally:
            H.set_fp64_tc(True)
        out.append((npy(core.Q), npy(core.R), npy(core.C)))
    (Q1, R1, C1), (Q0, R0, C0) = out
    assert np.array_equal(C1, C0)   # the same core matrix
    assert np.linalg.norm(R1 - R0) <= 3e-11 * np.linalg.norm(R0)
    assert np.linalg.norm(Q1 - Q0) <= 3e-11 * np.linalg.norm(Q0)
    assert np.linalg.norm(C1 - Q1 @ R1) <= 1e-11 * np.linalg.norm(C1)
    assert np.linalg.norm(C0 - Q0 @ R0) <= 1e-13 * np.linalg.norm(C0)
    assert np.linalg.norm(Q1.T @ Q1 - np.eye(r)) <= 1e-12 * r
