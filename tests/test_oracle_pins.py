"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each test names the passage it follows.  None of them re-types an oracle
formula: they check closed forms, invariants, library routines (LAPACK QR /
SVD), hand-derived worked examples and finite differences, chosen so that a
dropped term, a wrong sign, a wrong index or a transposed operand in the oracle
fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

from oracle import gn_oracle as O
import gn_synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


def _np(t):
    return t.numpy() if hasattr(t, "numpy") else np.asarray(t)


def _lowrank(m, n, k, seed, decay=None):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)))
    s = np.ones(k) if decay is None else decay
    return (U * s) @ V.T, s


def _sk(m, n, r, l, seed):
    rng = np.random.default_rng(seed + 1)
    return rng.standard_normal((n, r)), rng.standard_normal((m, r + l))


# --------------------------------------------------------------------------- QR
@pytest.mark.parametrize("shape", [(7, 5), (30, 20), (120, 80), (64, 64)])
def test_householder_qr_backward_stable_and_orthonormal(shape):
    """Textbook Householder: ||C - QR|| <= c u ||C||, ||Q^T Q - I|| <= c u."""
    C = RNG.standard_normal(shape)
    Q, R = O.householder_qr(C)
    u = O.U64
    assert np.allclose(R, np.triu(R))
    assert np.all(np.diag(R) >= 0)
    assert np.linalg.norm(C - Q @ R) <= 50 * u * np.linalg.norm(C) * shape[1]
    assert np.linalg.norm(Q.T @ Q - np.eye(shape[1])) <= 50 * u * shape[1]


def test_householder_qr_matches_lapack_up_to_signs():
    """LAPACK's R equals ours after making its diagonal non-negative."""
    C = RNG.standard_normal((50, 30))
    Ql, Rl = np.linalg.qr(C)
    s = np.sign(np.diag(Rl))
    Q, R = O.householder_qr(C)
    assert np.allclose(R, s[:, None] * Rl, atol=1e-12)
    assert np.allclose(Q, Ql * s[None, :], atol=1e-12)


def test_householder_qr_zero_and_dependent_columns():
    """A zero column gives R_jj = 0 with no reflection; Q stays orthonormal."""
    C = RNG.standard_normal((10, 4))
    C[:, 2] = 0.0
    Q, R = O.householder_qr(C)
    assert abs(R[2, 2]) < 1e-15
    assert np.linalg.norm(C - Q @ R) < 1e-13
    assert np.linalg.norm(Q.T @ Q - np.eye(4)) < 1e-13


def test_householder_reflector_sign_avoids_cancellation():
    """beta = -sign(alpha)||x|| keeps alpha - beta free of cancellation: on
    columns that are already almost e_j the computed Q stays orthonormal to
    roundoff (the other sign choice loses orthogonality here)."""
    C = np.eye(12, 8) + 1e-9 * RNG.standard_normal((12, 8))
    Q, R = O.householder_qr(C)
    assert np.linalg.norm(Q.T @ Q - np.eye(8)) <= 100 * O.U64
    assert np.linalg.norm(C - Q @ R) <= 100 * O.U64


def test_truncation_rank_rule():
    """Section 5.1.1: k is the first index whose |R_ii| <= eps (ties dropped)."""
    R = np.diag([3.0, 2.0, 1e-9, 5e-10]) + np.triu(np.ones((4, 4)), 1)
    assert O.truncation_rank(R, 1e-9) == 2
    assert O.truncation_rank(R, 0.9e-9) == 3
    assert O.truncation_rank(R, 1e-12) == 4
    R2 = np.diag([3.0, -1e-12, 2.0])
    assert O.truncation_rank(R2, 1e-10) == 1


# ----------------------------------------------------- hand-derived worked examples
@pytest.mark.parametrize("name", ["worked_rank1_r1.json", "worked_rank1_r2_sgn.json"])
def test_golden_worked_examples(name):
    g = json.load(open(os.path.join(GOLDEN, name)))
    A, X, Y = (np.array(g[k], float) for k in ("A", "X", "Y"))
    mode = {"plain": O.PLAIN, "sgn": O.SGN}[g["mode"]]
    Ahat, p = O.gn(A, X, Y, g["eps"], mode)
    e = g["expect"]
    assert p["k"] == e["k"]
    for key in ("AX", "YtA", "C", "R", "Q", "F", "G"):
        if key in e:
            assert np.allclose(p[key], np.array(e[key]), atol=1e-14), key
    if "R_row0" in e:
        assert np.allclose(p["R"][0], e["R_row0"], atol=1e-14)
        assert np.allclose(p["Q"][:, 0], e["Q_col0"], atol=1e-14)
        assert np.allclose(p["R2"], e["R2"], atol=1e-14)
        assert np.allclose(p["Q2"], e["Q2"], atol=1e-14)
    assert np.allclose(Ahat, np.array(e["Ahat"]), atol=1e-13)


# ------------------------------------------------------------ GN: what it must do
@pytest.mark.parametrize("k0,r,l", [(5, 5, 3), (8, 12, 6), (20, 20, 10)])
def test_exact_recovery_of_low_rank_inputs(k0, r, l):
    """rank(A) <= r => range(AX) = range(A) and GN returns A (Section 3.1).

    For k0 < r the core is rank deficient, so SGN (eq. 2.2) is used."""
    m, n = 80, 60
    A, _ = _lowrank(m, n, k0, 7)
    X, Y = _sk(m, n, r, l, 7)
    mode = O.PLAIN if k0 == r else O.SGN
    eps = O.scale_eps(1.0, np.linalg.norm(X, 2), np.linalg.norm(Y, 2), O.U64)
    Ahat, p = O.gn(A, X, Y, eps, mode)
    assert np.linalg.norm(A - Ahat) / np.linalg.norm(A) < 1e-12
    if k0 < r:
        assert p["k"] == k0


def test_eckart_young_lower_bound_and_rank():
    """||A - Ahat||_F >= (sum_{i>r} sigma_i^2)^(1/2) and rank(Ahat) <= r."""
    m, n, r, l = 60, 40, 8, 4
    A = RNG.standard_normal((m, n)) * (0.7 ** np.arange(n))[None, :]
    X, Y = _sk(m, n, r, l, 3)
    Ahat, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.linalg.norm(A - Ahat) >= np.sqrt(np.sum(s[r:] ** 2)) * (1 - 1e-12)
    assert np.linalg.norm(A - Ahat, 2) >= s[r] * (1 - 1e-12)
    sh = np.linalg.svd(Ahat, compute_uv=False)
    assert sh[r] <= 1e-12 * sh[0]


def test_interpolation_AhatX_equals_AX():
    """eq. (anni): (I - P_{AX,Y}) AX = 0, so Ahat X = AX (Section 3.1)."""
    m, n, r, l = 50, 40, 6, 3
    A = RNG.standard_normal((m, n))
    X, Y = _sk(m, n, r, l, 4)
    Ahat, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
    assert np.linalg.norm(Ahat @ X - A @ X) <= 1e-11 * np.linalg.norm(A @ X)


def test_invariance_under_sketch_mixing():
    """P_{XM,YN} = P_{X,Y} (Notation, Section 1).  With a tall core (l > 0) the
    identity holds for X -> XM; the Y -> YN part needs Y^T A X square (l = 0),
    because (N^T C)^+ N^T differs from C^+ for a tall C."""
    m, n, r, l = 45, 35, 5, 3
    A = RNG.standard_normal((m, n))
    X, Y = _sk(m, n, r, l, 5)
    M = np.eye(r) + 0.3 * RNG.standard_normal((r, r))
    A1, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
    A2, _ = O.gn(A, X @ M, Y, 0.0, O.PLAIN)
    assert np.linalg.norm(A1 - A2) <= 1e-10 * np.linalg.norm(A1)
    Ys = Y[:, :r]
    N = np.eye(r) + 0.3 * RNG.standard_normal((r, r))
    B1, _ = O.gn(A, X, Ys, 0.0, O.PLAIN)
    B2, _ = O.gn(A, X @ M, Ys @ N, 0.0, O.PLAIN)
    assert np.linalg.norm(B1 - B2) <= 1e-9 * np.linalg.norm(B1)


def test_matches_pinv_definition_when_well_conditioned():
    """The QR route of eq. 5.1 equals the definition of eq. 2.1 (LAPACK pinv)."""
    m, n, r, l = 40, 30, 6, 3
    A = RNG.standard_normal((m, n))
    X, Y = _sk(m, n, r, l, 6)
    Ahat, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
    assert np.linalg.norm(Ahat - O.gn_definition(A, X, Y)) <= 1e-11 * np.linalg.norm(Ahat)


def test_equals_tropp17():
    """GN and Q(Y^T Q)^+ Y^T A with Q = orth(AX) agree (Section 7.1)."""
    m, n, r, l = 70, 50, 10, 5
    A = RNG.standard_normal((m, n)) * (0.8 ** np.arange(n))[None, :]
    X, Y = _sk(m, n, r, l, 8)
    Ahat, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
    assert np.linalg.norm(Ahat - O.tropp17(A, X, Y)) <= 1e-9 * np.linalg.norm(Ahat)


def test_gn_with_Y_equal_AX_is_hmt():
    """With Y = AX (l = 0), GN = Q Q^T A = HMT (Section 2.4.1)."""
    m, n, r = 60, 45, 7
    A = RNG.standard_normal((m, n))
    X = RNG.standard_normal((n, r))
    Ahat, _ = O.gn(A, X, A @ X, 0.0, O.PLAIN)
    Q, B = O.hmt(A, X)
    assert np.linalg.norm(Ahat - Q @ B) <= 1e-10 * np.linalg.norm(A)


def test_sgn_qr_truncation_equals_svd_eps_pinv():
    """Section 5.1.1: the QR truncation + second QR gives the SVD eps-pinv when
    there is a gap around eps.  Also fixes the transpose on R_2: the printed
    R_2^{-1} form disagrees with the SVD by O(1)."""
    m, n, k0, r, l = 60, 50, 6, 10, 5
    A, _ = _lowrank(m, n, k0, 9, decay=np.linspace(1.0, 0.1, k0))
    X, Y = _sk(m, n, r, l, 9)
    eps = 1e-8 * np.linalg.norm(Y.T @ A @ X, 2)
    Ahat, p = O.gn(A, X, Y, eps, O.SGN)
    assert p["k"] == k0
    ref = O.sgn_svd(A, X, Y, eps)
    assert np.linalg.norm(Ahat - ref) <= 1e-10 * np.linalg.norm(ref)
    # the untransposed reading
    bad = (A @ X) @ (p["Q2"] @ np.linalg.inv(p["R2"]) @ p["Q"][:, :p["k"]].T) @ (Y.T @ A)
    assert np.linalg.norm(bad - ref) > 1e-3 * np.linalg.norm(ref)


def test_sgn_without_truncation_equals_plain():
    m, n, r, l = 40, 30, 6, 3
    A = RNG.standard_normal((m, n))
    X, Y = _sk(m, n, r, l, 10)
    A1, p1 = O.gn(A, X, Y, 1e-14, O.SGN)
    A2, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
    assert p1["k"] == r
    assert np.linalg.norm(A1 - A2) <= 1e-12 * np.linalg.norm(A1)


def test_detector_and_stress_input():
    """Section 4.2 / 5.1.1 / 5.1.2.  An exactly low-rank A makes R's trailing
    diagonal fall to roundoff: SGN then truncates to the true rank and the error
    stays at roundoff level, and plain GN is also accurate there (its
    instability needs ||R^{-1}|| >> 1/u).  An exactly zero column of C (a zero
    column of X) gives R_jj = 0, an infinite estimate, and AUTO switches."""
    m, n, k0, r, l = 100, 80, 7, 12, 6
    A, _ = _lowrank(m, n, k0, 11)
    X, Y = _sk(m, n, r, l, 11)
    eps = O.scale_eps(1.0, np.linalg.norm(X, 2), np.linalg.norm(Y, 2), O.U64)
    Ahat, p = O.gn(A, X, Y, eps, O.SGN)
    assert p["sgn"] and p["k"] == k0
    assert np.linalg.norm(A - Ahat) / np.linalg.norm(A) < 1e-12
    Arel, p2 = O.gn(A, X, Y, 10 * O.U64, O.SGN, eps_relative=True)
    assert k0 <= p2["k"] <= r and np.linalg.norm(A - Arel) / np.linalg.norm(A) < 1e-12
    Aplain, q = O.gn(A, X, Y, 10 * O.U64, O.AUTO, eps_relative=True)
    assert np.linalg.norm(A - Aplain) / np.linalg.norm(A) < 1e-12
    est = q["rinv_est"]
    assert est * np.linalg.norm(q["C"], 2) * O.U64 > 0.5     # kappa(R) ~ 1/u, not >> 1/u
    # exactly singular core: AUTO takes the SGN branch
    B = RNG.standard_normal((m, n))
    Xz = X.copy()
    Xz[:, 5] = 0.0
    Bhat, z = O.gn(B, Xz, Y, 10 * O.U64, O.AUTO, eps_relative=True)
    assert z["rinv_est"] == np.inf and z["sgn"] and z["k"] == 5
    # well-conditioned: AUTO stays plain
    _, w = O.gn(B, X, Y, 10 * O.U64, O.AUTO, eps_relative=True)
    assert not w["sgn"] and w["k"] == r
    # the relative threshold is eps * ||C||_2
    assert abs(w["eps_abs"] - 10 * O.U64 * np.linalg.norm(w["C"], 2)) <= 1e-3 * w["eps_abs"]


def test_rinv_norm_estimate_matches_svd():
    """Power method on R^{-1} R^{-T} converges to 1/sigma_min(R)."""
    C = RNG.standard_normal((40, 25)) @ np.diag(np.logspace(0, -6, 25))
    _, R = O.householder_qr(C)
    est = O.rinv_norm_estimate(R, iters=200)
    true = 1.0 / np.linalg.svd(R, compute_uv=False)[-1]
    assert abs(est - true) <= 1e-6 * true
    Z = R.copy()
    Z[3, 3] = 0.0
    assert O.rinv_norm_estimate(Z) == np.inf


def test_triangular_solves_against_library():
    """F R = B and F R^T = B, checked against LAPACK's triangular solver via
    numpy.linalg.solve on the dense triangle."""
    R = np.triu(RNG.standard_normal((9, 9))) + 4 * np.eye(9)
    B = RNG.standard_normal((13, 9))
    F1 = O.right_solve_upper(B, R)
    F2 = O.right_solve_upper_transpose(B, R)
    assert np.allclose(F1, np.linalg.solve(R.T, B.T).T, atol=1e-12)
    assert np.allclose(F2, np.linalg.solve(R, B.T).T, atol=1e-12)


def test_hmt_orthonormal_and_projection():
    """Algorithm 1: Q^T Q = I, Q B = Q Q^T A, and ||A - QB|| >= sigma_{r+1}."""
    m, n, r = 70, 40, 9
    A = RNG.standard_normal((m, n)) * (0.75 ** np.arange(n))[None, :]
    X = RNG.standard_normal((n, r))
    Q, B = O.hmt(A, X)
    assert np.linalg.norm(Q.T @ Q - np.eye(r)) < 1e-13
    Qa, _ = np.linalg.qr(A @ X)
    assert np.linalg.norm(Q @ B - Qa @ (Qa.T @ A)) < 1e-12 * np.linalg.norm(A)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.linalg.norm(A - Q @ B, 2) >= s[r] * (1 - 1e-12)


def test_expected_error_bounds_over_seeds():
    """Theorems 3.1 and 3.2 in expectation (20 seeds): the HMT error is within
    sqrt(1 + r/(r - rhat - 1)) of the best rank-rhat error, and GN's is within
    sqrt(1 + (r+l)/(l-1)) of HMT's root-mean-square error."""
    m, n, r, l, rhat = 120, 90, 16, 8, 8
    rng = np.random.default_rng(21)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = 0.8 ** np.arange(n)
    A = (U * s) @ V.T
    e_gn, e_hmt2 = [], []
    for t in range(20):
        X, Y = _sk(m, n, r, l, 100 + t)
        Ahat, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
        Q, B = O.hmt(A, X)
        e_gn.append(np.linalg.norm(A - Ahat))
        e_hmt2.append(np.linalg.norm(A - Q @ B) ** 2)
    tail = np.sqrt(np.sum(s[rhat:] ** 2))
    hmt_rms = np.sqrt(np.mean(e_hmt2))
    assert hmt_rms <= np.sqrt(1 + r / (r - rhat - 1)) * tail * 1.05
    assert np.mean(e_gn) <= np.sqrt(1 + (r + l) / (l - 1)) * hmt_rms * 1.05


def test_config1_error_above_truncated_svd_tail():
    """The 1000 x 500 geometric case: sigma is known by construction, so the
    GN error is at least the tail (sum_{i>20} sigma_i^2)^(1/2) and, by
    Theorem 3.2, not far above it."""
    p = gn_synth.config1()
    A, X, Y = _np(p.a), _np(p.x), _np(p.y)
    Ahat, q = O.gn(A, X, Y, p.eps, O.AUTO)
    s = 2.0 ** (-np.arange(1, 501) / 10.0)
    tail = np.sqrt(np.sum(s[p.r:] ** 2))
    err = np.linalg.norm(A - Ahat)
    assert tail * (1 - 1e-9) <= err <= 6 * tail
    assert q["k"] == p.r and not q["sgn"]


def test_adjoint_matches_central_differences():
    """Gradient of <G, Ahat> (plain GN, X and Y fixed) against central
    differences in FP64 on 64 x 48, r = 8, l = 4: 16 random directions and 200
    single entries."""
    m, n, r, l = 64, 48, 8, 4
    rng = np.random.default_rng(31)
    A = rng.standard_normal((m, n)) * (0.9 ** np.arange(n))[None, :]
    X, Y = rng.standard_normal((n, r)), rng.standard_normal((m, r + l))
    G = rng.standard_normal((m, n))
    grad = O.gn_backward(A, X, Y, G)
    h = 1e-6 * np.linalg.norm(A)
    for _ in range(16):
        D = rng.standard_normal((m, n))
        D /= np.linalg.norm(D)
        fd = (O.gn_loss(A + h * D, X, Y, G) - O.gn_loss(A - h * D, X, Y, G)) / (2 * h)
        an = np.sum(grad * D)
        assert abs(fd - an) <= 1e-6 * max(1.0, np.linalg.norm(grad))
    idx = rng.choice(m * n, size=200, replace=False)
    for f in idx:
        i, j = divmod(int(f), n)
        E = np.zeros((m, n))
        E[i, j] = 1.0
        fd = (O.gn_loss(A + h * E, X, Y, G) - O.gn_loss(A - h * E, X, Y, G)) / (2 * h)
        assert abs(fd - grad[i, j]) <= 1e-6 * max(1.0, np.linalg.norm(grad))


def test_adjoint_linear_in_G_and_zero_for_zero_G():
    m, n, r, l = 20, 15, 4, 2
    rng = np.random.default_rng(32)
    A = rng.standard_normal((m, n))
    X, Y = rng.standard_normal((n, r)), rng.standard_normal((m, r + l))
    G1, G2 = rng.standard_normal((m, n)), rng.standard_normal((m, n))
    g1, g2 = O.gn_backward(A, X, Y, G1), O.gn_backward(A, X, Y, G2)
    g12 = O.gn_backward(A, X, Y, 2 * G1 - G2)
    assert np.allclose(g12, 2 * g1 - g2, atol=1e-9)
    assert np.allclose(O.gn_backward(A, X, Y, 0 * G1), 0.0)


# -------------------------------------------------------------- quantisation
def test_quantize_bf16_against_torch():
    """Round to nearest even on the FP32 pattern equals torch's bfloat16 cast
    of the FP32 value, and integers below 256 are exact."""
    import torch
    x = RNG.standard_normal(10000) * 10.0 ** RNG.integers(-6, 6, 10000)
    f32 = torch.tensor(x).to(torch.float32)
    ref = f32.to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.quantize_bf16(x), ref)
    ints = np.arange(-255, 256, dtype=float)
    assert np.array_equal(O.quantize_bf16(ints), ints)
    # exact halfway cases round to the even neighbour (7 fraction bits)
    ties = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 2 + 2.0 ** -7])
    assert np.array_equal(O.quantize_bf16(ties), [1.0, 1 + 2.0 ** -6, -1.0, 2.0])


def test_split_bf16_is_accurate_to_16_bits():
    x = RNG.standard_normal(5000)
    hi, lo = O.split_bf16(x)
    f = x.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(hi + lo - f) <= 2.0 ** -16 * np.abs(f) + 1e-300)
    assert np.array_equal(O.quantize_bf16(hi), hi)
    assert np.array_equal(O.quantize_bf16(lo), lo)


def _e4m3_values():
    """Every non-negative finite e4m3 value, built from the format's fields:
    exponent field f (bias 7), mantissa field t; f = 0 is subnormal (t/8 2^-6);
    f = 15, t = 7 is NaN."""
    vals = []
    for f in range(16):
        for t in range(8):
            if f == 15 and t == 7:
                continue
            vals.append((t / 8.0) * 2.0 ** -6 if f == 0 else (1 + t / 8.0) * 2.0 ** (f - 7))
    return np.array(vals)


def test_e4m3_round_fixed_points_and_ties():
    """Representable values round to themselves; midpoints go to the neighbour
    with the even mantissa field; anything off the midpoint goes to the nearer."""
    v = _e4m3_values()
    assert v.max() == O.E4M3_MAX and len(v) == 127
    assert np.array_equal(O.e4m3_round(v), v)
    assert np.array_equal(O.e4m3_round(-v), -v)
    lo, hi = v[:-1], v[1:]
    mid = (lo + hi) / 2
    even_is_lo = (np.arange(len(lo)) % 2) == 0      # codes 0, 1, 2 ...: mantissa parity follows the index
    assert np.array_equal(O.e4m3_round(mid), np.where(even_is_lo, lo, hi))
    gap = hi - lo
    assert np.array_equal(O.e4m3_round(mid - gap / 64), lo)
    assert np.array_equal(O.e4m3_round(mid + gap / 64), hi)
    assert O.e4m3_round(np.float32(460.0)) == 448.0       # below the 464 midpoint
    assert O.e4m3_round(np.float32(470.0)) == 448.0       # would round to 480: saturates
    assert O.e4m3_round(np.float32(-1e6)) == -448.0
    assert O.e4m3_round(np.float32(2.0 ** -11)) == 0.0    # below half the smallest subnormal


def test_e4m3_round_against_torch():
    """An independent implementation: torch's float8_e4m3fn cast (round to
    nearest even) on in-range FP32 values."""
    import torch
    rng = np.random.default_rng(8)
    y = np.concatenate([rng.uniform(-448, 448, 20000), rng.standard_normal(20000) * 0.01]).astype(np.float32)
    ref = torch.tensor(y).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(O.e4m3_round(y), ref)


def test_e4m3_tile_scale_rule():
    """The scale is the smallest power of two that brings the tile maximum to at
    most 448; every stored value is then an e4m3 value times 2^e."""
    assert int(O.e4m3_tile_exponent(448.0)) == 0
    assert int(O.e4m3_tile_exponent(448.0 * (1 + 2.0 ** -20))) == 1
    assert int(O.e4m3_tile_exponent(449.0)) == 1
    assert int(O.e4m3_tile_exponent(224.0)) == -1
    assert int(O.e4m3_tile_exponent(448.0 * 2.0 ** -30)) == -30
    assert int(O.e4m3_tile_exponent(0.0)) == 0
    rng = np.random.default_rng(9)
    x = rng.standard_normal((300, 260)) * np.exp(rng.uniform(-8, 8, (300, 1)))
    q, e = O.quantize_e4m3_tiles(x)
    assert e.shape == (3, 3)
    vals = set(_e4m3_values().tolist())
    x32 = x.astype(np.float32).astype(np.float64)
    for i in range(3):
        for j in range(3):
            blk = q[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128] / 2.0 ** e[i, j]
            assert set(np.abs(blk).ravel().tolist()) <= vals
            amax = np.abs(x32[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128]).max()
            assert amax <= 448.0 * 2.0 ** e[i, j] and amax > 448.0 * 2.0 ** (e[i, j] - 1)
            # half a quantum: 2^-4 relative in the normal range, 2^-10 2^e below it
            err = np.abs(q[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128] - x32[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128])
            bound = np.maximum(2.0 ** -4 * np.abs(x32[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128]),
                               2.0 ** (e[i, j] - 10))
            assert np.all(err <= bound)


# ------------------------------------------------ sketch-state operations (Section 6)
def _decaying(m, n, seed, p=1.0):
    """A with singular values i^-p over min(m, n) modes (a full-rank test matrix)."""
    k = min(m, n)
    A, _ = _lowrank(m, n, k, seed, decay=np.arange(1, k + 1, dtype=float) ** -p)
    return A


@pytest.mark.parametrize("truncate", [False, True])
def test_apply_without_forming_matches_formed_product(truncate):
    """Ahat W and W Ahat in the orders the text after Algorithm 2 gives equal the
    formed F G times W (the pinned factors) and, after a truncation, the SVD
    epsilon-pseudoinverse form; W Ahat W' is consistent both ways."""
    m, n, r, l = 70, 50, 12, 6
    A = _decaying(m, n, 21, p=2.0)
    X, Y = _sk(m, n, r, l, 21)
    if truncate:
        X[:, 9:] = X[:, :3] @ np.random.default_rng(3).standard_normal((3, 3))   # rank-deficient core
    eps = O.scale_eps(1.0, np.linalg.norm(X, 2), np.linalg.norm(Y, 2), O.U64) * 1e3
    mode = O.SGN if truncate else O.PLAIN
    Ahat, p = O.gn(A, X, Y, eps, mode)
    c = {k: p[k] for k in ("Q", "R", "k", "Q2", "R2")}
    if truncate:
        assert p["k"] < r
    rng = np.random.default_rng(4)
    W = rng.standard_normal((n, 5))
    Wl = rng.standard_normal((4, m))
    AW = O.apply_right(p["AX"], p["YtA"], c, W)
    WA = O.apply_left(Wl, p["AX"], p["YtA"], c)
    assert np.linalg.norm(AW - Ahat @ W) <= 1e-11 * np.linalg.norm(Ahat @ W)
    assert np.linalg.norm(WA - Wl @ Ahat) <= 1e-11 * np.linalg.norm(Wl @ Ahat)
    assert np.allclose(Wl @ AW, WA @ W, rtol=1e-11, atol=1e-11 * np.linalg.norm(Wl @ AW))
    if truncate:
        As = O.sgn_svd(A, X, Y, eps)
        assert np.linalg.norm(AW - As @ W) <= 1e-8 * np.linalg.norm(As @ W)


def test_apply_without_forming_recovers_low_rank():
    """rank(A) <= r: Ahat = A (Section 3.1), so Ahat W = A W and W Ahat = W A."""
    m, n, r, l = 60, 45, 8, 4
    A, _ = _lowrank(m, n, 6, 31)
    X, Y = _sk(m, n, r, l, 31)
    eps = O.scale_eps(1.0, np.linalg.norm(X, 2), np.linalg.norm(Y, 2), O.U64)
    _, p = O.gn(A, X, Y, eps, O.SGN)
    c = {k: p[k] for k in ("Q", "R", "k", "Q2", "R2")}
    W = np.random.default_rng(5).standard_normal((n, 3))
    assert np.linalg.norm(O.apply_right(p["AX"], p["YtA"], c, W) - A @ W) <= 1e-11 * np.linalg.norm(A @ W)
    Wl = np.random.default_rng(6).standard_normal((2, m))
    assert np.linalg.norm(O.apply_left(Wl, p["AX"], p["YtA"], c) - Wl @ A) <= 1e-11 * np.linalg.norm(Wl @ A)


def test_resample_matches_fresh_sketch_and_recovers_added_rank():
    """r -> r + dr (Section 6): the resampled state equals the sketch taken with
    [X, Xd], [Y, Yd] from scratch, and a rank-(r + dr) matrix that r could not
    capture is recovered exactly after resampling."""
    m, n, r, l, dr, dl = 64, 48, 6, 3, 4, 2
    A, _ = _lowrank(m, n, r + dr, 41)
    X, Y = _sk(m, n, r, l, 41)
    rng = np.random.default_rng(42)
    Xd, Yd = rng.standard_normal((n, dr)), rng.standard_normal((m, dr + dl))
    AX, YtA = O.sketch(A, X, Y)
    before, _ = O.gn_from_sketches(AX, YtA, X, 0.0, O.PLAIN)
    assert np.linalg.norm(A - before) > 1e-3 * np.linalg.norm(A)
    AXn, YtAn, Xn, Yn = O.resample(A, AX, YtA, X, Y, Xd, Yd)
    AXs, YtAs = O.sketch(A, Xn, Yn)
    assert np.linalg.norm(AXn - AXs) <= 1e-14 * np.linalg.norm(AXs)
    assert np.linalg.norm(YtAn - YtAs) <= 1e-14 * np.linalg.norm(YtAs)
    after, c = O.gn_from_sketches(AXn, YtAn, Xn, 0.0, O.PLAIN)
    assert c["R"].shape == (r + dr, r + dr)
    assert np.linalg.norm(A - after) <= 1e-11 * np.linalg.norm(A)


@pytest.mark.parametrize("where", ["rows", "cols"])
def test_append_matches_gn_of_the_enlarged_matrix(where):
    """Appended rows [A; B] (the display in Section 6) or columns [A, B] (its
    analogue): the updated state gives the same approximant as GN run from
    scratch on the enlarged matrix with the enlarged sketch, and recovers an
    enlarged matrix of rank <= r exactly."""
    m, n, r, l = 50, 40, 10, 5
    rng = np.random.default_rng(51)
    for lowrank in (False, True):
        if lowrank:
            U, V = rng.standard_normal((m + 12, 7)), rng.standard_normal((n + 9, 7))
            big = U @ V.T
        else:
            big = _decaying(m + 12, n + 9, 52, p=1.5)
        if where == "rows":
            A, B = big[:m, :n], big[m:, :n]
            X, Y = rng.standard_normal((n, r)), rng.standard_normal((m, r + l))
            Yb = rng.standard_normal((B.shape[0], r + l))
            AX, YtA = O.sketch(A, X, Y)
            AXn, YtAn, Xn, Yn = O.append_rows(AX, YtA, X, Y, B, Yb)
            whole = np.vstack([A, B])
        else:
            A, B = big[:m, :n], big[:m, n:]
            X, Y = rng.standard_normal((n, r)), rng.standard_normal((m, r + l))
            Xb = rng.standard_normal((B.shape[1], r))
            AX, YtA = O.sketch(A, X, Y)
            AXn, YtAn, Xn, Yn = O.append_cols(AX, YtA, X, Y, B, Xb)
            whole = np.hstack([A, B])
        upd, _ = O.gn_from_sketches(AXn, YtAn, Xn, 0.0, O.PLAIN)
        fresh, _ = O.gn(whole, Xn, Yn, 0.0, O.PLAIN)
        assert np.linalg.norm(upd - fresh) <= 1e-10 * np.linalg.norm(fresh)
        if lowrank:
            assert np.linalg.norm(upd - whole) <= 1e-10 * np.linalg.norm(whole)


def test_streaming_update_matches_gn_of_the_updated_matrix():
    """A <- A + E (Section 6): the updated sketches equal the sketches of A + E,
    the approximant equals GN of A + E from scratch, and it interpolates:
    Ahat X = (A + E) X (Section 3's annihilation property)."""
    m, n, r, l = 60, 44, 9, 5
    A = _decaying(m, n, 61, p=1.0)
    E = 1e-2 * _decaying(m, n, 62, p=0.5)
    X, Y = _sk(m, n, r, l, 61)
    AX, YtA = O.sketch(A, X, Y)
    AXn, YtAn, _, _ = O.update(AX, YtA, X, Y, E)
    AXs, YtAs = O.sketch(A + E, X, Y)
    assert np.linalg.norm(AXn - AXs) <= 1e-13 * np.linalg.norm(AXs)
    assert np.linalg.norm(YtAn - YtAs) <= 1e-13 * np.linalg.norm(YtAs)
    upd, _ = O.gn_from_sketches(AXn, YtAn, X, 0.0, O.PLAIN)
    fresh, _ = O.gn(A + E, X, Y, 0.0, O.PLAIN)
    assert np.linalg.norm(upd - fresh) <= 1e-10 * np.linalg.norm(fresh)
    assert np.linalg.norm(upd @ X - (A + E) @ X) <= 1e-10 * np.linalg.norm((A + E) @ X)


# ------------------------------------------------ structured sketches (Section 7)
@pytest.mark.parametrize("n,r", [(64, 10), (97, 33), (128, 128)])
def test_dct_sketch_orthonormal_and_matches_fast_transform(n, r):
    """The subsampled DCT sketch has orthonormal columns, and A X equals the
    fast route (flip the signs of A's columns, orthonormal DCT-II along rows by
    SciPy's FFT-based transform, keep the sampled frequencies)."""
    scipy_fft = pytest.importorskip("scipy.fft")
    signs, cols = gn_synth.dct_sketch_draws(n, r, seed=n + r)
    signs, cols = _np(signs), _np(cols)
    X = O.dct_sketch(n, signs, cols)
    assert np.linalg.norm(X.T @ X - np.eye(r)) <= 1e-13 * r
    A = np.random.default_rng(n).standard_normal((23, n))
    fast = scipy_fft.dct(A * signs[None, :], type=2, norm="ortho", axis=1)[:, cols]
    assert np.linalg.norm(A @ X - fast) <= 1e-13 * np.linalg.norm(fast)


def test_gn_with_dct_sketches_recovers_low_rank_and_tracks_gaussian():
    """GN with subsampled DCT X and Y (Section 7's choice): exact recovery of a
    rank-r matrix, and on a decaying spectrum an error within a small factor of
    GN with Gaussian sketches of the same sizes (any O(1), well-conditioned
    sketch works, Section 3)."""
    m, n, r, l = 96, 80, 12, 6
    sx, cx = (_np(t) for t in gn_synth.dct_sketch_draws(n, r, seed=71))
    sy, cy = (_np(t) for t in gn_synth.dct_sketch_draws(m, r + l, seed=72))
    X, Y = O.dct_sketch(n, sx, cx), O.dct_sketch(m, sy, cy)
    A, _ = _lowrank(m, n, r, 73)
    Ahat, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
    assert np.linalg.norm(A - Ahat) <= 1e-11 * np.linalg.norm(A)
    A = _decaying(m, n, 74, p=2.0)
    e_dct = np.linalg.norm(A - O.gn(A, X, Y, 0.0, O.PLAIN)[0])
    Xg, Yg = _sk(m, n, r, l, 74)
    e_g = np.linalg.norm(A - O.gn(A, Xg, Yg, 0.0, O.PLAIN)[0])
    s = np.linalg.svd(A, compute_uv=False)
    assert e_dct >= np.sqrt(np.sum(s[r:] ** 2)) * (1 - 1e-12)
    assert e_dct <= 10 * e_g


# ------------------------------------------- core stabilised by perturbation (Section 5.1.1)
@pytest.mark.parametrize("shape", [(30, 20), (45, 45), (60, 12)])
def test_pivoted_qr_is_rank_revealing_and_backward_stable(shape):
    """C P = Q R with orthonormal Q, non-increasing |R_ii| (the pivoting rule),
    backward error at the rounding level, and on an exactly rank-k matrix the
    trailing diagonal at the rounding level."""
    rng = np.random.default_rng(shape[0])
    C = rng.standard_normal(shape) * np.exp2(rng.uniform(-6, 6, shape[1]))[None, :]
    Q, R, perm = O.pivoted_householder_qr(C)
    n = shape[1]
    assert sorted(perm.tolist()) == list(range(n))
    assert np.linalg.norm(C[:, perm] - Q @ R) <= 50 * n * O.U64 * np.linalg.norm(C)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 50 * n * O.U64
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-12)) and np.all(np.diag(R) >= 0)
    k = 7
    Ck = rng.standard_normal((shape[0], k)) @ rng.standard_normal((k, n))
    _, Rk, _ = O.pivoted_householder_qr(Ck)
    dk = np.abs(np.diag(Rk))
    assert dk[k - 1] > 1e-6 * dk[0] and np.all(dk[k:] <= 1e-12 * dk[0])


@pytest.mark.parametrize("variant", ["svd", "rrqr", "diag"])
def test_perturbed_core_equals_plain_gn_when_nothing_is_below_the_floor(variant):
    m, n, r, l = 70, 55, 10, 5
    A = _decaying(m, n, 91, p=1.0)
    X, Y = _sk(m, n, r, l, 91)
    AX, YtA = O.sketch(A, X, Y)
    plain, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
    F, G = O.perturbed_core_factors(AX, YtA, X, 1e-300, variant)
    assert np.linalg.norm(F @ G - plain) <= 1e-11 * np.linalg.norm(plain)


@pytest.mark.parametrize("variant", ["svd", "rrqr", "diag"])
def test_perturbed_core_recovers_rank_deficient_inputs(variant):
    """rank(A) = k0 < r makes Y^T A X exactly singular: the unperturbed core has
    no inverse, the perturbed one (floor at the rounding level of C) keeps
    ||R^{-1}|| bounded by 1 / floor and still returns A (Section 5.1.1: the
    perturbation replaces the truncation)."""
    m, n, r, l, k0 = 70, 55, 12, 6, 5
    A, _ = _lowrank(m, n, k0, 92)
    X, Y = _sk(m, n, r, l, 92)
    AX, YtA = O.sketch(A, X, Y)
    C = O.core_matrix(YtA, X)
    floor = 10 * O.U64 * np.linalg.norm(C, 2)
    F, G = O.perturbed_core_factors(AX, YtA, X, floor, variant)
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(G))
    assert np.linalg.norm(F @ G - A) <= 1e-12 * np.linalg.norm(A)
    sv = np.linalg.svd(C, compute_uv=False)
    assert sv[k0] <= 1e-12 * sv[0]                  # the core really is singular


@pytest.mark.parametrize("variant", ["svd", "rrqr", "diag"])
def test_perturbed_core_handles_an_exactly_zero_pivot(variant):
    """A zero column of X gives R_jj = 0 exactly: without the perturbation the
    solve divides by zero; with it the factors stay finite and the error is
    SGN's to within 2 % (each variant is a valid approximant of the same
    quality); the pivoted QR moves the zero column last, where the raised
    diagonal multiplies nothing, so it returns SGN's approximant itself."""
    m, n, r, l = 60, 45, 10, 5
    A = _decaying(m, n, 93, p=1.5)
    X, Y = _sk(m, n, r, l, 93)
    X[:, 4] = 0.0
    AX, YtA = O.sketch(A, X, Y)
    C = O.core_matrix(YtA, X)
    floor = 10 * O.U64 * np.linalg.norm(C, 2)
    F, G = O.perturbed_core_factors(AX, YtA, X, floor, variant)
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(G))
    sgn = O.sgn_svd(A, X, Y, floor)
    e_sgn = np.linalg.norm(A - sgn)
    assert np.linalg.norm(A - F @ G) <= 1.02 * e_sgn
    if variant == "rrqr":
        assert np.linalg.norm(F @ G - sgn) <= 1e-10 * np.linalg.norm(sgn)


# ------------------------------------------------ sparse A and CountSketch (Section 2.5, Section 7)
def test_countsketch_structure_and_input_sparsity_product():
    """One +-1 per row, X^T X = diag(bucket counts), and the bucket-sum product
    on a sparse A equals the dense product."""
    m, n, r = 120, 90, 16
    b, s = (_np(t) for t in gn_synth.countsketch_draws(n, r, seed=101))
    X = O.countsketch(n, r, b, s)
    assert np.all(np.count_nonzero(X, axis=1) == 1) and set(np.unique(np.abs(X[X != 0]))) == {1.0}
    counts = np.bincount(b, minlength=r).astype(float)
    assert np.array_equal(X.T @ X, np.diag(counts))
    rr, cc, vv = (_np(t) for t in gn_synth.sparse_lowrank_plus_noise(m, n, 4, 10, seed=102))
    As = O.sparse_from_coo(m, n, rr, cc, vv)
    Ad = As.toarray()
    fast = O.countsketch_apply_right(As, b, s, r)
    assert np.linalg.norm(fast - Ad @ X) <= 1e-14 * max(np.linalg.norm(Ad @ X), 1e-300)


def test_gn_with_countsketch_on_sparse_input():
    """GN with CountSketch X, Y on a sparse matrix of rank k <= r (no noise):
    the sketches by the input-sparsity route give the approximant of the dense
    route, and it recovers A (the Clarkson-Woodruff special case of GN the
    paper notes in Section 7)."""
    m, n, k, r, l = 200, 150, 5, 12, 6
    rr, cc, vv = (_np(t) for t in gn_synth.sparse_lowrank_plus_noise(m, n, k, 12, seed=103))
    keep = np.abs(vv) > 1e-6                                   # drop the noise: exactly rank <= k
    As = O.sparse_from_coo(m, n, rr[keep], cc[keep], vv[keep])
    Ad = As.toarray()
    bx, sx = (_np(t) for t in gn_synth.countsketch_draws(n, r, seed=104))
    by, sy = (_np(t) for t in gn_synth.countsketch_draws(m, r + l, seed=105))
    X, Y = O.countsketch(n, r, bx, sx), O.countsketch(m, r + l, by, sy)
    AX = O.countsketch_apply_right(As, bx, sx, r)
    YtA = O.countsketch_apply_right(As.T.tocsr(), by, sy, r + l).T
    eps = O.scale_eps(np.linalg.norm(Ad, 2), np.linalg.norm(X, 2), np.linalg.norm(Y, 2), O.U64)
    Ahat, c = O.gn_from_sketches(AX, YtA, X, eps, O.SGN)       # rank k < r: SGN truncates
    ref, p = O.gn(Ad, X, Y, eps, O.SGN)
    assert c["k"] == p["k"] <= k
    assert np.linalg.norm(Ahat - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.linalg.norm(Ahat - Ad) <= 1e-9 * np.linalg.norm(Ad)
