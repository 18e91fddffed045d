"""Section 5.1.1's perturbed cores and SGN with the SVD epsilon-pseudoinverse
(eq. 2.2) on the GPU (gn_factors_variant) against the oracle's
perturbed_core_factors / sgn_svd / pivoted_householder_qr on the same sketches.
Tolerances: the approximant F G within 1e-9 relative (FP64 throughout; the
floors are chosen inside a gap of the spectrum so that no singular value or
pivot sits near them), singular values within 1e-12 of the largest, the
pivot order exactly."""
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


def _gap_floor(vals):
    """A floor in the middle of the widest gap of the descending values (middle third)."""
    v = np.sort(np.abs(np.asarray(vals)))[::-1]
    n = len(v)
    lo, hi = n // 3, 2 * n // 3
    ratios = v[lo:hi] / np.maximum(v[lo + 1:hi + 1], 1e-300)
    i = lo + int(np.argmax(ratios))
    return float(np.sqrt(v[i] * v[i + 1])), v[i] / v[i + 1]


def _state(gn, H, m, n, r, l, seed, rank=None):
    rng = np.random.default_rng(seed)
    if rank is None:
        A = gn_synth.config2(m=m, n=n, r=r, l=l, seed=seed).a.numpy()
    else:
        A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    X, Y = rng.standard_normal((n, r)), rng.standard_normal((m, r + l))
    cu = lambda t: torch.from_numpy(np.ascontiguousarray(t)).cuda()
    AX, YtA = O.sketch(A, X, Y)
    return A, X, Y, AX, YtA, cu


def _run(gn, H, AX, YtA, X, eps, variant, cu):
    m, r = AX.shape
    n = YtA.shape[1]
    F = torch.zeros(m, r, dtype=torch.float64, device="cuda")
    G = torch.zeros(r, n, dtype=torch.float64, device="cuda")
    sv = torch.zeros(r, dtype=torch.float64, device="cuda")
    k = H.factors_variant(cu(AX), cu(YtA), cu(X), eps, variant, F, G, sv)
    assert H.sync_status() == 0
    return k, F[:, :k].cpu().numpy(), G[:k].cpu().numpy(), sv.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_svd_truncate_recovers_rank_deficient_and_matches_oracle(gn, H):
    """Exact rank 10 < r = 24: the SVD eps-pseudoinverse keeps k = 10 singular
    values and GN recovers A; the approximant equals the oracle's sgn_svd."""
    m, n, r, l = 500, 300, 24, 12
    A, X, Y, AX, YtA, cu = _state(gn, H, m, n, r, l, 1, rank=10)
    C = YtA @ X
    s = np.linalg.svd(C, compute_uv=False)
    eps = 1e-9 * s[0]
    k, F, G, sv = _run(gn, H, AX, YtA, X, eps, gn.SVD_TRUNCATE, cu)
    assert k == 10
    assert np.max(np.abs(sv - s)) <= 1e-12 * s[0]
    Ah = F @ G
    assert rel(Ah, A) <= 1e-10
    assert rel(Ah, O.sgn_svd(A, X, Y, eps)) <= 1e-10


@pytest.mark.parametrize("variant", ["svd", "rrqr", "diag"])
def test_raised_floor_variants_match_oracle(gn, H, variant):
    """Full-rank decaying spectrum with the floor inside a gap of the relevant
    values (singular values of C, or the pivoted / unpivoted diag(R)): the
    approximant of each Section 5.1.1 alternative against the oracle's."""
    m, n, r, l = 600, 400, 40, 20
    A, X, Y, AX, YtA, cu = _state(gn, H, m, n, r, l, 2)
    C = YtA @ X
    if variant == "svd":
        vals = np.linalg.svd(C, compute_uv=False)
    elif variant == "rrqr":
        vals = np.diag(O.pivoted_householder_qr(C)[1])
    else:
        vals = np.diag(O.householder_qr(C)[1])
    floor, gap = _gap_floor(vals)
    assert gap > 1.05
    code = {"svd": gn.SVD_RAISE, "rrqr": gn.RRQR_RAISE, "diag": gn.DIAG_RAISE}[variant]
    k, F, G, sv = _run(gn, H, AX, YtA, X, floor, code, cu)
    assert k == r
    Fo, Go = O.perturbed_core_factors(AX, YtA, X, floor, variant)
    assert rel(F @ G, Fo @ Go) <= 1e-9
    if variant == "svd":
        assert np.max(np.abs(sv - vals)) <= 1e-12 * vals[0]


def test_pivoted_qr_order_and_factors(gn, H):
    """The pivot order of the GPU's column-pivoted Householder QR equals the
    oracle's (largest remaining norm first), and diag(R) before raising is
    non-increasing and equal to the oracle's."""
    m, n, r, l = 300, 200, 32, 16
    A, X, Y, AX, YtA, cu = _state(gn, H, m, n, r, l, 3)
    C = YtA @ X
    Qo, Ro, perm = O.pivoted_householder_qr(C)
    floor = 1e-300   # nothing raised
    k, F, G, sv = _run(gn, H, AX, YtA, X, floor, gn.RRQR_RAISE, cu)
    d = np.diag(Ro)
    assert np.max(np.abs(sv - d)) <= 1e-12 * d[0]
    assert np.all(np.diff(sv) <= 1e-12 * d[0])
    Fo = O.right_solve_upper(AX[:, perm], Ro)
    assert rel(F, Fo) <= 1e-9
    assert rel(F @ G, O.gn(A, X, Y, 0.0, O.PLAIN)[0]) <= 1e-9


def test_fp32_sketches_and_bf16_x(gn, H):
    """FP32 sketch state (as the tensor-core sketch writes it) with a BF16 X:
    C and every product in FP64 on the FP32 values, against the oracle on the
    same values."""
    m, n, r, l = 700, 500, 48, 24
    rng = np.random.default_rng(4)
    A = gn_synth.config2(m=m, n=n, r=r, l=l, seed=4).a.numpy()
    Xq = O.quantize_bf16(rng.standard_normal((n, r)))
    Yq = O.quantize_bf16(rng.standard_normal((m, r + l)))
    AX, YtA = O.sketch(A, Xq, Yq)
    AX32, YtA32 = AX.astype(np.float32), YtA.astype(np.float32)
    C = YtA32.astype(np.float64) @ Xq
    floor, gap = _gap_floor(np.linalg.svd(C, compute_uv=False))
    Xb = H.quantize(torch.from_numpy(Xq).cuda())
    F = torch.zeros(m, r, dtype=torch.float64, device="cuda")
    G = torch.zeros(r, n, dtype=torch.float64, device="cuda")
    k = H.factors_variant(torch.from_numpy(AX32).cuda(), torch.from_numpy(YtA32).cuda(), Xb, floor, gn.SVD_RAISE, F, G)
    assert H.sync_status() == 0 and k == r
    Fo, Go = O.perturbed_core_factors(AX32.astype(np.float64), YtA32.astype(np.float64), Xq, floor, "svd")
    assert rel((F @ G).cpu().numpy(), Fo @ Go) <= 1e-9


def test_diag_raise_any_r(gn, H):
    """DIAG_RAISE uses the blocked Householder QR, so r beyond the shared-memory
    limit (r = 200) works; the SVD variants refuse it (GN_ERR_UNSUPPORTED)."""
    m, n, r, l = 1200, 800, 200, 100
    A, X, Y, AX, YtA, cu = _state(gn, H, m, n, r, l, 5)
    vals = np.diag(O.householder_qr(YtA @ X)[1])
    floor, gap = _gap_floor(vals)
    k, F, G, sv = _run(gn, H, AX, YtA, X, floor, gn.DIAG_RAISE, cu)
    Fo, Go = O.perturbed_core_factors(AX, YtA, X, floor, "diag")
    assert rel(F @ G, Fo @ Go) <= 1e-9
    with pytest.raises(gn.GNError) as ei:
        _run(gn, H, AX, YtA, X, floor, gn.SVD_RAISE, cu)
    assert ei.value.status == 8


@pytest.mark.parametrize("r,l", [(9, 5), (37, 19), (128, 64)])
def test_svd_variants_cluster_edges(gn, H, r, l):
    """The Jacobi sweeps run over an 8-CTA cluster, each CTA holding a slice of
    the columns: r = 9 leaves CTAs with no column, r = 37 is odd (a dummy player
    every round), r = 128 and r + l = 192 are the largest core.  Singular values
    against LAPACK's, and both SVD variants' approximants against the oracle's."""
    m, n = 700, 500
    A, X, Y, AX, YtA, cu = _state(gn, H, m, n, r, l, 9 + r)
    C = YtA @ X
    s = np.linalg.svd(C, compute_uv=False)
    floor, gap = _gap_floor(s)
    assert gap > 1.05
    k, F, G, sv = _run(gn, H, AX, YtA, X, floor, gn.SVD_RAISE, cu)
    assert k == r
    assert np.max(np.abs(sv - s)) <= 1e-12 * s[0]
    Fo, Go = O.perturbed_core_factors(AX, YtA, X, floor, "svd")
    assert rel(F @ G, Fo @ Go) <= 1e-9
    k, F, G, sv = _run(gn, H, AX, YtA, X, floor, gn.SVD_TRUNCATE, cu)
    assert k == int(np.sum(s > floor))
    assert rel(F @ G, O.sgn_svd(A, X, Y, floor)) <= 1e-9
