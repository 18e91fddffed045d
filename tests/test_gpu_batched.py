"""Batched path (one grouped sketch launch, one grouped core-product launch and
one CTA per core) against the unbatched C-ABI calls and the oracle, on
problems of uneven m, n, r."""
import numpy as np
import pytest
import torch

import gn_synth
from oracle import gn_oracle as O

pytestmark = pytest.mark.gpu

SHAPES = [(300, 200, 16), (520, 390, 40), (257, 129, 24), (700, 640, 64), (1024, 512, 100), (333, 333, 128)]


@pytest.fixture(scope="module")
def gn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_11392_gb300 as g
    return g


@pytest.fixture(scope="module")
def H(gn):
    return gn.Handle()


def _problem(gn, i, m, n, r, rankdef=False):
    l = r // 2
    rng = np.random.default_rng(100 + i)
    if rankdef:   # exactly rank r/2 and exactly representable in bf16 (small integers)
        k0 = r // 2
        U = rng.integers(-2, 3, (m, k0)).astype(float)
        V = rng.integers(-1, 2, (n, k0)).astype(float)
        A = U @ V.T
    else:
        A = rng.standard_normal((m, n)) * (0.97 ** np.arange(n))[None, :]
    X, Y = rng.standard_normal((n, r)), rng.standard_normal((m, r + l))
    q = lambda a: torch.from_numpy(O.quantize_bf16(a))
    dev = {}
    for name, a in (("A", A), ("X", X), ("Y", Y)):
        t = gn.padded(a.shape[0], a.shape[1], torch.bfloat16, "cuda")
        t.copy_(q(a).to(torch.bfloat16))
        dev[name] = t
    f32 = lambda a, b: torch.full((a, b), float("nan"), dtype=torch.float32, device="cuda")
    f64 = lambda a, b: torch.full((a, b), float("nan"), dtype=torch.float64, device="cuda")
    dev.update(AX=f32(m, r), YtA=f32(r + l, n), Q=f64(r + l, r), R=f64(r, r), Q2=f64(r, r), R2=f64(r, r),
               k=torch.full((1,), -1, dtype=torch.int32, device="cuda"))
    return dev


def test_batched_matches_unbatched_and_oracle(gn, H):
    probs = [_problem(gn, i, *s) for i, s in enumerate(SHAPES)]
    ws = H.batched_prepare(probs)
    H.batched_run(0.0, gn.PLAIN, ws)
    torch.cuda.synchronize()
    assert H.sync_status() == 0
    for (m, n, r), p in zip(SHAPES, probs):
        l = r // 2
        # unbatched path on the same operands
        wsu = H.workspace(m, n, r, l, gn.BF16)
        AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
        YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
        H.sketch(p["A"], p["X"], p["Y"], AX, YtA, wsu)
        # the unbatched core on the batched sketch: the QR comparisons below are exact-arithmetic ones
        core = gn.Core.empty(r, l, "cuda")
        H.core(p["YtA"], p["X"], 0.0, gn.PLAIN, core, wsu)
        torch.cuda.synchronize()
        assert torch.equal(p["AX"], AX)
        # Y^T A: the single launch may sum a long K in two halves; both are FP32
        # accumulations of the same products, within 2 m u32 (|Y|^T |A|) of each other
        Ya, Aa = p["Y"].double().abs(), p["A"].double().abs()
        bound = 2 * m * 2.0 ** -24 * (Ya.T @ Aa)
        assert torch.all((p["YtA"].double() - YtA.double()).abs() <= bound)
        assert int(p["k"].item()) == r
        C = core.C.cpu().numpy()
        Qb, Rb = p["Q"].cpu().numpy(), p["R"].cpu().numpy()
        # Householder QR of the same core: C = QR, Q^T Q = I, diag(R) >= 0, and the unbatched factors
        assert np.linalg.norm(C - Qb @ Rb) <= 1e-13 * np.linalg.norm(C)
        assert np.linalg.norm(Qb.T @ Qb - np.eye(r)) <= 1e-12
        assert np.all(np.diag(Rb) >= 0) and np.allclose(Rb, np.triu(Rb))
        kappa = np.linalg.cond(Rb)
        assert np.linalg.norm(Rb - core.R.cpu().numpy()) <= 1e-13 * kappa * np.linalg.norm(Rb)
        # and the oracle's QR of that core
        oq, orr = O.householder_qr(C)
        assert np.linalg.norm(Rb - orr) <= 1e-13 * kappa * np.linalg.norm(orr)


def test_batched_truncation_branch(gn, H):
    shapes = [(400, 300, 32), (600, 500, 64)]
    probs = [_problem(gn, 10 + i, *s, rankdef=True) for i, s in enumerate(shapes)]
    ws = H.batched_prepare(probs)
    eps = 1e-4
    H.batched_run(eps, gn.SGN | gn.EPS_RELATIVE, ws)
    torch.cuda.synchronize()
    assert H.sync_status() == 0
    for (m, n, r), p in zip(shapes, probs):
        l = r // 2
        wsu = H.workspace(m, n, r, l, gn.BF16)
        core = gn.Core.empty(r, l, "cuda")
        H.core(p["YtA"], p["X"], eps, gn.SGN | gn.EPS_RELATIVE, core, wsu)
        k = int(p["k"].item())
        assert k == core.k == r // 2
        Rb2, Ru2 = p["R2"].cpu().numpy()[:k, :k], core.R2.cpu().numpy()[:k, :k]
        assert np.linalg.norm(Rb2 - Ru2) <= 1e-9 * np.linalg.norm(Ru2)
        Qb2, Qu2 = p["Q2"].cpu().numpy()[:, :k], core.Q2.cpu().numpy()[:, :k]
        assert np.linalg.norm(Qb2 - Qu2) <= 1e-9 * np.linalg.norm(Qu2)


def _check_against_unbatched(gn, H, m, n, r, p):
    """AX bitwise equal to the unbatched launch; Y^T A within the FP32
    accumulation bound (the single launch may sum a long K in two halves)."""
    l = r // 2
    wsu = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    H.sketch(p["A"], p["X"], p["Y"], AX, YtA, wsu)
    torch.cuda.synchronize()
    assert torch.equal(p["AX"], AX)
    bound = 2 * m * 2.0 ** -24 * (p["Y"].double().abs().T @ p["A"].double().abs())
    assert torch.all((p["YtA"].double() - YtA.double()).abs() <= bound)


def test_batched_autotuner_keeps_results(gn, H):
    """The autotuner times every tile policy and keeps the fastest; the tile
    shape changes only the schedule, so every policy's sketches are bitwise
    equal to each other, agree with the unbatched path, and the cores are
    unchanged."""
    probs = [_problem(gn, 20 + i, *s) for i, s in enumerate(SHAPES)]
    ws = H.batched_prepare(probs)
    best, ms = H.batched_tune(0.0, gn.PLAIN, ws)
    assert best in (0, 1, 2, 4, 5, 6, 8, 9, 10, 12, 13, 14, 16, 17, 18, 20, 21, 22, 24, 25, 26, 28, 29, 30) and ms > 0
    for p in probs:
        p["AX"].fill_(float("nan"))
        p["YtA"].fill_(float("nan"))
    H.batched_run(0.0, gn.PLAIN, ws)
    torch.cuda.synchronize()
    assert H.sync_status() == 0
    ref = []
    for (m, n, r), p in zip(SHAPES, probs):
        _check_against_unbatched(gn, H, m, n, r, p)
        assert int(p["k"].item()) == r
        ref.append((p["AX"].clone(), p["YtA"].clone()))
    for pol in (1, 2, 4, 8, 14, 16, 30):   # every policy gives the same sketches
        H.batched_set_policy(pol)
        ws2 = H.batched_prepare(probs)
        H.batched_run(0.0, gn.PLAIN, ws2)
        torch.cuda.synchronize()
        for p, (ax, yta) in zip(probs, ref):
            assert torch.equal(p["AX"], ax) and torch.equal(p["YtA"], yta)
    H.batched_set_policy(0)


def test_batched_512_problem_batch_spot_parity(gn, H):
    """The bench's own batch: 512 problems, m ~ U[256,4096], n ~ U[128,m],
    r ~ U{16..128}, l = r/2, each W1 diag(2^(-i/10)) W2^T + 1e-8 N with its own
    seed, BF16 operands, AUTO mode with eps = 10 u32 relative.  On 16 sampled
    problems: both sketches against the oracle's products of the same
    (BF16-exact) operands within the FP32 accumulation bound, and the core
    against the oracle's Householder QR of (Y^T A) X formed from the GPU's
    sketch: C = QR to the FP32 level of the core product, Q orthonormal,
    diag(R) >= 0, R within kappa(R) times that level of the oracle's R, and k."""
    shapes = gn_synth.batched_shapes(512)
    probs = []
    for i, (m, n, r, l) in enumerate(shapes):
        p = gn_synth.config5_problem(i, (m, n, r, l), device="cuda")
        d = {"A": H.quantize(p.a), "X": H.quantize(p.x), "Y": H.quantize(p.y)}
        del p
        d["AX"] = torch.empty(m, r, dtype=torch.float32, device="cuda")
        d["YtA"] = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
        for nm, (a, b) in (("Q", (r + l, r)), ("R", (r, r)), ("Q2", (r, r)), ("R2", (r, r))):
            d[nm] = torch.empty(a, b, dtype=torch.float64, device="cuda")
        d["k"] = torch.empty(1, dtype=torch.int32, device="cuda")
        probs.append(d)
    ws = H.batched_prepare(probs)
    eps = 10 * 2.0 ** -24
    H.batched_run(eps, gn.AUTO | gn.EPS_RELATIVE, ws)
    torch.cuda.synchronize()
    assert H.sync_status() == 0
    rng = np.random.default_rng(512)
    for i in sorted(rng.choice(len(shapes), 16, replace=False)):
        m, n, r, l = shapes[i]
        p = probs[i]
        A, X, Y = (p[k].double().cpu().numpy() for k in ("A", "X", "Y"))
        oAX, oYtA = O.sketch(A, X, Y)
        assert np.all(np.abs(p["AX"].double().cpu().numpy() - oAX) <= 2 * n * 2.0 ** -24 * (np.abs(A) @ np.abs(X)))
        YtA = p["YtA"].double().cpu().numpy()
        assert np.all(np.abs(YtA - oYtA) <= 2 * m * 2.0 ** -24 * (np.abs(Y).T @ np.abs(A)))
        C = YtA @ X
        Qb, Rb = p["Q"].cpu().numpy(), p["R"].cpu().numpy()
        d = np.linalg.norm(C - Qb @ Rb) / np.linalg.norm(C)
        assert d <= 6 * n * 2.0 ** -24
        assert np.linalg.norm(Qb.T @ Qb - np.eye(r)) <= 1e-12 * r
        assert np.all(np.diag(Rb) >= 0) and np.allclose(Rb, np.triu(Rb))
        oc = O.core(YtA, X, eps, O.AUTO, eps_relative=True, diag_iters=6)
        kappa = np.linalg.cond(oc["R"])
        assert np.linalg.norm(Rb - oc["R"]) <= (10 * kappa * d + 1e-12) * np.linalg.norm(oc["R"])
        assert int(p["k"].item()) == oc["k"]
