"""Ahat W and W Ahat without forming Ahat (gn_apply), against the oracle's
apply_right / apply_left on the same sketches and core, and against the
formed factors F G."""
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


def npy(t):
    return t.detach().double().cpu().numpy()


def _run(gn, H, m, n, r, l, mixed, zero_cols=0, seed=0):
    A = gn_synth.gaussian((m, n), 81 + seed, 0) * (0.97 ** torch.arange(n, dtype=torch.float64))[None, :]
    X, Y = gn_synth.sketches(m, n, r, l, 82 + seed)
    X = X.clone()
    if zero_cols:
        X[:, r - zero_cols:] = 0.0                       # exactly singular core: the truncated branch
    eps, mode = (10 * 2.0 ** -24, gn.AUTO | gn.EPS_RELATIVE) if mixed else (10 * 2.0 ** -53, gn.AUTO | gn.EPS_RELATIVE)
    if mixed:
        Ad, Xd, Yd = H.quantize(A.cuda()), H.quantize(X.cuda()), H.quantize(Y.cuda())
        ws = H.workspace(m, n, r, l, gn.BF16)
        dt = torch.float32
    else:
        Ad, Xd, Yd = A.cuda(), X.cuda(), Y.cuda()
        ws = H.workspace(m, n, r, l, gn.F64)
        dt = torch.float64
    AX = torch.empty(m, r, dtype=dt, device="cuda")
    YtA = torch.empty(r + l, n, dtype=dt, device="cuda")
    F = torch.zeros(m, r, dtype=torch.float64, device="cuda")
    G = torch.zeros(r, n, dtype=torch.float64, device="cuda")
    core = gn.Core.empty(r, l, "cuda")
    H.approx(Ad, Xd, Yd, eps, mode, AX, YtA, core, F, G, ws)
    assert H.sync_status() == 0
    return AX, YtA, core, F, G


def _oracle_core(core):
    k = core.k
    c = dict(Q=npy(core.Q), R=npy(core.R), k=k, Q2=None, R2=None)
    if core.sgn and k < core.r:
        c["Q2"] = npy(core.Q2)[:, :k]
        c["R2"] = npy(core.R2)[:k, :k]
    return c


@pytest.mark.parametrize("mixed,zero_cols", [(True, 0), (True, 7), (False, 0), (False, 5)])
def test_apply_both_sides_against_oracle(gn, H, mixed, zero_cols):
    m, n, r, l = 900, 700, 60, 30
    AX, YtA, core, F, G = _run(gn, H, m, n, r, l, mixed, zero_cols)
    if zero_cols:
        assert core.sgn == 1 and core.k == r - zero_cols
    rng = np.random.default_rng(9)
    W = rng.standard_normal((n, 7))
    Wl = rng.standard_normal((5, m))
    out_r = H.apply(AX, YtA, core, torch.from_numpy(W).cuda(), side=0)
    out_l = H.apply(AX, YtA, core, torch.from_numpy(Wl).cuda(), side=1)
    assert H.sync_status() == 0
    c = _oracle_core(core)
    ref_r = O.apply_right(npy(AX), npy(YtA), c, W)
    ref_l = O.apply_left(Wl, npy(AX), npy(YtA), c)
    assert np.linalg.norm(npy(out_r) - ref_r) <= 1e-10 * np.linalg.norm(ref_r)
    assert np.linalg.norm(npy(out_l) - ref_l) <= 1e-10 * np.linalg.norm(ref_l)
    # the same operator as the formed factors (for FP32 sketches G is formed to
    # FP32-level accuracy on the tensor cores, so the agreement is at that level)
    k = core.k
    FG = npy(F)[:, :k] @ npy(G)[:k]
    tol = 1e-5 if mixed else 1e-9
    assert np.linalg.norm(npy(out_r) - FG @ W) <= tol * np.linalg.norm(FG @ W)
    assert np.linalg.norm(npy(out_l) - Wl @ FG) <= tol * np.linalg.norm(Wl @ FG)


def test_apply_rejects_mismatched_operands(gn, H):
    m, n, r, l = 300, 200, 20, 10
    AX, YtA, core, _, _ = _run(gn, H, m, n, r, l, True, seed=3)
    W = torch.zeros(n + 1, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(gn.GNError):
        H.apply(AX, YtA, core, W, side=0)
    W32 = torch.zeros(n, 3, dtype=torch.float32, device="cuda")
    with pytest.raises(gn.GNError):
        H.apply(AX, YtA, core, W32, side=0)
