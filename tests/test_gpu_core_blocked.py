"""The core's Householder QR in 256-column blocks (FP32 sketches, tensor-core
block updates, Q formed with the blocks' T) against the oracle's Householder
QR of the same C, at the shapes where the blocking has edges: exactly two
blocks (no side-stream update), a ragged last block, one extra row (l = 1),
and blocks with a tall core.  C is handed to gn_core (GN_CORE_C_GIVEN), so
the QR alone is compared.  Tolerances: each digit-sliced product errs by
~1e-13 of |A||B| per element; R and Q within 3e-11 of the oracle's relative to
their norms times the core's condition number over 100 (at least 1), Q
orthonormal to 1e-12 r and C = QR to 1e-11 relative."""
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


@pytest.mark.parametrize("r,l", [(512, 256), (520, 10), (768, 1), (700, 350)])
def test_blocked_core_qr_against_oracle(gn, H, r, l):
    n = 1024
    rng = np.random.default_rng(r + l)
    # a core with a decaying spectrum (singular values 1 .. 1e-3)
    U, _ = np.linalg.qr(rng.standard_normal((r + l, r)))
    V, _ = np.linalg.qr(rng.standard_normal((r, r)))
    C = (U * np.logspace(0, -3, r)) @ V.T
    YtA = torch.zeros(r + l, n, dtype=torch.float32, device="cuda")   # FP32 sketches: the tensor-core path
    X = H.quantize(torch.zeros(n, r, dtype=torch.float64, device="cuda"))
    ws = H.workspace(4096, n, r, l, gn.BF16)
    core = gn.Core.empty(r, l, "cuda")
    core.C.copy_(torch.from_numpy(C))
    H.set_fp64_tc(True)
    H.core(YtA, X, 0.0, gn.PLAIN | gn.CORE_C_GIVEN, core, ws)
    assert H.sync_status() == 0
    Q, R = core.Q.cpu().numpy(), core.R.cpu().numpy()
    Qo, Ro = O.householder_qr(C)
    kappa = max(1.0, np.linalg.cond(C) / 100)
    assert np.linalg.norm(R - Ro) <= 3e-11 * kappa * np.linalg.norm(Ro)
    assert np.linalg.norm(Q - Qo) <= 3e-11 * kappa * np.linalg.norm(Qo)
    assert np.linalg.norm(C - Q @ R) <= 1e-11 * np.linalg.norm(C)
    assert np.linalg.norm(Q.T @ Q - np.eye(r)) <= 1e-12 * r
    assert np.all(np.diag(R) >= 0)
