"""The adjoint of A -> A_hat on the GPU (through the C ABI) against the FP64
oracle's adjoint (itself pinned to central finite differences) and against
finite differences of the GPU forward map.  Tolerances: FP64 path 1e-9
relative to the oracle and 1e-6 to finite differences; FP32 contractions
1e-3 relative to the FP64 oracle gradient."""
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


def _case(m, n, r, l, seed, dtype=torch.float64):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * (0.9 ** np.arange(n))[None, :]
    X, Y = rng.standard_normal((n, r)), rng.standard_normal((m, r + l))
    G = rng.standard_normal((m, n))
    t = lambda a: torch.tensor(a, dtype=dtype, device="cuda")
    return (A, X, Y, G), (t(A), t(X), t(Y), t(G))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_forward_dense_matches_oracle(gn, H):
    (A, X, Y, _), (tA, tX, tY, _) = _case(120, 90, 12, 6, 1)
    ws = H.backward_workspace(120, 90, 12, 6, gn.F64)
    Ah = torch.empty_like(tA)
    H.forward_dense(tA, tX, tY, Ah, ws)
    ref, _ = O.gn(A, X, Y, 0.0, O.PLAIN)
    assert rel(Ah.cpu().numpy(), ref) <= 1e-10


def test_adjoint_fp64_fd_case(gn, H):
    """64 x 48, r = 8, l = 4 in FP64: oracle adjoint and central differences."""
    m, n, r, l = 64, 48, 8, 4
    (A, X, Y, G), (tA, tX, tY, tG) = _case(m, n, r, l, 2)
    ws = H.backward_workspace(m, n, r, l, gn.F64)
    dA = torch.empty_like(tA)
    H.backward(tA, tX, tY, tG, dA, ws)
    assert H.sync_status() == 0
    g = dA.cpu().numpy()
    assert rel(g, O.gn_backward(A, X, Y, G)) <= 1e-9
    # finite differences of the GPU forward map
    rng = np.random.default_rng(3)
    h = 1e-6 * np.linalg.norm(A)
    Ah = torch.empty_like(tA)

    def loss(Am):
        H.forward_dense(torch.tensor(Am, device="cuda"), tX, tY, Ah, ws)
        return float(torch.sum(tG * Ah).item())

    for _ in range(6):
        D = rng.standard_normal((m, n))
        D /= np.linalg.norm(D)
        fd = (loss(A + h * D) - loss(A - h * D)) / (2 * h)
        assert abs(fd - np.sum(g * D)) <= 1e-6 * max(1.0, np.linalg.norm(g))


def test_adjoint_fp32_against_fp64_reference(gn, H):
    m, n, r, l = 640, 384, 32, 16
    (A, X, Y, G), _ = _case(m, n, r, l, 4)
    t32 = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    A32, X32, Y32, G32 = (t32(a) for a in (A, X, Y, G))
    ws = H.backward_workspace(m, n, r, l, gn.F32)
    dA = torch.empty_like(A32)
    H.backward(A32, X32, Y32, G32, dA, ws)
    assert H.sync_status() == 0
    # reference on the FP32-rounded inputs, in FP64
    r64 = lambda t: t.double().cpu().numpy()
    ref = O.gn_backward(r64(A32), r64(X32), r64(Y32), r64(G32))
    assert rel(dA.double().cpu().numpy(), ref) <= 1e-3


def test_autograd_function_gradcheck(gn, H):
    m, n, r, l = 30, 22, 5, 3
    _, (tA, tX, tY, _) = _case(m, n, r, l, 5)
    tA.requires_grad_(True)
    f = lambda a: gn.gn_approx_dense(a, tX, tY, H)
    assert torch.autograd.gradcheck(f, (tA,), eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)
    # backward through a scalar loss equals the C-ABI adjoint
    Gup = torch.randn(m, n, dtype=torch.float64, device="cuda")
    (f(tA) * Gup).sum().backward()
    ws = H.backward_workspace(m, n, r, l, gn.F64)
    dA = torch.empty_like(tA)
    H.backward(tA.detach(), tX, tY, Gup, dA, ws)
    assert torch.allclose(tA.grad, dA, rtol=1e-12, atol=1e-12)


def test_adjoint_config4_fp32_against_oracle(gn, H):
    """The 4096 x 4096 FP32 case the bench times (sigma_i = i^-1.5 over 1024
    modes + 1e-6 noise, r = 256, l = 128): the FP32 GPU gradient against the
    FP64 oracle's adjoint on the same (FP32-rounded) inputs, 1e-3 relative."""
    import gn_synth
    m = n = 4096
    r, l = 256, 128
    p, G = gn_synth.config4(device="cuda", m=m, n=n, r=r, l=l, dtype=torch.float32)
    A, X, Y = p.a, p.x, p.y
    ws = H.backward_workspace(m, n, r, l, gn.F32)
    dA = torch.empty_like(A)
    H.backward(A, X, Y, G, dA, ws)
    assert H.sync_status() == 0
    h = lambda t: t.double().cpu().numpy()
    ref = O.gn_backward(h(A), h(X), h(Y), h(G))
    assert rel(h(dA), ref) <= 1e-3


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-6)])
def test_backward_saved_matches_backward(gn, H, dtype, tol):
    """gn_backward_saved from the front gn_forward_dense left in the workspace
    equals gn_backward (which forms the front again), for two Gup on one front;
    in FP64 also against the oracle's adjoint."""
    m, n, r, l = 320, 192, 16, 8
    (A, X, Y, G), (tA, tX, tY, tG) = _case(m, n, r, l, 6, dtype)
    G2 = torch.randn(m, n, dtype=dtype, device="cuda")
    dt = gn.F64 if dtype == torch.float64 else gn.F32
    ws = H.backward_workspace(m, n, r, l, dt)
    Ah = torch.empty_like(tA)
    H.forward_dense(tA, tX, tY, Ah, ws)
    saved = []
    for Gup in (tG, G2):
        dA = torch.empty_like(tA)
        H.backward_saved(tX, tY, Gup, dA, ws)
        saved.append(dA)
    assert H.sync_status() == 0
    ws2 = H.backward_workspace(m, n, r, l, dt)
    for Gup, dA in zip((tG, G2), saved):
        full = torch.empty_like(tA)
        H.backward(tA, tX, tY, Gup, full, ws2)
        assert H.sync_status() == 0
        assert torch.linalg.norm(dA - full) <= tol * torch.linalg.norm(full)
    if dtype == torch.float64:
        assert rel(saved[0].cpu().numpy(), O.gn_backward(A, X, Y, G)) <= 1e-9


def test_backward_saved_needs_the_matching_front(gn, H):
    """The handle keeps the front of its last gn_forward_dense / gn_backward:
    another workspace, other X or Y, or a later forward on another workspace
    make gn_backward_saved fail (GN_ERR_INVALID_ARG, checked on the host)."""
    m, n, r, l = 96, 64, 8, 4
    _, (tA, tX, tY, tG) = _case(m, n, r, l, 7)
    ws1 = H.backward_workspace(m, n, r, l, gn.F64)
    ws2 = H.backward_workspace(m, n, r, l, gn.F64)
    Ah, dA = torch.empty_like(tA), torch.empty_like(tA)
    H.forward_dense(tA, tX, tY, Ah, ws1)
    with pytest.raises(gn.GNError) as e:
        H.backward_saved(tX, tY, tG, dA, ws2)
    assert e.value.status == 1
    with pytest.raises(gn.GNError):
        H.backward_saved(tX.clone(), tY, tG, dA, ws1)
    H.backward_saved(tX, tY, tG, dA, ws1)          # the matching front
    H.forward_dense(tA, tX, tY, Ah, ws2)           # replaces the record
    with pytest.raises(gn.GNError):
        H.backward_saved(tX, tY, tG, dA, ws1)
    assert H.sync_status() == 0


def test_autograd_uses_the_saved_front(gn, H):
    """The autograd wrapper's backward from the forward's front equals the
    C-ABI adjoint, and so does a backward after another forward on the same
    handle (which re-forms the front)."""
    m, n, r, l = 40, 30, 6, 3
    _, (tA, tX, tY, _) = _case(m, n, r, l, 8)
    Gup = torch.randn(m, n, dtype=torch.float64, device="cuda")
    ws = H.backward_workspace(m, n, r, l, gn.F64)
    ref = torch.empty_like(tA)
    H.backward(tA, tX, tY, Gup, ref, ws)
    a1 = tA.clone().requires_grad_(True)
    (gn.gn_approx_dense(a1, tX, tY, H) * Gup).sum().backward()
    a2 = tA.clone().requires_grad_(True)
    out2 = gn.gn_approx_dense(a2, tX, tY, H)
    gn.gn_approx_dense(tA.clone(), tX, tY, H)      # another forward on the handle
    (out2 * Gup).sum().backward()
    for g in (a1.grad, a2.grad):
        assert torch.allclose(g, ref, rtol=1e-12, atol=1e-12)
