"""The core without a host wait (GN_CORE_DEFER + gn_core_finish), failure
detection on the device (a bounded wait that runs out, a non-finite core), and
two approximations in flight on two handles.

No test here faults, traps or hangs the GPU: the timeout test turns on the
library's test hook, under which the sketch kernel's epilogue waits on a
barrier that nothing completes; that bounded wait runs out after a 50 ms
limit, the kernel latches GN_ERR_TIMEOUT, drains its own copies and MMAs (those
waits keep at least a second) and returns; the context stays usable and the
next call is checked."""
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


def _ints(g, a, b):
    return torch.randint(-3, 4, (a, b), generator=g).double()


def _problem(gn, H, m, n, r, l, seed):
    g = torch.Generator().manual_seed(seed)
    A, X, Y = _ints(g, m, n), _ints(g, n, r), _ints(g, m, r + l)
    return (A, X, Y), tuple(H.quantize(t.cuda()) for t in (A, X, Y))


def test_deferred_core_equals_blocking_core(gn):
    """Same inputs through gn_core with and without GN_CORE_DEFER (AUTO mode):
    identical Q, R and host fields once gn_core_finish has run."""
    m, n, r, l = 900, 700, 96, 48
    H1, H2 = gn.Handle(), gn.Handle()
    (A, X, Y), (Ab, Xb, Yb) = _problem(gn, H1, m, n, r, l, 3)
    ws1, ws2 = H1.workspace(m, n, r, l, gn.BF16), H2.workspace(m, n, r, l, gn.BF16)
    out = []
    for H, ws, defer in ((H1, ws1, True), (H2, ws2, False)):
        AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
        YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
        c = gn.Core.empty(r, l, "cuda")
        H.sketch(Ab, Xb, Yb, AX, YtA, ws)
        mode = gn.AUTO | gn.EPS_RELATIVE | (gn.CORE_DEFER if defer else 0)
        H.core(YtA, Xb, 10 * 2.0 ** -24, mode, c, ws)
        if defer:
            assert c.k == -1 and c.sgn == -1      # pending until finished
            H.core_finish(c)
        out.append(c)
    torch.cuda.synchronize()
    assert H1.sync_status() == 0 and H2.sync_status() == 0
    c1, c2 = out
    assert (c1.k, c1.sgn) == (c2.k, c2.sgn) == (r, 0)
    assert c1.rinv_est == c2.rinv_est and c1.eps_abs == c2.eps_abs
    assert torch.equal(c1.Q, c2.Q) and torch.equal(c1.R, c2.R)
    # and the R of the oracle's Householder QR of the same (exact) core matrix
    oAX, oYtA = O.sketch(A.numpy(), X.numpy(), Y.numpy())
    _, oR = O.householder_qr(oYtA @ X.numpy())
    assert np.linalg.norm(c1.R.cpu().numpy() - oR) <= 1e-12 * np.linalg.norm(oR)
    # finishing twice is harmless; finishing a core that is not pending is not
    H1.core_finish(c1)
    c3 = gn.Core.empty(r, l, "cuda")
    c3.k = -1
    with pytest.raises(gn.GNError):
        H1.core_finish(c3)
    H1.close()
    H2.close()


def test_two_approximations_in_flight(gn):
    """Two handles on two streams, each step's core deferred and finished after
    the next step is enqueued (the bench's pipelined loop): every step's Q and R
    equal those of the same problem run alone."""
    m, n, r, l = 1200, 800, 128, 64
    Hs = [gn.Handle(torch.cuda.Stream()) for _ in range(2)]
    probs = [_problem(gn, Hs[0], m, n, r, l, 20 + i) for i in range(4)]
    torch.cuda.synchronize()
    ws = [H.workspace(m, n, r, l, gn.BF16) for H in Hs]
    mode = gn.AUTO | gn.EPS_RELATIVE
    eps = 10 * 2.0 ** -24
    res = []
    pending = None
    for i, (_, (Ab, Xb, Yb)) in enumerate(probs):
        H = Hs[i % 2]
        AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
        YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
        c = gn.Core.empty(r, l, "cuda")
        H.sketch(Ab, Xb, Yb, AX, YtA, ws[i % 2])
        H.core(YtA, Xb, eps, mode | gn.CORE_DEFER, c, ws[i % 2])
        if pending is not None:
            pending[0].core_finish(pending[1])
        pending = (H, c)
        res.append(c)
    pending[0].core_finish(pending[1])
    torch.cuda.synchronize()
    H1 = gn.Handle()
    w1 = H1.workspace(m, n, r, l, gn.BF16)
    for c, (_, (Ab, Xb, Yb)) in zip(res, probs):
        AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
        YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
        ref = gn.Core.empty(r, l, "cuda")
        H1.sketch(Ab, Xb, Yb, AX, YtA, w1)
        H1.core(YtA, Xb, eps, mode, ref, w1)
        torch.cuda.synchronize()
        assert c.k == ref.k and torch.equal(c.R, ref.R) and torch.equal(c.Q, ref.Q)
    for H in Hs + [H1]:
        assert H.sync_status() == 0
        H.close()


def test_nonfinite_input_latched(gn):
    """A NaN in A reaches every later column of R: AUTO mode returns
    GN_ERR_NONFINITE (the estimates are NaN) and the device status word holds
    it; PLAIN mode latches it on the device.  A clean call afterwards works."""
    m, n, r, l = 600, 500, 64, 32
    H = gn.Handle()
    (A, X, Y), (Ab, Xb, Yb) = _problem(gn, H, m, n, r, l, 9)
    A_nan = A.clone()
    A_nan[17, 5] = float("nan")
    Anb = H.quantize(A_nan.cuda())
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    c = gn.Core.empty(r, l, "cuda")
    H.sketch(Anb, Xb, Yb, AX, YtA, ws)
    with pytest.raises(gn.GNError) as ei:
        H.core(YtA, Xb, 10 * 2.0 ** -24, gn.AUTO | gn.EPS_RELATIVE, c, ws)
    assert ei.value.status == 6
    assert H.sync_status() == 6
    H.sketch(Anb, Xb, Yb, AX, YtA, ws)
    H.core(YtA, Xb, 0.0, gn.PLAIN, c, ws)
    assert H.sync_status() == 6
    assert H.sync_status() == 0            # reading the status clears it
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    H.core(YtA, Xb, 10 * 2.0 ** -24, gn.AUTO | gn.EPS_RELATIVE, c, ws)
    assert H.sync_status() == 0 and c.k == r
    H.close()


def test_sketch_wait_limit_expires_and_recovers(gn):
    """The timeout path: with the test hook on, the sketch kernel's epilogue
    waits on a barrier that nothing completes; after the 50 ms limit that wait
    latches GN_ERR_TIMEOUT (7), the launch stops, its producer and MMA roles
    drain their own copies and MMAs and free tensor memory, and the kernel
    returns.  With the hook off and the default limit, the next sketch on the
    same handle is exact (integer inputs)."""
    import time
    m, n, r, l = 1024, 4096, 128, 64
    H = gn.Handle()
    (A, X, Y), (Ab, Xb, Yb) = _problem(gn, H, m, n, r, l, 12)
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device="cuda")
    YtA = torch.empty(r + l, n, dtype=torch.float32, device="cuda")
    H.set_wait_limit(50_000_000)
    H.set_stall_test(True)
    t0 = time.perf_counter()
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    st = H.sync_status()
    dt = time.perf_counter() - t0
    H.set_stall_test(False)
    H.set_wait_limit(2_000_000_000)
    assert st == 7
    assert dt < 5.0
    AX.fill_(float("nan"))
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    assert H.sync_status() == 0
    oAX, oYtA = O.sketch(A.numpy(), X.numpy(), Y.numpy())
    assert np.array_equal(AX.double().cpu().numpy(), oAX)
    assert np.array_equal(YtA.double().cpu().numpy(), oYtA)
    H.close()
