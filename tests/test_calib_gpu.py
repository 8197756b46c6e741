"""FP32 calibration kernels (forward, loss, hand-written backward) against the
FP64 CPU reference in oracle/calib.py: analytic gradient and central finite
differences, relative error 1e-4; the integer table is not involved."""
import numpy as np
import pytest

from oracle import calib as ref
from paper_1311_0380_gb300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def make(n, S, seed):
    consts = synth.make_constants(S)
    return synth.make_calib(n, consts, seed=seed)


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check_grad(dF, dq, rF, rq):
    assert rel_err(dF, rF) <= REL, rel_err(dF, rF)
    assert rel_err(dq, rq) <= REL, rel_err(dq, rq)
    for got, want in ((dF, rF), (dq, rq)):
        big = np.abs(want) > 1e-3 * np.abs(want).max()
        err = np.abs(got[big] - want[big]) / np.abs(want[big])
        assert err.max() <= REL, err.max()


@pytest.mark.parametrize("n,S", [(2000, 4), (20000, 64), (1 << 20, 512)])
def test_loss_and_gradient_match_fp64(n, S):
    import torch
    from paper_1311_0380_gb300 import calib
    cs = make(n, S, seed=n + S)
    data = calib.CalibData(cs.x, cs.sector, cs.theta, S, cs.weight)
    F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
    q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
    loss = calib.calib_loss(F, q, data)
    loss.backward()
    L64 = ref.loss(cs.x, cs.sector, cs.theta, cs.weight, cs.F0, cs.q0)
    assert abs(loss.item() - L64) <= REL * abs(L64)
    rF, rq = ref.grad(cs.x, cs.sector, cs.theta, cs.weight, cs.F0, cs.q0)
    check_grad(F.grad.cpu().numpy(), q.grad.cpu().numpy(), rF, rq)


def test_gradient_matches_fp64_finite_differences():
    import torch
    from paper_1311_0380_gb300 import calib
    S = 4
    cs = make(4000, S, seed=5)
    data = calib.CalibData(cs.x, cs.sector, cs.theta, S, cs.weight)
    F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
    q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
    calib.calib_loss(F, q, data).backward()
    rng = np.random.default_rng(1)
    entries = [("F", *map(int, rng.integers(0, [S, 6, 6]))) for _ in range(40)]
    entries += [("q", *map(int, rng.integers(0, [S, 6]))) for _ in range(16)]
    fd = ref.fd_grad(cs.x, cs.sector, cs.theta, cs.weight, cs.F0, cs.q0, entries)
    gF, gq = F.grad.cpu().numpy(), q.grad.cpu().numpy()
    got = np.array([gF[e[1:]] if e[0] == "F" else gq[e[1:]] for e in entries])
    scale = np.abs(fd).max()
    big = np.abs(fd) > 1e-3 * scale
    assert np.max(np.abs(got[big] - fd[big]) / np.abs(fd[big])) <= REL


def test_forward_and_general_backward():
    import torch
    from paper_1311_0380_gb300 import calib
    S = 16
    cs = make(30000, S, seed=7)
    data = calib.CalibData(cs.x, cs.sector, cs.theta, S, cs.weight)
    perm = data.perm.cpu().numpy()
    F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
    q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
    y = calib.fit_fp32(F, q, data)
    y64 = ref.forward(cs.x, cs.sector, cs.F0, cs.q0)[perm]
    scale = np.abs(cs.F0).sum(axis=2).max() * 32768
    assert np.max(np.abs(y.detach().cpu().numpy() - y64)) <= 1e-6 * scale
    # sorted order really is by sector, stable
    s_sorted = cs.sector[perm]
    assert np.all(np.diff(s_sorted) >= 0)
    for s in range(S):
        idx = perm[s_sorted == s]
        assert np.all(np.diff(idx) > 0)
    gy = torch.randn_like(y)
    (y * gy).sum().backward()
    g = gy.cpu().numpy().astype(np.float64)
    x = cs.x[perm].astype(np.float64)
    rF = np.zeros((S, 6, 6))
    rq = np.zeros((S, 6))
    np.add.at(rF, s_sorted, g[:, :, None] * x[:, None, :])
    np.add.at(rq, s_sorted, g)
    check_grad(F.grad.cpu().numpy(), q.grad.cpu().numpy(), rF, rq)


def test_results_are_bitwise_reproducible():
    import torch
    from paper_1311_0380_gb300 import calib
    S = 32
    cs = make(50000, S, seed=9)
    out = []
    for _ in range(2):
        data = calib.CalibData(cs.x, cs.sector, cs.theta, S, cs.weight)
        F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
        q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
        loss = calib.calib_loss(F, q, data)
        loss.backward()
        out.append((loss.item(), F.grad.cpu().numpy().copy(), q.grad.cpu().numpy().copy()))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_calibration_descent_reduces_loss():
    import torch
    from paper_1311_0380_gb300 import calib
    S = 8
    cs = make(40000, S, seed=11)
    data = calib.CalibData(cs.x, cs.sector, cs.theta, S, cs.weight)
    F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
    q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([F, q], lr=1e-4)
    first = None
    for _ in range(60):
        opt.zero_grad()
        loss = calib.calib_loss(F, q, data)
        if first is None:
            first = loss.item()
        loss.backward()
        opt.step()
    assert calib.calib_loss(F, q, data).item() < 0.7 * first


def test_fused_and_unfused_paths_empty_sectors_and_upstream_scale():
    """The fused loss-and-gradient pass and the separate backward pass both
    match the FP64 gradient; sectors without tracks get exactly zero; an
    upstream gradient of 3 scales the result; the loss without a gradient
    request uses the loss-only pass and gives the same value."""
    import torch
    from paper_1311_0380_gb300 import calib
    S = 64
    cs = make(20000, S, seed=21)
    sector = (cs.sector % 41).astype(np.int32)          # sectors 41..63 stay empty
    data = calib.CalibData(cs.x, sector, cs.theta, S, cs.weight)
    rF, rq = ref.grad(cs.x, sector, cs.theta, cs.weight, cs.F0, cs.q0)
    L64 = ref.loss(cs.x, sector, cs.theta, cs.weight, cs.F0, cs.q0)
    for fused in (True, False):
        F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
        q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
        loss = calib.calib_loss(F, q, data, fused=fused)
        assert abs(loss.item() - L64) <= REL * abs(L64)
        (3.0 * loss).backward()
        gF, gq = F.grad.cpu().numpy(), q.grad.cpu().numpy()
        check_grad(gF / 3.0, gq / 3.0, rF, rq)
        assert np.all(gF[41:] == 0) and np.all(gq[41:] == 0)
    with torch.no_grad():
        F = torch.tensor(cs.F0, device="cuda")
        q = torch.tensor(cs.q0, device="cuda")
        l0 = calib.calib_loss(F, q, data).item()
    assert abs(l0 - L64) <= REL * abs(L64)


def test_fused_pass_on_one_track_and_on_no_tracks():
    import torch
    from paper_1311_0380_gb300 import calib
    S = 4
    cs = make(2000, S, seed=23)
    for n in (1, 0):
        data = calib.CalibData(cs.x[:n], cs.sector[:n], cs.theta[:n], S, cs.weight)
        F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
        q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
        loss = calib.calib_loss(F, q, data)
        loss.backward()
        if n == 0:
            assert loss.item() == 0.0
            assert np.all(F.grad.cpu().numpy() == 0) and np.all(q.grad.cpu().numpy() == 0)
        else:
            L64 = ref.loss(cs.x[:n], cs.sector[:n], cs.theta[:n], cs.weight, cs.F0, cs.q0)
            assert abs(loss.item() - L64) <= REL * abs(L64)
            rF, rq = ref.grad(cs.x[:n], cs.sector[:n], cs.theta[:n], cs.weight, cs.F0, cs.q0)
            check_grad(F.grad.cpu().numpy(), q.grad.cpu().numpy(), rF, rq)


def test_loss_and_fit_in_one_pass_match_the_separate_calls():
    """calib_loss_and_fit gives the fitted parameters bit for bit as the
    forward kernel writes them, the same loss and gradient as calib_loss, and
    repeated calls on one CalibData (whose workspace keeps the pass's
    tickets) give identical bits."""
    import torch
    from paper_1311_0380_gb300 import calib
    S = 32
    cs = make(60000, S, seed=31)
    data = calib.CalibData(cs.x, cs.sector, cs.theta, S, cs.weight)
    runs = []
    for _ in range(3):
        F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
        q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
        loss, y = calib.calib_loss_and_fit(F, q, data)
        loss.backward()
        runs.append((loss.item(), y.cpu().numpy(), F.grad.cpu().numpy(), q.grad.cpu().numpy()))
    for r in runs[1:]:
        assert r[0] == runs[0][0]
        assert all(np.array_equal(a, b) for a, b in zip(r[1:], runs[0][1:]))
    F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
    q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
    y_ref = calib.fit_fp32(F, q, data).detach().cpu().numpy()
    assert np.array_equal(runs[0][1], y_ref)
    loss = calib.calib_loss(F, q, data)
    loss.backward()
    assert loss.item() == runs[0][0]
    assert np.array_equal(F.grad.cpu().numpy(), runs[0][2])
    rF, rq = ref.grad(cs.x, cs.sector, cs.theta, cs.weight, cs.F0, cs.q0)
    check_grad(runs[0][2], runs[0][3], rF, rq)


@pytest.mark.parametrize("n", [1, 3, 5, 7, 1029, 4099, 70001])
def test_staged_and_register_passes_on_ragged_sizes(n):
    """The fused pass stages each item's tracks in shared memory by bulk
    copies when x and theta start on 16-byte boundaries (copies widened to
    multiples of four tracks and cut below n; the last tracks past the cut
    read directly; final sums in a second, dependent kernel), and loads them
    per lane otherwise (final sums by tickets).  Both match the FP64 loss and
    gradient, give exactly zero for sectors without tracks, write the same y
    bit for bit, and leave the workspace's tickets and flag at zero, for
    sizes that are not multiples of four, with sectors of one to a few
    tracks."""
    import torch
    from paper_1311_0380_gb300 import _native as N, calib
    from paper_1311_0380_gb300.api import _p, _stream
    S = 16
    cs = make(max(n, 8), S, seed=n)
    x, theta = cs.x[:n], cs.theta[:n]
    sector = (cs.sector[:n] % 11).astype(np.int32)       # sectors 11, 14, 15 stay empty
    if n > 40:
        sector[-3:] = 12                                 # sectors of three and five tracks
        sector[:5] = 13
    data = calib.CalibData(x, sector, theta, S, cs.weight)
    F = torch.tensor(cs.F0, device="cuda", dtype=torch.float32)
    q = torch.tensor(cs.q0, device="cuda", dtype=torch.float32)
    L = N.load()
    L64 = ref.loss(x, sector, theta, cs.weight, cs.F0, cs.q0)
    rF, rq = ref.grad(x, sector, theta, cs.weight, cs.F0, cs.q0)
    # the same sorted tracks off 16-byte boundaries (x keeps the 8 bytes its
    # pair loads need)
    xu = torch.zeros(n * 6 + 4, dtype=torch.float32, device="cuda")
    tu = torch.zeros(n * 3 + 4, dtype=torch.float32, device="cuda")
    xu[2:2 + n * 6] = data.x[:n].reshape(-1)
    tu[1:1 + n * 3] = data.theta[:n].reshape(-1)
    ys = []
    for xp, tp in ((data.x.data_ptr(), data.theta.data_ptr()),
                   (xu.data_ptr() + 8, tu.data_ptr() + 4)):
        assert ((xp | tp) % 16 == 0) == (xp == data.x.data_ptr())
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        dF = torch.empty_like(F)
        dq = torch.empty_like(q)
        y = torch.empty((n, 6), dtype=torch.float32, device="cuda")
        N.check(L.svt_calib_loss_grad(xp, tp, _p(data.w), n, S, _p(data.index), _p(F), _p(q),
                                      _p(loss), _p(dF), _p(dq), _p(y), _p(data.workspace),
                                      data.workspace.numel(), _stream(None)),
                "svt_calib_loss_grad")
        torch.cuda.synchronize()
        assert abs(loss.item() - L64) <= REL * abs(L64)
        check_grad(dF.cpu().numpy(), dq.cpu().numpy(), rF, rq)
        empty = np.setdiff1d(np.arange(S), sector)
        assert np.all(dF.cpu().numpy()[empty] == 0) and np.all(dq.cpu().numpy()[empty] == 0)
        ys.append(y.cpu().numpy())
        lo = torch.empty(1, dtype=torch.float32, device="cuda")   # the loss alone
        N.check(L.svt_calib_loss(xp, tp, _p(data.w), n, S, _p(data.index), _p(F), _p(q),
                                 _p(lo), _p(data.workspace), data.workspace.numel(),
                                 _stream(None)), "svt_calib_loss")
        assert abs(lo.item() - L64) <= REL * abs(L64)
        g = torch.tensor([2.5], dtype=torch.float32, device="cuda")   # the separate backward
        bF, bq = torch.empty_like(F), torch.empty_like(q)
        N.check(L.svt_calib_loss_backward(xp, tp, _p(data.w), n, S, _p(data.index), _p(F), _p(q),
                                          _p(g), _p(bF), _p(bq), _p(data.workspace),
                                          data.workspace.numel(), _stream(None)),
                "svt_calib_loss_backward")
        check_grad(bF.cpu().numpy() / 2.5, bq.cpu().numpy() / 2.5, rF, rq)
        tail = ((S + 2) * 4 + 255) // 256 * 256           # the tickets and the flag, last
        assert not data.workspace[-tail:].any()
    assert np.array_equal(ys[0], ys[1])


def _calib_flag_offset(n, S):
    """Byte offset of the staged pass's copy-wait flag in the workspace:
    item losses, item partials (42 per item), sector losses, the loss, then
    the tickets (S per sector, the batch's, the flag), each at a multiple of
    256 bytes."""
    items = (n + 255) // 256 + S
    off = 0
    for count in (items, items * 42, S, 1):
        off = (off + 255) // 256 * 256 + 4 * count
    return (off + 255) // 256 * 256 + 4 * (S + 1)


def test_staged_pass_reports_a_failed_copy_wait_as_nan():
    """A copy wait that gives up sets the workspace's flag; the final kernel
    then writes a NaN loss and clears the flag.  The flag is set here from
    the host (no copy is made to fail), so the next call is clean again."""
    import torch
    from paper_1311_0380_gb300 import calib
    S = 8
    cs = make(5000, S, seed=41)
    data = calib.CalibData(cs.x, cs.sector, cs.theta, S, cs.weight)
    F = torch.tensor(cs.F0, device="cuda", requires_grad=True)
    q = torch.tensor(cs.q0, device="cuda", requires_grad=True)
    off = _calib_flag_offset(data.n, S)
    assert data.workspace.numel() >= off + 4
    flag = data.workspace[off:off + 4]
    assert not flag.any()
    flag.copy_(torch.tensor([1, 0, 0, 0], dtype=torch.uint8, device="cuda"))
    loss = calib.calib_loss(F, q, data)
    assert np.isnan(loss.item())
    assert not flag.any()                                  # cleared by the call
    L64 = ref.loss(cs.x, cs.sector, cs.theta, cs.weight, cs.F0, cs.q0)
    loss = calib.calib_loss(F, q, data)
    assert abs(loss.item() - L64) <= REL * abs(L64)
