"""qsi_bta_solve: the whole solve in one call, captured as a CUDA graph on the
context's (non-default) stream and replayed while the buffers repeat.  Every
call's result bitwise equal to factor + backward sweep on the same inputs,
including replays after the inputs changed in place, a new buffer set
(re-capture), SI only, several right-hand sides and the direct path on the
legacy default stream."""
import numpy as np
import pytest

from conftest import make_problem
from oracle import rgf
from paper_2601_04904_gb300 import inputs
from paper_2601_04904_gb300.metrics import max_block_rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04904_gb300 import qsi

    return torch, qsi


def _ref(ctx, qsi, Ad, Bds, prec):
    f = ctx.factor_multi(Ad, Bds, prec)
    if Bds:
        R, X = ctx.selquad_multi(f)
    else:
        R, X = ctx.selinv(f), []
    ctx.synchronize()
    f.close()
    return R, X


def _same(qsi, x, y):
    for key in qsi.KEYS:
        assert np.array_equal(x[key].cpu().numpy(), y[key].cpu().numpy()), key


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
@pytest.mark.parametrize("k", [1, 0, 2])
def test_solve_graph_replays_match_factor_path(env, prec_name, k):
    torch, qsi = env
    prec = getattr(qsi, prec_name)
    n, b, a = 4, 40, 16
    _, A, _ = make_problem(n, b, a, seed=41)
    Bs = [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 400 + r) for r in range(k)]
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    Ad = qsi.to_device(A)
    Bds = [qsi.to_device(B) for B in Bs]
    GR = qsi.device_zeros(n, b, a)
    GX = [qsi.device_zeros(n, b, a) for _ in range(k)]
    torch.cuda.synchronize()
    for call in range(3):
        if call == 2:  # new values in the same buffers: the replay must read them
            _, A2, _ = make_problem(n, b, a, seed=42)
            Ad["diag"].copy_(torch.from_numpy(A2["diag"]).to(Ad["diag"].device))
            for Bd in Bds:
                Bd["diag"].mul_(0.5)
            torch.cuda.synchronize()
        ctx.solve(Ad, Bds, GR, GX, prec)
        ctx.synchronize()
        R, X = _ref(ctx, qsi, Ad, Bds, prec)
        _same(qsi, GR, R)
        for r in range(k):
            _same(qsi, GX[r], X[r])
    # against the oracle as well (inputs of the last call)
    Ah = qsi.to_host(Ad)
    assert max_block_rel_err(qsi.to_host(GR), rgf.selinv(Ah)) < TOL
    for r in range(k):
        assert max_block_rel_err(qsi.to_host(GX[r]), rgf.selquad(Ah, qsi.to_host(Bds[r]))[1]) < TOL
    ctx.close()


def test_solve_new_buffers_recapture_and_default_stream(env):
    torch, qsi = env
    n, b, a = 3, 24, 8
    _, A, B = make_problem(n, b, a, seed=43)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    Ad, Bd = qsi.to_device(A), qsi.to_device(B)
    torch.cuda.synchronize()
    outs = []
    for _ in range(2):  # two buffer sets, alternating: every call re-captures
        GR, GX = qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)]
        torch.cuda.synchronize()
        ctx.solve(Ad, [Bd], GR, GX, qsi.FP64_EMU)
        ctx.synchronize()
        outs.append((GR, GX))
    R, X = _ref(ctx, qsi, Ad, [Bd], qsi.FP64_EMU)
    for GR, GX in outs:
        _same(qsi, GR, R)
        _same(qsi, GX[0], X[0])
    ctx.close()
    # legacy default stream: the direct path, same bits
    ctx0 = qsi.Context(0)
    GR0, GX0 = ctx0.solve(Ad, [Bd], precision=qsi.FP64_EMU)
    ctx0.synchronize()
    _same(qsi, GR0, R)
    _same(qsi, GX0[0], X[0])
    ctx0.close()


def test_solve_counts_replayed_launches(env):
    torch, qsi = env
    n, b, a = 3, 32, 8
    _, A, B = make_problem(n, b, a, seed=44)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    Ad, Bd = qsi.to_device(A), qsi.to_device(B)
    GR, GX = qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)]
    torch.cuda.synchronize()
    ctx.solve(Ad, [Bd], GR, GX, qsi.FP64_EMU)  # direct + capture
    ctx.synchronize()
    ctx.stats_reset(False)
    ctx.solve(Ad, [Bd], GR, GX, qsi.FP64_EMU)  # replay
    ctx.synchronize()
    per_replay = ctx.stats()["launches"]
    ctx.stats_reset(False)
    f = ctx.factor(Ad, Bd, qsi.FP64_EMU)
    ctx.selquad(f)
    ctx.synchronize()
    f.close()
    assert per_replay == ctx.stats()["launches"] > 0
    ctx.close()


def test_host_entry_repeats_bitwise(env):
    """qsi_bta_selquad_host on a stream context: staging kept, the second call
    replays the captured solve; both equal the device factor path."""
    torch, qsi = env
    n, b, a = 3, 40, 8
    _, A, B = make_problem(n, b, a, seed=45)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    shapes = {"diag": (n, b, b), "upper": (n - 1, b, b), "lower": (n - 1, b, b),
              "arrow_r": (n, b, a), "arrow_b": (n, a, b), "tip": (a, a)}
    Rd, Xd = _ref(ctx, qsi, qsi.to_device(A), [qsi.to_device(B)], qsi.FP64_EMU)
    for _ in range(3):
        GR = {k: np.zeros(s, np.complex128) for k, s in shapes.items()}
        GL = {k: np.zeros(s, np.complex128) for k, s in shapes.items()}
        ctx.selquad_host(A, B, GR, GL, qsi.FP64_EMU)
        for key in qsi.KEYS:
            assert np.array_equal(GR[key], Rd[key].cpu().numpy()), key
            assert np.array_equal(GL[key], Xd[0][key].cpu().numpy()), key
    ctx.close()


@pytest.mark.parametrize("diag_only", [False, True])
def test_host_entry_pinned_overlapped(env, diag_only):
    """Pinned host buffers on a stream context: block transfers overlapped with
    the sweeps, the call captured and replayed; every call (also after the host
    inputs changed in place) bitwise equal to the device factor path."""
    torch, qsi = env
    n, b, a = 4, 40, 12
    _, A, B = make_problem(n, b, a, seed=46)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    A_h = {k: pin(A[k]) for k in qsi.KEYS}
    B_h = {k: pin(B[k]) for k in qsi.KEYS}
    out = lambda: {k: (None if diag_only and k in ("upper", "lower") else torch.zeros_like(A_h[k]).pin_memory())
                   for k in qsi.KEYS}
    GR_h, GL_h = out(), out()
    for call in range(3):
        if call == 2:
            _, A2, _ = make_problem(n, b, a, seed=47)
            A_h["diag"].copy_(torch.from_numpy(A2["diag"]))
            B_h["arrow_r"].mul_(0.25)
        ctx.selquad_host(A_h, B_h, GR_h, GL_h, qsi.FP64_EMU)
        Rd, Xd = _ref(ctx, qsi, {k: A_h[k].cuda() for k in qsi.KEYS}, [{k: B_h[k].cuda() for k in qsi.KEYS}],
                      qsi.FP64_EMU)
        for key in qsi.KEYS:
            if GR_h[key] is None:
                continue
            assert np.array_equal(GR_h[key].numpy(), Rd[key].cpu().numpy()), (call, key)
            assert np.array_equal(GL_h[key].numpy(), Xd[0][key].cpu().numpy()), (call, key)
    ctx.close()
