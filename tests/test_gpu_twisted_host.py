"""QSI_TWISTED_SPLIT: qsi_bta_solve and the host entry through the twisted
two-way split (Sec. III-B with two partitions, the bottom half eliminated from
block n-1 up).  The fused solve under the flag equals qsi_bta_solve_partitioned
with two partitions bit for bit; the pinned host entry (partition blocks copied
straight into their slots as the forward sweep reaches them and back as the
backward sweep finishes them) equals the same device solve bit for bit, on
every replay of its captured graph, with and without B, with diagonal-only
outputs and with an interior padded by one identity block (n even).  Fewer
than three blocks leave the plain solve in place."""
import numpy as np
import pytest

from conftest import make_problem
from oracle import rgf
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


def _np(m):
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in m.items()}


def _device_twisted(qsi, A, Bs, prec, diag_only):
    """qsi_bta_solve_partitioned(partitions = 2) on device buffers, its own context."""
    n, b, a = rgf.shape_of(A)
    ctx = qsi.Context(0)
    GR = qsi.device_zeros(n, b, a, off_diagonal=not diag_only)
    GX = [qsi.device_zeros(n, b, a, off_diagonal=not diag_only) for _ in Bs]
    ctx.solve_partitioned(qsi.to_device(A), [qsi.to_device(B) for B in Bs], 2, GR, GX, prec)
    ctx.synchronize()
    ctx.close()
    return _np(GR), [_np(G) for G in GX]


def _assert_same(x, y, what):
    for k, v in y.items():
        if v is None:
            continue
        assert x[k] is not None, (what, k)
        assert np.array_equal(np.asarray(x[k]), v), (what, k)


@pytest.mark.parametrize("n,b,a", [(5, 40, 12), (6, 32, 8), (3, 24, 0)])
def test_flag_routes_solve_to_twisted_split(env, n, b, a):
    torch, qsi = env
    _, A, B = make_problem(n, b, a, seed=150 + n, eta=0.1)
    ref_R, ref_X = _device_twisted(qsi, A, [B], qsi.FP64_EMU, False)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    ctx.set_flags(qsi.TWISTED_SPLIT)
    Ad, Bd = qsi.to_device(A), qsi.to_device(B)
    GR = qsi.device_zeros(n, b, a)
    GX = [qsi.device_zeros(n, b, a)]
    for _ in range(3):  # direct run, then graph replays
        ctx.solve(Ad, [Bd], GR, GX, qsi.FP64_EMU)
        ctx.synchronize()
        _assert_same(_np(GR), ref_R, "GR")
        _assert_same(_np(GX[0]), ref_X[0], "GX")
    assert max_block_rel_err(_np(GX[0]), rgf.selquad(A, B)[1]) < TOL
    ctx.close()


def test_flag_below_three_blocks_is_plain(env):
    torch, qsi = env
    n, b, a = 2, 32, 8
    _, A, B = make_problem(n, b, a, seed=160, eta=0.1)
    stream = torch.cuda.Stream()
    outs = []
    for flags in (0, qsi.TWISTED_SPLIT):
        ctx = qsi.Context(0, stream=stream)
        ctx.set_flags(flags)
        GR, GX = ctx.solve(qsi.to_device(A), [qsi.to_device(B)], precision=qsi.FP64_EMU)
        ctx.synchronize()
        outs.append((_np(GR), _np(GX[0])))
        ctx.close()
    _assert_same(outs[1][0], outs[0][0], "GR")
    _assert_same(outs[1][1], outs[0][1], "GX")


@pytest.mark.parametrize("with_b", [True, False])
@pytest.mark.parametrize("diag_only", [False, True])
@pytest.mark.parametrize("n,b,a", [(7, 40, 12), (8, 32, 16)])
def test_host_entry_twisted_pinned(env, n, b, a, diag_only, with_b):
    torch, qsi = env
    _, A, B = make_problem(n, b, a, seed=170 + n, eta=0.1)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    ctx.set_flags(qsi.TWISTED_SPLIT)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    A_h = {k: pin(A[k]) for k in qsi.KEYS}
    B_h = {k: pin(B[k]) for k in qsi.KEYS} if with_b else None
    out = lambda: {k: (None if diag_only and k in ("upper", "lower") else torch.zeros_like(A_h[k]).pin_memory())
                   for k in qsi.KEYS}
    GR_h = out()
    GL_h = out() if with_b else None
    for call in range(3):  # direct run, capture, replays (the last after the inputs changed in place)
        if call == 2:
            _, A2, _ = make_problem(n, b, a, seed=190 + n, eta=0.1)
            A_h["diag"].copy_(torch.from_numpy(A2["diag"]))
            A["diag"] = A2["diag"]
            if with_b:
                B_h["arrow_r"].mul_(0.25)
                B["arrow_r"] = B["arrow_r"] * 0.25
        for G in [GR_h] + ([GL_h] if with_b else []):
            for v in G.values():
                if v is not None:
                    v.fill_(float("nan"))
        ctx.selquad_host(A_h, B_h, GR_h, GL_h, qsi.FP64_EMU)
        ref_R, ref_X = _device_twisted(qsi, A, [B] if with_b else [], qsi.FP64_EMU, diag_only)
        _assert_same(_np(GR_h), ref_R, ("GR", call))
        if with_b:
            _assert_same(_np(GL_h), ref_X[0], ("GL", call))
    ref = rgf.selquad(A, B)[1] if with_b else rgf.selinv(A)
    got = _np(GL_h) if with_b else _np(GR_h)
    keys = ("diag", "arrow_r", "arrow_b", "tip") if diag_only else ("diag", "upper", "lower", "arrow_r",
                                                                      "arrow_b", "tip")
    assert max_block_rel_err(got, ref, keys) < TOL
    ctx.close()


def test_twisted_with_antihermitian_flag(env):
    """Both flags: the twisted split's sweeps mirror the blocks an
    anti-Hermitian B implies (the reversed bottom half's B stays
    anti-Hermitian), fused solve and host entry alike."""
    torch, qsi = env
    n, b, a = 7, 40, 12
    _, A, B = make_problem(n, b, a, seed=200, eta=0.1)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    ctx.set_flags(qsi.TWISTED_SPLIT | qsi.ASSUME_ANTIHERMITIAN_B)
    GR, GX = ctx.solve(qsi.to_device(A), [qsi.to_device(B)], precision=qsi.FP64_EMU)
    ctx.synchronize()
    ref_R, ref_X = rgf.selinv(A), rgf.selquad(A, B)[1]
    assert max_block_rel_err(_np(GR), ref_R) < TOL
    assert max_block_rel_err(_np(GX[0]), ref_X) < TOL
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    A_h = {k: pin(A[k]) for k in qsi.KEYS}
    B_h = {k: pin(B[k]) for k in qsi.KEYS}
    GR_h = {k: torch.zeros_like(A_h[k]).pin_memory() for k in qsi.KEYS}
    GL_h = {k: torch.zeros_like(A_h[k]).pin_memory() for k in qsi.KEYS}
    for _ in range(2):
        ctx.selquad_host(A_h, B_h, GR_h, GL_h, qsi.FP64_EMU)
        _assert_same(_np(GR_h), _np(GR), "GR")
        _assert_same(_np(GL_h), _np(GX[0]), "GL")
    ctx.close()


def test_partitions_one_stays_plain_under_flag(env):
    """qsi_bta_solve_partitioned with partitions = 1 is the plain sweep even
    under QSI_TWISTED_SPLIT (the flag reroutes qsi_bta_solve only)."""
    torch, qsi = env
    n, b, a = 5, 32, 8
    _, A, B = make_problem(n, b, a, seed=210, eta=0.1)
    stream = torch.cuda.Stream()
    outs = []
    for flags, call in ((0, "solve"), (qsi.TWISTED_SPLIT, "p1")):
        ctx = qsi.Context(0, stream=stream)
        ctx.set_flags(flags)
        Ad, Bd = qsi.to_device(A), qsi.to_device(B)
        if call == "solve":
            GR, GX = ctx.solve(Ad, [Bd], precision=qsi.FP64_EMU)
        else:
            GR, GX = ctx.solve_partitioned(Ad, [Bd], 1, precision=qsi.FP64_EMU)
        ctx.synchronize()
        outs.append((_np(GR), _np(GX[0])))
        ctx.close()
    _assert_same(outs[1][0], outs[0][0], "GR")
    _assert_same(outs[1][1], outs[0][1], "GX")
