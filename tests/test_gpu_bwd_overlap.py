"""GPU tests of the split backward sweep (the default; QSI_BWD_OVERLAP=0 at
context creation gives the joint phases):
the SI chain on the main stream, the SQ chain one step behind on the side
stream, U and P double-buffered by step parity.  The products and their
arithmetic are those of the joint phases, so every output must be bitwise
equal to the default path: FP64 and FP64_EMU, full and diagonal-only
outputs, one to three right-hand sides, a single block (a one-step backward
pass), the partitioned solve, direct calls and the graph-cached solve."""
import numpy as np
import pytest

from conftest import make_problem
from oracle import rgf
from paper_2601_04904_gb300.metrics import max_block_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04904_gb300 import qsi

    return torch, qsi


def _contexts(monkeypatch, qsi, torch, stream):
    monkeypatch.setenv("QSI_BWD_OVERLAP", "0")
    s0 = torch.cuda.Stream() if stream else None
    plain = qsi.Context(0, stream=s0)
    monkeypatch.delenv("QSI_BWD_OVERLAP")
    s1 = torch.cuda.Stream() if stream else None
    split = qsi.Context(0, stream=s1)
    return plain, split


def _rhs(n, b, a, nrhs, seed):
    from paper_2601_04904_gb300 import inputs

    return [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 100 + seed + r) for r in range(nrhs)]


def _host(qsi, m):
    return {k: v.cpu().numpy() for k, v in m.items()}


def _equal(qsi, X, Y):
    for k in qsi.KEYS:
        if X[k] is None or Y[k] is None:  # diagonal-only outputs have no upper / lower
            assert X[k] is None and Y[k] is None, k
            continue
        assert np.array_equal(X[k].cpu().numpy(), Y[k].cpu().numpy()), k


@pytest.mark.parametrize("prec", ["fp64", "fp64_emu"])
@pytest.mark.parametrize("n,b,a,nrhs,diag_only", [(5, 24, 8, 1, False), (4, 40, 0, 2, False), (6, 32, 16, 3, False),
                                                  (5, 24, 8, 1, True), (1, 30, 10, 1, False), (2, 20, 6, 2, True),
                                                  (1, 16, 0, 1, False)])
def test_split_backward_bitwise_direct_calls(env, monkeypatch, prec, n, b, a, nrhs, diag_only):
    torch, qsi = env
    p = qsi.PRECISIONS[prec]
    _, A, _ = make_problem(n, b, a, seed=n + b)
    Bs = _rhs(n, b, a, nrhs, n * b)
    plain, split = _contexts(monkeypatch, qsi, torch, stream=False)
    outs = []
    for c in (plain, split):
        f = c.factor_multi(qsi.to_device(A), [qsi.to_device(B) for B in Bs], p)
        GR = qsi.device_zeros(n, b, a, off_diagonal=not diag_only)
        GX = [qsi.device_zeros(n, b, a, off_diagonal=not diag_only) for _ in Bs]
        c.selquad_multi(f, GR, GX)
        c.synchronize()
        f.close()
        outs.append((GR, GX))
    _equal(qsi, outs[0][0], outs[1][0])
    for X, Y in zip(outs[0][1], outs[1][1]):
        _equal(qsi, X, Y)
    if not diag_only:
        oR, oL = rgf.selquad(A, Bs[0])
        assert max_block_rel_err(_host(qsi, outs[1][1][0]), oL) < 1e-10
    plain.close()
    split.close()


@pytest.mark.parametrize("prec", ["fp64", "fp64_emu"])
@pytest.mark.parametrize("n,b,a,nrhs", [(6, 32, 16, 1), (1, 24, 8, 2), (5, 40, 0, 3)])
def test_split_backward_bitwise_graph_cached_solve(env, monkeypatch, prec, n, b, a, nrhs):
    """qsi_bta_solve on stream contexts: the first call solves and captures,
    the next replay; split and plain contexts agree bit for bit on every call."""
    torch, qsi = env
    p = qsi.PRECISIONS[prec]
    _, A, _ = make_problem(n, b, a, seed=3 * n + b)
    Bs = _rhs(n, b, a, nrhs, 7 * n + b)
    plain, split = _contexts(monkeypatch, qsi, torch, stream=True)
    Ad, Bd = qsi.to_device(A), [qsi.to_device(B) for B in Bs]
    res = []
    for c in (plain, split):
        GR = qsi.device_zeros(n, b, a)
        GX = [qsi.device_zeros(n, b, a) for _ in Bs]
        torch.cuda.synchronize()
        for _ in range(3):
            c.solve(Ad, Bd, GR, GX, p)
            c.synchronize()
        res.append((GR, GX))
    _equal(qsi, res[0][0], res[1][0])
    for X, Y in zip(res[0][1], res[1][1]):
        _equal(qsi, X, Y)
    plain.close()
    split.close()


@pytest.mark.parametrize("prec", ["fp64", "fp64_emu"])
def test_split_backward_bitwise_partitioned(env, monkeypatch, prec):
    torch, qsi = env
    p = qsi.PRECISIONS[prec]
    n, b, a, P = 13, 24, 8, 3
    _, A, _ = make_problem(n, b, a, seed=41, eta=0.1)
    Bs = _rhs(n, b, a, 2, 41)
    plain, split = _contexts(monkeypatch, qsi, torch, stream=False)
    res = [c.solve_partitioned(qsi.to_device(A), [qsi.to_device(B) for B in Bs], P, precision=p)
           for c in (plain, split)]
    plain.synchronize()
    split.synchronize()
    _equal(qsi, res[0][0], res[1][0])
    for X, Y in zip(res[0][1], res[1][1]):
        _equal(qsi, X, Y)
    plain.close()
    split.close()
