"""Diagonal-only outputs: G^R / G^< containers whose upper and lower block
arrays are absent.  The sweep then keeps the off-diagonal blocks of the
backward recurrence (Alg. 1 / Alg. 2, Sec. III-A) in scratch; the diagonal,
arrow and tip blocks it writes must be bit-identical to those of a full-output
solve (same kernels, same order), and match the oracle."""
import numpy as np
import pytest

from conftest import make_problem
from oracle import rgf
from paper_2601_04904_gb300 import inputs

pytestmark = pytest.mark.gpu
KEPT = ("diag", "arrow_r", "arrow_b", "tip")
TOL = 1e-10


@pytest.fixture(scope="module")
def qsi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04904_gb300 import qsi as q

    return q


def _rel(x, y):
    d = np.linalg.norm((x - y).ravel())
    s = np.linalg.norm(y.ravel())
    return d / s if s > 0 else d


def _same_kept(qsi, full, part):
    assert part["upper"] is None and part["lower"] is None
    for k in KEPT:
        x, y = full[k], part[k]
        if hasattr(x, "cpu"):
            x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.array_equal(x, y), k


def _close_to_oracle(got, ora):
    n = got["diag"].shape[0]
    for i in range(n):
        assert _rel(got["diag"][i], ora["diag"][i]) < TOL, ("diag", i)
        if got["arrow_r"].size:
            assert _rel(got["arrow_r"][i], ora["arrow_r"][i]) < TOL, ("arrow_r", i)
            assert _rel(got["arrow_b"][i], ora["arrow_b"][i]) < TOL, ("arrow_b", i)
    if got["tip"].size:
        assert _rel(got["tip"], ora["tip"]) < TOL


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
@pytest.mark.parametrize("n,b,a", [(1, 3, 2), (2, 5, 0), (4, 33, 17), (3, 64, 0), (5, 48, 24)])
def test_selquad_diag_only_equals_full(qsi, prec_name, n, b, a):
    prec = getattr(qsi, prec_name)
    _, A, B = make_problem(n, b, a, seed=11)
    ctx = qsi.Context(0)
    Ad, Bd = qsi.to_device(A), qsi.to_device(B)
    f = ctx.factor(Ad, Bd, prec)
    R1, L1 = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    f = ctx.factor(Ad, Bd, prec)
    R2 = qsi.device_zeros(n, b, a, off_diagonal=False)
    L2 = qsi.device_zeros(n, b, a, off_diagonal=False)
    ctx.selquad(f, R2, L2)
    ctx.synchronize()
    f.close()
    _same_kept(qsi, R1, R2)
    _same_kept(qsi, L1, L2)
    if prec == qsi.FP64:
        oR, oL = rgf.selquad(A, B)
        _close_to_oracle(qsi.to_host(R2), oR)
        _close_to_oracle(qsi.to_host(L2), oL)
    ctx.close()


@pytest.mark.parametrize("n,b,a", [(1, 4, 3), (5, 33, 17), (3, 80, 0)])
def test_selinv_diag_only_equals_full(qsi, n, b, a):
    _, A, _ = make_problem(n, b, a, seed=12)
    ctx = qsi.Context(0)
    Ad = qsi.to_device(A)
    f = ctx.factor(Ad)
    R1 = ctx.selinv(f)
    ctx.synchronize()
    f.close()
    f = ctx.factor(Ad)
    R2 = ctx.selinv(f, qsi.device_zeros(n, b, a, off_diagonal=False))
    ctx.synchronize()
    f.close()
    _same_kept(qsi, R1, R2)
    _close_to_oracle(qsi.to_host(R2), rgf.selinv(A))
    ctx.close()


def test_host_entry_diag_only(qsi):
    n, b, a = 4, 40, 16
    _, A, B = make_problem(n, b, a, seed=13)

    def host_out(full):
        shapes = {"diag": (n, b, b), "upper": (n - 1, b, b), "lower": (n - 1, b, b),
                  "arrow_r": (n, b, a), "arrow_b": (n, a, b), "tip": (a, a)}
        return {k: (np.zeros(s, np.complex128) if (full or k in KEPT) else None) for k, s in shapes.items()}

    ctx = qsi.Context(0)
    R1, L1 = host_out(True), host_out(True)
    ctx.selquad_host(A, B, R1, L1)
    R2, L2 = host_out(False), host_out(False)
    ctx.selquad_host(A, B, R2, L2)
    _same_kept(qsi, R1, R2)
    _same_kept(qsi, L1, L2)
    oR, oL = rgf.selquad(A, B)
    _close_to_oracle(R2, oR)
    _close_to_oracle(L2, oL)
    ctx.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
def test_batched_diag_only_equals_full(qsi, prec_name):
    prec = getattr(qsi, prec_name)
    n, b, a, nE = 3, 48, 24, 4
    h = inputs.hamiltonian(n, b, a, seed=inputs.BASE_SEED + 21)
    E, g = inputs.energy_grid(nE, seed=inputs.BASE_SEED + 22)
    Bs = [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 200 + k) for k in range(nE)]
    Bst = {k: np.ascontiguousarray(np.stack([Bk[k] for Bk in Bs])) for k in qsi.KEYS}
    ctx = qsi.Context(0)
    Hd, Bd = qsi.to_device(h), qsi.to_device(Bst)
    R1, L1 = ctx.selquad_batched(Hd, E, 1e-3, g, Bd, precision=prec)
    ctx.synchronize()
    R2 = qsi.batched_zeros(nE, n, b, a, off_diagonal=False)
    L2 = qsi.batched_zeros(nE, n, b, a, off_diagonal=False)
    ctx.selquad_batched(Hd, E, 1e-3, g, Bd, R2, L2, precision=prec)
    ctx.synchronize()
    _same_kept(qsi, R1, R2)
    _same_kept(qsi, L1, L2)
    ctx.close()


def test_half_given_off_diagonal_is_an_argument_error(qsi):
    n, b, a = 3, 8, 4
    _, A, B = make_problem(n, b, a, seed=14)
    ctx = qsi.Context(0)
    f = ctx.factor(qsi.to_device(A), qsi.to_device(B))
    R = qsi.device_zeros(n, b, a)
    R["lower"] = None
    with pytest.raises(qsi.QsiError) as ei:
        ctx.selquad(f, R, qsi.device_zeros(n, b, a))
    assert ei.value.status == qsi.ERR_ARG
    f.close()
    ctx.close()
