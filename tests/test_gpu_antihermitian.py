"""GPU tests of QSI_ASSUME_ANTIHERMITIAN_B (qsi_set_flags): with an
anti-Hermitian right-hand side (the recipe's B, like the lesser self-energy of
Sec. I) the sweeps mirror B-hat_{t,i+1}, Y21 and Y_{R,i} instead of forming
them.  Flagged results match the oracle at 1e-10; G^R is bitwise the
unflagged one; the mirrored blocks of G^< are exactly minus the conjugate
transpose of their partners; clearing the flag restores the unflagged bits,
and a cached graph is never replayed across a flag change."""
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


def _solve(qsi, ctx, A, Bs, prec, diag_only=False):
    f = ctx.factor_multi(qsi.to_device(A), [qsi.to_device(B) for B in Bs], prec)
    n, b, a = qsi.shape_of(A)
    GR = qsi.device_zeros(n, b, a, off_diagonal=not diag_only)
    GX = [qsi.device_zeros(n, b, a, off_diagonal=not diag_only) for _ in Bs]
    ctx.selquad_multi(f, GR, GX)
    ctx.synchronize()
    f.close()
    return qsi.to_host(GR), [qsi.to_host(G) for G in GX]


def _mirrored(G, n):
    for i in range(n - 1):
        assert np.array_equal(G["lower"][i], -np.conj(G["upper"][i].T)), i
    for i in range(n):
        assert np.array_equal(G["arrow_b"][i], -np.conj(G["arrow_r"][i].T)), i


@pytest.mark.parametrize("prec", ["fp64", "fp64_emu", "mixed"])
@pytest.mark.parametrize("n,b,a,nrhs", [(6, 32, 16, 1), (4, 70, 33, 2), (1, 40, 8, 1), (5, 48, 0, 1),
                                        (3, 200, 100, 1)])
def test_flagged_matches_oracle_and_unflagged(env, prec, n, b, a, nrhs):
    torch, qsi = env
    p = qsi.PRECISIONS[prec]
    tol = 1e-6 if prec == "mixed" else TOL
    _, A, B = make_problem(n, b, a, seed=n + b)
    Bs = [B] + [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 900 + r) for r in range(1, nrhs)]
    ctx = qsi.Context(0)
    R0, X0 = _solve(qsi, ctx, A, Bs, p)
    ctx.set_flags(qsi.ASSUME_ANTIHERMITIAN_B)
    R1, X1 = _solve(qsi, ctx, A, Bs, p)
    ctx.set_flags(0)
    R2, X2 = _solve(qsi, ctx, A, Bs, p)
    ctx.close()
    for k in qsi.KEYS:
        assert np.array_equal(R0[k], R1[k]), k          # G^R untouched by the flag
        assert np.array_equal(R0[k], R2[k]), k
        for r in range(nrhs):
            assert np.array_equal(X0[r][k], X2[r][k]), (r, k)  # flag cleared: the unflagged bits
    for r in range(nrhs):
        assert max_block_rel_err(X1[r], rgf.selquad(A, Bs[r])[1]) < tol, r
        _mirrored(X1[r], n)


def test_flagged_diagonal_only_outputs(env):
    torch, qsi = env
    n, b, a = 5, 40, 12
    _, A, B = make_problem(n, b, a, seed=7)
    ctx = qsi.Context(0)
    ctx.set_flags(qsi.ASSUME_ANTIHERMITIAN_B)
    Rf, Xf = _solve(qsi, ctx, A, [B], qsi.FP64_EMU)
    Rd, Xd = _solve(qsi, ctx, A, [B], qsi.FP64_EMU, diag_only=True)
    ctx.close()
    for k in ("diag", "arrow_r", "arrow_b", "tip"):
        assert np.array_equal(Xf[0][k], Xd[0][k]), k
    assert max_block_rel_err(Xf[0], rgf.selquad(A, B)[1]) < TOL


def test_flag_change_drops_cached_graph(env):
    """qsi_bta_solve on a stream context captures and replays; after
    qsi_set_flags the next call is solved and captured anew (its lower blocks
    are exact mirrors), and clearing the flag brings the unflagged bits back."""
    torch, qsi = env
    n, b, a = 6, 48, 16
    _, A, B = make_problem(n, b, a, seed=11)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    Ad, Bd = qsi.to_device(A), [qsi.to_device(B)]
    GR, GX = qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)]
    torch.cuda.synchronize()
    runs = []
    for flags in (0, 0, qsi.ASSUME_ANTIHERMITIAN_B, qsi.ASSUME_ANTIHERMITIAN_B, 0):
        ctx.set_flags(flags)
        ctx.solve(Ad, Bd, GR, GX, qsi.FP64_EMU)
        ctx.synchronize()
        runs.append(qsi.to_host(GX[0]))
    _mirrored(runs[2], n)
    _mirrored(runs[3], n)
    for k in qsi.KEYS:
        assert np.array_equal(runs[0][k], runs[1][k]) and np.array_equal(runs[0][k], runs[4][k]), k
        assert np.array_equal(runs[2][k], runs[3][k]), k
    assert not np.array_equal(runs[0]["lower"], runs[2]["lower"])  # really the mirrored path
    assert max_block_rel_err(runs[3], rgf.selquad(A, B)[1]) < TOL
    with pytest.raises(qsi.QsiError) as ei:
        ctx.set_flags(4)  # the first bit no flag uses
    assert ei.value.status == qsi.ERR_ARG
    ctx.close()


@pytest.mark.parametrize("prec", ["FP64", "FP64_EMU"])
def test_flagged_batched_matches_oracle(env, prec):
    torch, qsi = env
    n, b, a, nE = 4, 32, 16, 5
    h = inputs.hamiltonian(n, b, a, seed=inputs.BASE_SEED + 31)
    E, g = inputs.energy_grid(nE)
    Bs = [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 40 + k) for k in range(nE)]
    Bst = {k: np.stack([Bk[k] for Bk in Bs]) for k in qsi.KEYS}
    ctx = qsi.Context(0)
    ctx.set_flags(qsi.ASSUME_ANTIHERMITIAN_B)
    GR, GL = ctx.selquad_batched(qsi.to_device(h), E, 1e-3, g, qsi.to_device(Bst), precision=getattr(qsi, prec))
    ctx.synchronize()
    for k in range(nE):
        oR, oL = rgf.selquad(rgf.assemble_a(h, E[k], 1e-3, g[k]), Bs[k])
        got = {key: GL[key][k].cpu().numpy() for key in qsi.KEYS}
        assert max_block_rel_err(got, oL) < TOL, k
        _mirrored(got, n)
    ctx.close()
