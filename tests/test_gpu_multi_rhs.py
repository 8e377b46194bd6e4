"""Several right-hand sides in one sweep (qsi_bta_factor_multi /
qsi_bta_selquad_multi): G^R once and G_r = A^{-1} B_r A^{-H} for every B_r,
as RGF does for the lesser and greater Green's functions (Sec. I).  Every G_r
against the oracle and bitwise against a single-RHS solve; the linearity of SQ
in B pinned through the identity A^{-1}(A^H - A)A^{-H} = G^R - G^A."""
import numpy as np
import pytest

from conftest import make_problem
from oracle import rgf
from paper_2601_04904_gb300 import inputs
from paper_2601_04904_gb300.metrics import max_block_rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def qsi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04904_gb300 import qsi as q

    return q


def _rhs(n, b, a, k, seed):
    return [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 300 + seed * 10 + r) for r in range(k)]


def _host(qsi, m):
    return qsi.to_host(m)


@pytest.mark.parametrize("n,b,a,k", [(1, 3, 2, 2), (3, 5, 7, 3), (4, 33, 17, 2), (3, 64, 0, 4), (2, 70, 33, 3),
                                     (5, 8, 0, 1)])
def test_multi_rhs_matches_oracle(qsi, n, b, a, k):
    _, A, _ = make_problem(n, b, a, seed=31)
    Bs = _rhs(n, b, a, k, seed=n + b)
    ctx = qsi.Context(0)
    f = ctx.factor_multi(qsi.to_device(A), [qsi.to_device(B) for B in Bs])
    GR, GX = ctx.selquad_multi(f)
    ctx.synchronize()
    f.close()
    assert max_block_rel_err(_host(qsi, GR), rgf.selinv(A)) < TOL
    for r, B in enumerate(Bs):
        assert max_block_rel_err(_host(qsi, GX[r]), rgf.selquad(A, B)[1]) < TOL, r
    ctx.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
def test_multi_rhs_bitwise_equals_single_rhs(qsi, prec_name):
    prec = getattr(qsi, prec_name)
    n, b, a, k = 4, 48, 24, 3
    _, A, _ = make_problem(n, b, a, seed=32)
    Bs = _rhs(n, b, a, k, seed=2)
    ctx = qsi.Context(0)
    Ad = qsi.to_device(A)
    f = ctx.factor_multi(Ad, [qsi.to_device(B) for B in Bs], prec)
    GR, GX = ctx.selquad_multi(f)
    ctx.synchronize()
    f.close()
    for r, B in enumerate(Bs):
        f1 = ctx.factor(Ad, qsi.to_device(B), prec)
        R1, L1 = ctx.selquad(f1)
        ctx.synchronize()
        f1.close()
        for key in qsi.KEYS:
            assert np.array_equal(GX[r][key].cpu().numpy(), L1[key].cpu().numpy()), (r, key)
            assert np.array_equal(GR[key].cpu().numpy(), R1[key].cpu().numpy()), (r, key)
    ctx.close()


def _ah_minus_a(A):
    """A^H - A on the BTA pattern, block by block (exact)."""
    H = lambda x: np.conj(np.swapaxes(x, -1, -2))
    return {"diag": H(A["diag"]) - A["diag"], "upper": H(A["lower"]) - A["upper"],
            "lower": H(A["upper"]) - A["lower"], "arrow_r": H(A["arrow_b"]) - A["arrow_r"],
            "arrow_b": H(A["arrow_r"]) - A["arrow_b"], "tip": H(A["tip"]) - A["tip"]}


def test_greater_minus_lesser_is_retarded_minus_advanced(qsi):
    """With B_2 = B_1 + (A^H - A), G_2 - G_1 = A^{-1}(A^H - A)A^{-H} = G^R - G^A,
    i.e. blockwise G_2 - G_1 = X - X^H on the pattern (the relation between
    lesser, greater, retarded and advanced functions when the self-energies
    satisfy it)."""
    n, b, a = 4, 40, 16
    _, A, B1 = make_problem(n, b, a, seed=33)
    D = _ah_minus_a(A)
    B2 = {k: B1[k] + D[k] for k in qsi.KEYS}
    ctx = qsi.Context(0)
    f = ctx.factor_multi(qsi.to_device(A), [qsi.to_device(B1), qsi.to_device(B2)])
    GR, (G1, G2) = ctx.selquad_multi(f)
    ctx.synchronize()
    f.close()
    X, g1, g2 = _host(qsi, GR), _host(qsi, G1), _host(qsi, G2)
    H = lambda x: np.conj(np.swapaxes(x, -1, -2))
    spec = {"diag": X["diag"] - H(X["diag"]), "upper": X["upper"] - H(X["lower"]),
            "lower": X["lower"] - H(X["upper"]), "arrow_r": X["arrow_r"] - H(X["arrow_b"]),
            "arrow_b": X["arrow_b"] - H(X["arrow_r"]), "tip": X["tip"] - H(X["tip"])}
    diff = {k: g2[k] - g1[k] for k in qsi.KEYS}
    assert max_block_rel_err(diff, spec) < 1e-9
    ctx.close()


def test_multi_rhs_diagonal_only_and_selinv(qsi):
    n, b, a, k = 3, 24, 8, 2
    _, A, _ = make_problem(n, b, a, seed=34)
    Bs = _rhs(n, b, a, k, seed=4)
    ctx = qsi.Context(0)
    Ad = qsi.to_device(A)
    f = ctx.factor_multi(Ad, [qsi.to_device(B) for B in Bs])
    GRf, GXf = ctx.selquad_multi(f)
    GRd = qsi.device_zeros(n, b, a, off_diagonal=False)
    GXd = [qsi.device_zeros(n, b, a, off_diagonal=False) for _ in range(k)]
    ctx.selquad_multi(f, GRd, GXd)
    Rsi = ctx.selinv(f)  # SI alone from a factor with right-hand sides
    ctx.synchronize()
    f.close()
    for key in ("diag", "arrow_r", "arrow_b", "tip"):
        assert np.array_equal(GRd[key].cpu().numpy(), GRf[key].cpu().numpy()), key
        for r in range(k):
            assert np.array_equal(GXd[r][key].cpu().numpy(), GXf[r][key].cpu().numpy()), (r, key)
    for key in qsi.KEYS:
        assert np.array_equal(Rsi[key].cpu().numpy(), GRf[key].cpu().numpy()), key
    # a factor without right-hand sides: SI only
    f0 = ctx.factor_multi(Ad, [])
    R0 = ctx.selinv(f0)
    ctx.synchronize()
    with pytest.raises(qsi.QsiError) as ei:
        ctx.selquad_multi(f0, None, [])
    assert ei.value.status == qsi.ERR_STATE
    f0.close()
    assert max_block_rel_err(_host(qsi, R0), rgf.selinv(A)) < TOL
    ctx.close()


def test_multi_rhs_argument_errors(qsi):
    n, b, a = 2, 8, 4
    _, A, B = make_problem(n, b, a, seed=35)
    ctx = qsi.Context(0)
    Ad, Bd = qsi.to_device(A), qsi.to_device(B)
    with pytest.raises(qsi.QsiError) as ei:
        ctx.factor_multi(Ad, [Bd] * (qsi.MAX_RHS + 1))
    assert ei.value.status == qsi.ERR_ARG
    f = ctx.factor_multi(Ad, [Bd, Bd])
    with pytest.raises(qsi.QsiError) as ei:  # one output for two right-hand sides
        ctx.selquad_multi(f, None, [qsi.device_zeros(n, b, a)])
    assert ei.value.status == qsi.ERR_ARG
    with pytest.raises(qsi.QsiError) as ei:  # the single-RHS call on a two-RHS factor
        ctx.selquad(f)
    assert ei.value.status == qsi.ERR_STATE
    GR, (G1, G2) = ctx.selquad_multi(f)
    ctx.synchronize()
    f.close()
    for key in qsi.KEYS:  # the same right-hand side twice: the same bits
        assert np.array_equal(G1[key].cpu().numpy(), G2[key].cpu().numpy()), key
    ctx.close()
