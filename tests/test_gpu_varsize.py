"""GPU parity of the non-uniform-block solve (qsi_bta_solve_varsize; block i
of size b_i) against the oracle, and bitwise against the uniform solve when
all sizes are equal."""
import numpy as np
import pytest

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


def _dev(torch, flat):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in flat.items()}


def _problem(sizes, a, seed):
    h = inputs.hamiltonian_sizes(sizes, a, seed=inputs.BASE_SEED + 800 + seed)
    B = inputs.lesser_rhs_sizes(sizes, a, seed=inputs.BASE_SEED + 900 + seed)
    return rgf.assemble_a(h, 0.3, 1e-3, 0.5), B


def _host(qsi, flat, sizes, a):
    return inputs.unpack_sizes({k: (v.cpu().numpy() if v is not None else np.zeros(0, complex))
                                for k, v in flat.items()}, sizes, a)


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
@pytest.mark.parametrize("sizes,a", [([24, 40, 16, 33], 12), ([8, 64, 8], 0), ([50], 20), ([17, 31], 45),
                                     ([64, 48, 32, 16, 8, 4, 2, 1], 16), ([130, 70, 129, 5, 96], 24)])
def test_varsize_matches_oracle(env, prec_name, sizes, a):
    torch, qsi = env
    A, B = _problem(sizes, a, seed=len(sizes) + a)
    ctx = qsi.Context(0)
    GR, GX = ctx.solve_varsize(sizes, _dev(torch, inputs.pack_sizes(A)), [_dev(torch, inputs.pack_sizes(B))],
                               precision=getattr(qsi, prec_name))
    ctx.synchronize()
    oR, oL = rgf.selquad(A, B)
    keys = qsi.KEYS if len(sizes) > 1 else ("diag", "arrow_r", "arrow_b", "tip")
    assert max_block_rel_err(_host(qsi, GR, sizes, a), oR, keys) < TOL
    assert max_block_rel_err(_host(qsi, GX[0], sizes, a), oL, keys) < TOL
    ctx.close()


def test_varsize_equal_sizes_bitwise_uniform_and_diag_only(env, monkeypatch):
    """Equal sizes given as a list run the same products as the uniform solve:
    bitwise equal with the uniform solve's FP32 shadow off (QSI_NO_SHADOW; the
    non-uniform sweep has none, and the shadow changes only the Newton starts),
    within 1e-12 of it with the shadow on; diagonal-only outputs bitwise equal."""
    torch, qsi = env
    n, b, a = 5, 48, 20
    sizes = [b] * n
    A, B = _problem(sizes, a, seed=1)
    ctx = qsi.Context(0)
    Af, Bf = _dev(torch, inputs.pack_sizes(A)), _dev(torch, inputs.pack_sizes(B))
    GR, GX = ctx.solve_varsize(sizes, Af, [Bf], precision=qsi.FP64_EMU)
    stack = lambda m: {k: (np.stack(v) if isinstance(v, list) else v) for k, v in m.items()}
    Au, Bu = qsi.to_device(stack(A)), qsi.to_device(stack(B))
    SR, SX = ctx.solve(Au, [Bu], precision=qsi.FP64_EMU)  # with the shadow
    ctx.synchronize()
    monkeypatch.setenv("QSI_NO_SHADOW", "1")
    UR, UX = ctx.solve(Au, [Bu], qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)], precision=qsi.FP64_EMU)
    ctx.synchronize()
    monkeypatch.delenv("QSI_NO_SHADOW")
    for k in qsi.KEYS:
        assert np.array_equal(GR[k].cpu().numpy().ravel(), UR[k].cpu().numpy().ravel()), k
        assert np.array_equal(GX[0][k].cpu().numpy().ravel(), UX[0][k].cpu().numpy().ravel()), k
    assert max_block_rel_err(qsi.to_host(SX[0]), qsi.to_host(UX[0])) < 1e-12
    assert max_block_rel_err(qsi.to_host(SR), qsi.to_host(UR)) < 1e-12
    # diagonal-only outputs: the kept blocks bitwise equal
    DR, DX = qsi.flat_zeros(sizes, a, off_diagonal=False), [qsi.flat_zeros(sizes, a, off_diagonal=False)]
    ctx.solve_varsize(sizes, Af, [Bf], DR, DX, precision=qsi.FP64_EMU)
    ctx.synchronize()
    for k in ("diag", "arrow_r", "arrow_b", "tip"):
        assert np.array_equal(DR[k].cpu().numpy(), GR[k].cpu().numpy()), k
        assert np.array_equal(DX[0][k].cpu().numpy(), GX[0][k].cpu().numpy()), k
    ctx.close()


def test_varsize_si_only_and_argument_errors(env):
    torch, qsi = env
    sizes, a = [12, 20, 7], 5
    A, _ = _problem(sizes, a, seed=2)
    ctx = qsi.Context(0)
    GR, _ = ctx.solve_varsize(sizes, _dev(torch, inputs.pack_sizes(A)), [])
    ctx.synchronize()
    assert max_block_rel_err(_host(qsi, GR, sizes, a), rgf.selinv(A)) < TOL
    with pytest.raises(qsi.QsiError) as ei:
        ctx.solve_varsize([12, 0, 7], _dev(torch, inputs.pack_sizes(A)), [])
    assert ei.value.status == qsi.ERR_ARG
    ctx.close()
