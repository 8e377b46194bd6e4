"""Handle lifetimes across the C-ABI: a factor that outlives its context.

qsi_destroy releases the memory of the context's live factors and detaches
them; a later qsi_factor_destroy frees only the handle, and a detached factor
given to another context is an argument error.  Several contexts created,
used and closed in turn in one process (each with live factors) must not
disturb one another."""
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


def test_factor_outlives_context(env):
    torch, qsi = env
    n, b, a = 5, 24, 8
    _, A, B = make_problem(n, b, a, seed=5, eta=0.1)
    Ad, Bd = qsi.to_device(A), qsi.to_device(B)
    kept = []
    for k, prec in enumerate((qsi.FP64, qsi.FP64_EMU, qsi.FP64, qsi.FP64_EMU)):
        stream = torch.cuda.Stream() if k % 2 else None
        ctx = qsi.Context(0, stream=stream)
        f = ctx.factor(Ad, Bd, prec)
        GR, GL = ctx.selquad(f)
        ctx.synchronize()
        assert max_block_rel_err(qsi.to_host(GL), rgf.selquad(A, B)[1]) < 1e-10
        kept.append(ctx.factor(Ad, Bd, prec))  # alive when its context closes
        ctx.close()
    other = qsi.Context(0)
    with pytest.raises(qsi.QsiError) as ei:
        other.selinv(kept[0])
    assert ei.value.status == qsi.ERR_ARG
    for f in kept:
        f.close()  # only the handle remains to free
    other.close()
