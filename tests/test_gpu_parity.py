"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerance: 1e-10 max per-block relative Frobenius error (FP64 mode), over every
pattern block of G^R and G^<.
"""
import numpy as np
import pytest

from conftest import make_problem
from oracle import rgf
from paper_2601_04904_gb300 import inputs
from paper_2601_04904_gb300.metrics import max_block_rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04904_gb300 import qsi

    c = qsi.Context(0)
    yield c
    c.close()


def _gpu_selquad(ctx, A, B):
    from paper_2601_04904_gb300 import qsi

    f = ctx.factor(qsi.to_device(A), qsi.to_device(B) if B is not None else None)
    if B is None:
        GR, GL = ctx.selinv(f), None
    else:
        GR, GL = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    return qsi.to_host(GR), (qsi.to_host(GL) if GL is not None else None)


# (n, b, a): degenerate, ragged (not multiples of the 32-wide tiles or the
# 16-wide inversion panels), small-kernel and blocked-kernel inversion sizes.
SHAPES = [(1, 1, 0), (1, 1, 1), (2, 1, 0), (4, 3, 2), (1, 4, 3), (3, 5, 7), (6, 8, 0), (8, 32, 16),
          (3, 64, 65), (3, 65, 0), (2, 70, 33), (5, 96, 40), (4, 128, 64), (2, 200, 1)]


@pytest.mark.parametrize("n,b,a", SHAPES)
def test_selquad_matches_oracle(ctx, n, b, a):
    _, A, B = make_problem(n, b, a)
    gr, gl = _gpu_selquad(ctx, A, B)
    oR, oL = rgf.selquad(A, B)
    assert max_block_rel_err(gr, oR) < TOL
    assert max_block_rel_err(gl, oL) < TOL


@pytest.mark.parametrize("n,b,a", [(1, 2, 0), (5, 33, 17), (3, 80, 0)])
def test_selinv_matches_oracle(ctx, n, b, a):
    _, A, _ = make_problem(n, b, a)
    gr, gl = _gpu_selquad(ctx, A, None)
    assert gl is None
    assert max_block_rel_err(gr, rgf.selinv(A)) < TOL


def test_unstructured_inputs(ctx):
    n, b, a = 4, 40, 24
    A = inputs.random_bta(n, b, a, seed=5)
    for i in range(n):
        A["diag"][i] += 6 * np.eye(b)
    A["tip"] += 6 * np.eye(a)
    B = inputs.random_bta(n, b, a, seed=6)
    gr, gl = _gpu_selquad(ctx, A, B)
    oR, oL = rgf.selquad(A, B)
    assert max_block_rel_err(gr, oR) < TOL
    assert max_block_rel_err(gl, oL) < TOL


@pytest.mark.parametrize("n,b,a", [(1, 3, 0), (5, 7, 3), (3, 40, 20)])
def test_assemble_is_exact(ctx, n, b, a):
    from paper_2601_04904_gb300 import qsi

    h = inputs.hamiltonian(n, b, a)
    got = qsi.to_host(ctx.assemble(qsi.to_device(h), 0.3, 1e-3, 0.5))
    ctx.synchronize()
    want = rgf.assemble_a(h, 0.3, 1e-3, 0.5)
    for k in qsi.KEYS:
        assert np.array_equal(got[k], want[k]), k


def test_host_end_to_end(ctx):
    from paper_2601_04904_gb300 import qsi

    n, b, a = 5, 48, 20
    _, A, B = make_problem(n, b, a, seed=2)
    GR = {k: np.zeros_like(v) for k, v in A.items()}
    GL = {k: np.zeros_like(v) for k, v in A.items()}
    ctx.selquad_host(A, B, GR, GL)
    oR, oL = rgf.selquad(A, B)
    assert max_block_rel_err(GR, oR) < TOL
    assert max_block_rel_err(GL, oL) < TOL
    # SI only from host buffers
    GR2 = {k: np.zeros_like(v) for k, v in A.items()}
    ctx.selquad_host(A, None, GR2, None)
    assert max_block_rel_err(GR2, oR) < TOL


def test_repeatable(ctx):
    """Same inputs, same launch order: bitwise identical results."""
    _, A, B = make_problem(3, 70, 30, seed=4)
    r1 = _gpu_selquad(ctx, A, B)
    r2 = _gpu_selquad(ctx, A, B)
    for k in r1[0]:
        assert np.array_equal(r1[0][k], r2[0][k])
        assert np.array_equal(r1[1][k], r2[1][k])


def test_singular_block_reported(ctx):
    """A zero diagonal block gives QSI_ERR_SINGULAR with the block index; the
    context stays usable."""
    from paper_2601_04904_gb300 import qsi

    for b in (8, 80):  # small-kernel and blocked-kernel inversion
        _, A, B = make_problem(3, b, 4)
        A["diag"][0] = 0.0
        f = ctx.factor(qsi.to_device(A), qsi.to_device(B))
        ctx.selquad(f)
        with pytest.raises(qsi.QsiError) as ei:
            ctx.synchronize()
        assert ei.value.status == qsi.ERR_SINGULAR
        assert "block 0" in str(ei.value)
        f.close()
    _, A, B = make_problem(2, 8, 4)
    gr, gl = _gpu_selquad(ctx, A, B)
    assert max_block_rel_err(gr, rgf.selquad(A, B)[0]) < TOL


def test_argument_errors(ctx):
    from paper_2601_04904_gb300 import qsi

    _, A, B = make_problem(2, 4, 2)
    Ad = qsi.to_device(A)
    f = ctx.factor(Ad)  # SI-only factor
    with pytest.raises(qsi.QsiError) as ei:
        ctx.selquad(f)
    assert ei.value.status == qsi.ERR_STATE
    f.close()
    with pytest.raises(qsi.QsiError) as ei:
        ctx.factor(Ad, precision=7)
    assert ei.value.status == qsi.ERR_UNSUPPORTED
    bad = dict(Ad)
    bad["diag"] = Ad["diag"][:0]  # n = 0
    with pytest.raises(qsi.QsiError) as ei:
        ctx.factor(bad)
    assert ei.value.status == qsi.ERR_ARG


def test_full_size_bench_workload(ctx):
    """The benchmark's workload (n_blocks=64, b=512, a=256) in the benchmark's
    launch configuration (factor + selquad on the context stream), every block
    of G^R and G^< against the full oracle."""
    from paper_2601_04904_gb300 import qsi

    n, b, a = 64, 512, 256
    h = inputs.hamiltonian(n, b, a)
    bl = inputs.lesser_rhs(n, b, a)
    Ad = ctx.assemble(qsi.to_device(h), 0.3, 1e-3, 0.5)
    f = ctx.factor(Ad, qsi.to_device(bl))
    GR, GL = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    gr, gl = qsi.to_host(GR), qsi.to_host(GL)
    del GR, GL, Ad
    oR, oL = rgf.selquad(rgf.assemble_a(h, 0.3, 1e-3, 0.5), bl)
    eR, eL = max_block_rel_err(gr, oR), max_block_rel_err(gl, oL)
    print(f"full-size max block rel err: G^R {eR:.3e}  G^< {eL:.3e}")
    assert eR < TOL
    assert eL < TOL
