"""GPU tests of the tensor-core precisions: the FP64 emulation (QSI_FP64_EMU),
its reduced-moduli form (QSI_MIXED) and the 3-term BF16 split (QSI_SPLIT3).

Single GEMMs are compared with numpy complex128 products (FP64_EMU at 1e-13,
MIXED elementwise within the bound of its CRT range); sweeps are compared with
the oracle per block at 1e-10 (FP64_EMU) and 1e-6 (MIXED).
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


def _c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _gemm(ctx, A, B, C, opA, opB, alpha, beta, prec):
    import torch
    from paper_2601_04904_gb300 import qsi

    dA, dB, dC = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (A, B, C))
    ctx.zgemm(dA, dB, dC, opA, opB, alpha, beta, precision=prec)
    ctx.synchronize()
    return dC.cpu().numpy()


def _ref(A, B, C, opA, opB, alpha, beta):
    oa = A if opA == 0 else np.conj(A.T)
    ob = B if opB == 0 else np.conj(B.T)
    return alpha * (oa @ ob) + beta * C


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (5, 7, 3), (128, 128, 64), (130, 257, 100), (300, 200, 1000),
                                   (64, 1000, 33), (512, 512, 512), (256, 384, 2000), (97, 33, 4100)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_emulated_gemm_matches_fp64(ctx, M, N, K, opA, opB):
    from paper_2601_04904_gb300 import qsi

    rng = np.random.default_rng(M * 1000 + N + K + 7 * opA + 13 * opB)
    A = _c(rng, *((M, K) if opA == 0 else (K, M)))
    B = _c(rng, *((K, N) if opB == 0 else (N, K)))
    C = _c(rng, M, N)
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0), (1.0, 0.5 - 0.25j)):
        got = _gemm(ctx, A, B, C, opA, opB, alpha, beta, qsi.FP64_EMU)
        ref = _ref(A, B, C, opA, opB, alpha, beta)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-13, (alpha, beta, err)


def test_emulated_gemm_exact_on_integers(ctx):
    """Gaussian-integer operands: the integer product is formed exactly; the
    only error left is the final FP64 scaling (a few units in the last place)."""
    from paper_2601_04904_gb300 import qsi

    rng = np.random.default_rng(3)
    M, N, K = 200, 150, 777
    A = (rng.integers(-1000, 1001, (M, K)) + 1j * rng.integers(-1000, 1001, (M, K))).astype(complex)
    B = (rng.integers(-1000, 1001, (K, N)) + 1j * rng.integers(-1000, 1001, (K, N))).astype(complex)
    got = _gemm(ctx, A, B, np.zeros((M, N), complex), 0, 0, 1.0, 0.0, qsi.FP64_EMU)
    ar, ai = A.real.astype(np.int64), A.imag.astype(np.int64)
    br, bi = B.real.astype(np.int64), B.imag.astype(np.int64)
    exact_re = (ar @ br - ai @ bi).astype(float)
    exact_im = (ar @ bi + ai @ br).astype(float)
    ulp4 = 4 * np.spacing(np.maximum(np.abs(exact_re), np.abs(exact_im)))
    assert np.all(np.abs(got.real - exact_re) <= ulp4)
    assert np.all(np.abs(got.imag - exact_im) <= ulp4)


def test_emulated_gemm_dynamic_range_and_zeros(ctx):
    """Rows and columns spanning 2^-60..2^60 and all-zero rows/columns: each
    element is accurate relative to its own row and column scales."""
    from paper_2601_04904_gb300 import qsi

    rng = np.random.default_rng(5)
    M, N, K = 160, 140, 300
    A = _c(rng, M, K) * np.exp2(rng.integers(-60, 61, M))[:, None]
    B = _c(rng, K, N) * np.exp2(rng.integers(-60, 61, N))[None, :]
    A[7] = 0
    B[:, 11] = 0
    got = _gemm(ctx, A, B, np.zeros((M, N), complex), 0, 0, 1.0, 0.0, qsi.FP64_EMU)
    ref = A @ B
    scale = np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :] * np.sqrt(K)
    ok = scale > 0
    assert np.all(np.abs(got - ref)[ok] <= 1e-13 * scale[ok])
    assert np.all(got[7] == 0) and np.all(got[:, 11] == 0)


@pytest.mark.parametrize("n,b,a", [(1, 1, 0), (4, 3, 2), (8, 32, 16), (3, 65, 0), (2, 70, 33), (4, 128, 64),
                                   (3, 200, 100)])
def test_selquad_emulated_matches_oracle(ctx, n, b, a):
    from paper_2601_04904_gb300 import qsi

    _, A, B = make_problem(n, b, a)
    f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.FP64_EMU)
    GR, GL = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    oR, oL = rgf.selquad(A, B)
    assert max_block_rel_err(qsi.to_host(GR), oR) < TOL
    assert max_block_rel_err(qsi.to_host(GL), oL) < TOL


def test_full_size_emulated(ctx):
    """The benchmark workload (n_blocks=64, b=512, a=256) in the emulated mode,
    every block of G^R and G^< against the full oracle, without and with the
    anti-Hermitian mirroring of QSI_ASSUME_ANTIHERMITIAN_B."""
    from paper_2601_04904_gb300 import qsi

    n, b, a = 64, 512, 256
    h = inputs.hamiltonian(n, b, a)
    bl = inputs.lesser_rhs(n, b, a)
    Ad = ctx.assemble(qsi.to_device(h), 0.3, 1e-3, 0.5)
    Bd = qsi.to_device(bl)
    res = []
    # unflagged, then with QSI_ASSUME_ANTIHERMITIAN_B (the recipe's B is anti-Hermitian)
    for flags in (0, qsi.ASSUME_ANTIHERMITIAN_B):
        ctx.set_flags(flags)
        f = ctx.factor(Ad, Bd, precision=qsi.FP64_EMU)
        GR, GL = ctx.selquad(f)
        ctx.synchronize()
        f.close()
        res.append((qsi.to_host(GR), qsi.to_host(GL)))
        del GR, GL
    ctx.set_flags(0)
    del Ad, Bd
    oR, oL = rgf.selquad(rgf.assemble_a(h, 0.3, 1e-3, 0.5), bl)
    for name, (gr, gl) in zip(("unflagged", "anti-Hermitian B"), res):
        eR, eL = max_block_rel_err(gr, oR), max_block_rel_err(gl, oL)
        print(f"full-size emulated ({name}) max block rel err: G^R {eR:.3e}  G^< {eL:.3e}")
        assert eR < TOL
        assert eL < TOL


# QSI_MIXED: the modular-integer emulation with a prefix of the 17 moduli of
# the FP64 scheme (13 by default).  With nm moduli, M = p_0 ... p_{nm-1} and the
# operands are scaled integers of t = floor((log2 M - 2 - log2(2 K)) / 2) bits
# relative to the exponent bound 2^e of their row (A) / column (B), so each
# real component is off by at most 2^(e - t - 1) <= 2^-t max|row| and the
# product element (m, n) by at most
#   2^-t (max_m ||op(B)[:, n]||_1 + max_n ||op(A)[m, :]||_1)   (+ second order),
# with ||z||_1 summing |Re| + |Im|.  This is the bound the scheme guarantees.
MODULI = (256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193, 191)
MIX_TOL = 1e-6  # per-block relative Frobenius error of QSI_MIXED sweeps


def _tbits(nm, K):
    log2m = sum(np.log2(p) for p in MODULI[:nm])
    return min(62, int(np.floor((log2m - 2.0 - np.log2(2.0 * max(1, K))) / 2.0)))


def _moduli_bound(oa, ob, t):
    amax = np.maximum(np.abs(oa.real), np.abs(oa.imag)).max(axis=1)
    bmax = np.maximum(np.abs(ob.real), np.abs(ob.imag)).max(axis=0)
    a1 = (np.abs(oa.real) + np.abs(oa.imag)).sum(axis=1)
    b1 = (np.abs(ob.real) + np.abs(ob.imag)).sum(axis=0)
    K = oa.shape[1]
    first = 2.0 ** -t * (amax[:, None] * b1[None, :] + a1[:, None] * bmax[None, :])
    second = K * 2.0 ** (2 - 2 * t) * amax[:, None] * bmax[None, :]
    return 1.01 * (first + second)


def _mixed_ctx(monkeypatch, nm):
    from paper_2601_04904_gb300 import qsi

    if nm is not None:
        monkeypatch.setenv("QSI_MIXED_MODULI", str(nm))
    return qsi.Context(0)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (130, 257, 100), (512, 512, 512), (97, 33, 2100), (64, 300, 1536)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 1), (0, 1)])
def test_mixed_gemm_within_moduli_bound(ctx, M, N, K, opA, opB):
    """QSI_MIXED (13 moduli): every element within the bound the reduced CRT
    range guarantees; the error is really that of the reduced scheme (well
    above FP64 rounding for K > 1)."""
    from paper_2601_04904_gb300 import qsi

    rng = np.random.default_rng(M + 3 * N + 5 * K + opA + 2 * opB)
    A = _c(rng, *((M, K) if opA == 0 else (K, M)))
    B = _c(rng, *((K, N) if opB == 0 else (N, K)))
    C = _c(rng, M, N)
    oa = A if opA == 0 else np.conj(A.T)
    ob = B if opB == 0 else np.conj(B.T)
    t = _tbits(13, K)
    bound = _moduli_bound(oa, ob, t)
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0)):
        got = _gemm(ctx, A, B, C, opA, opB, alpha, beta, qsi.MIXED)
        ref = _ref(A, B, C, opA, opB, alpha, beta)
        fl = 4 * np.spacing(np.abs(ref))  # final FP64 rounding of beta C + product
        d = got - ref
        assert np.all(np.abs(d.real) <= bound + fl.real), (alpha, beta, np.max(np.abs(d.real) / bound))
        assert np.all(np.abs(d.imag) <= bound + fl.real), (alpha, beta, np.max(np.abs(d.imag) / bound))
        if K > 64:
            assert np.linalg.norm(d) / np.linalg.norm(ref) > 1e-15  # the reduced scheme, not FP64


@pytest.mark.parametrize("nm", [9, 10, 12, 14, 16])
def test_mixed_gemm_moduli_count(monkeypatch, nm):
    """QSI_MIXED_MODULI picks another prefix of the moduli (run-time moduli
    count in the conversion and reconstruction kernels): the bound of that
    count holds, and fewer moduli give a larger error."""
    from paper_2601_04904_gb300 import qsi

    rng = np.random.default_rng(nm)
    M, N, K = 200, 190, 700
    A, B, C = _c(rng, M, K), _c(rng, K, N), np.zeros((M, N), complex)
    errs = []
    for count in (nm, None):
        c = _mixed_ctx(monkeypatch, count)
        got = _gemm(c, A, B, C, 0, 0, 1.0, 0.0, qsi.MIXED)
        c.close()
        monkeypatch.delenv("QSI_MIXED_MODULI", raising=False)
        ref = A @ B
        d = got - ref
        bound = _moduli_bound(A, B, _tbits(nm if count else 13, K)) + 4 * np.spacing(np.abs(ref))
        assert np.all(np.abs(d.real) <= bound) and np.all(np.abs(d.imag) <= bound)
        errs.append(np.linalg.norm(d) / np.linalg.norm(ref))
    if nm < 13:
        assert errs[0] > errs[1]
    elif nm > 13:
        assert errs[0] < errs[1]


@pytest.mark.parametrize("n,b,a", [(1, 1, 0), (4, 3, 2), (8, 32, 16), (3, 70, 33), (6, 128, 64), (3, 200, 100)])
def test_selquad_mixed_matches_oracle(ctx, n, b, a):
    """Mixed-mode sweeps: every block of G^R and G^< within 1e-6 (relative
    Frobenius) of the oracle."""
    from paper_2601_04904_gb300 import qsi

    _, A, B = make_problem(n, b, a)
    f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.MIXED)
    GR, GL = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    oR, oL = rgf.selquad(A, B)
    eR, eL = max_block_rel_err(qsi.to_host(GR), oR), max_block_rel_err(qsi.to_host(GL), oL)
    print(f"mixed ({n},{b},{a}): G^R {eR:.2e} G^< {eL:.2e}")
    assert eR < MIX_TOL and eL < MIX_TOL


def test_selquad_mixed_large_blocks_matches_oracle(ctx):
    """The block and arrow sizes of the precision workload (b = 1024, a = 512;
    8 of its 128 blocks) in QSI_MIXED: every block within 1e-6 of the oracle."""
    from paper_2601_04904_gb300 import qsi

    n, b, a = 8, 1024, 512
    h = inputs.hamiltonian(n, b, a)
    bl = inputs.lesser_rhs(n, b, a)
    Ad = ctx.assemble(qsi.to_device(h), 0.3, 1e-3, 0.5)
    f = ctx.factor(Ad, qsi.to_device(bl), precision=qsi.MIXED)
    GR, GL = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    gr, gl = qsi.to_host(GR), qsi.to_host(GL)
    del GR, GL, Ad
    oR, oL = rgf.selquad(rgf.assemble_a(h, 0.3, 1e-3, 0.5), bl)
    eR, eL = max_block_rel_err(gr, oR), max_block_rel_err(gl, oL)
    print(f"mixed (8,1024,512): G^R {eR:.3e}  G^< {eL:.3e}")
    assert eR < MIX_TOL and eL < MIX_TOL
    assert max(eR, eL) > 1e-13  # the reduced products, not FP64


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (130, 257, 100), (512, 512, 512), (97, 33, 2100)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 1), (0, 1)])
def test_split3_gemm_is_fp32_accurate(ctx, M, N, K, opA, opB):
    """QSI_SPLIT3: 3-term BF16 split, FP32 accumulation in the tensor cores.
    The accumulation truncates, so the error grows about linearly with K
    (measured 5.7e-6 at K=512, 2.3e-5 at K=2100): bound 2e-8 * K.  This is why
    QSI_MIXED uses the reduced modular scheme instead."""
    from paper_2601_04904_gb300 import qsi

    rng = np.random.default_rng(M + 3 * N + 5 * K + opA + 2 * opB)
    A = _c(rng, *((M, K) if opA == 0 else (K, M)))
    B = _c(rng, *((K, N) if opB == 0 else (N, K)))
    C = _c(rng, M, N)
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0)):
        got = _gemm(ctx, A, B, C, opA, opB, alpha, beta, qsi.SPLIT3)
        ref = _ref(A, B, C, opA, opB, alpha, beta)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < max(2e-6, 2e-8 * K), (alpha, beta, err)
        assert err > 1e-12  # really the split path, not FP64


@pytest.mark.parametrize("n,b,a", [(4, 3, 2), (8, 32, 16), (3, 70, 33), (6, 128, 64)])
def test_selquad_split3_error_reported(ctx, n, b, a):
    """QSI_SPLIT3 sweeps: complex-FP32-level products; the per-block error
    against the oracle stays below 1e-3 on these shapes (it misses 1e-6)."""
    from paper_2601_04904_gb300 import qsi

    _, A, B = make_problem(n, b, a)
    f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.SPLIT3)
    GR, GL = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    oR, oL = rgf.selquad(A, B)
    eR, eL = max_block_rel_err(qsi.to_host(GR), oR), max_block_rel_err(qsi.to_host(GL), oL)
    print(f"split3 ({n},{b},{a}): G^R {eR:.2e} G^< {eL:.2e}")
    assert eR < 1e-3 and eL < 1e-3


@pytest.mark.parametrize("prec", ["fp64_emu", "mixed", "split3"])
def test_copy_problem_without_terms(ctx, prec):
    """K = 0: the product is empty and C <- beta * C exactly, in every mode."""
    from paper_2601_04904_gb300 import qsi

    rng = np.random.default_rng(1)
    C = _c(rng, 40, 30)
    A = np.zeros((40, 0), complex)
    B = np.zeros((0, 30), complex)
    got = _gemm(ctx, A, B, C, 0, 0, 1.0, 0.5 + 0.5j, qsi.PRECISIONS[prec])
    assert np.allclose(got, (0.5 + 0.5j) * C, rtol=0, atol=1e-15)


@pytest.mark.parametrize("prec", ["fp64_emu", "mixed", "split3"])
def test_refined_inversion_singular_block_reported(ctx, prec):
    """Tensor-core precisions invert with FP32 Gauss-Jordan + Newton: a zero
    first diagonal block (S_0 = A_00) still gives QSI_ERR_SINGULAR with its
    index, for one FP32 panel (b = 8) and several (b = 80)."""
    from paper_2601_04904_gb300 import qsi

    for b in (8, 80):
        _, A, B = make_problem(3, b, 4)
        A["diag"][0] = 0.0
        f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.PRECISIONS[prec])
        ctx.selquad(f)
        with pytest.raises(qsi.QsiError) as ei:
            ctx.synchronize()
        f.close()
        assert ei.value.status == qsi.ERR_SINGULAR
        assert "block 0" in str(ei.value)
    # the context stays usable
    _, A, B = make_problem(2, 8, 4)
    f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.PRECISIONS[prec])
    GR, GL = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    tol = {"fp64_emu": TOL, "mixed": MIX_TOL, "split3": 1e-3}[prec]
    assert max_block_rel_err(qsi.to_host(GR), rgf.selquad(A, B)[0]) < tol


def test_refined_inversion_ill_conditioned_block_reported(ctx):
    """A first block with condition number 1e12 is beyond the FP32 start of the
    Newton refinement: QSI_ERR_ACCURACY for block 0, not a silently wrong
    result; QSI_FP64 solves the same problem."""
    from paper_2601_04904_gb300 import qsi

    b = 48
    _, A, B = make_problem(2, b, 8, seed=3)
    rng = np.random.default_rng(9)
    U, _ = np.linalg.qr(rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b)))
    V, _ = np.linalg.qr(rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b)))
    A["diag"][0] = (U * np.logspace(0, -12, b)) @ V.conj().T
    f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.FP64_EMU)
    ctx.selquad(f)
    with pytest.raises(qsi.QsiError) as ei:
        ctx.synchronize()
    f.close()
    assert ei.value.status == qsi.ERR_ACCURACY
    assert "block 0" in str(ei.value)
    f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.FP64)
    ctx.selquad(f)
    ctx.synchronize()
    f.close()


@pytest.mark.parametrize("b,nb,rt", [(1, None, None), (31, None, None), (33, None, None), (257, None, None),
                                     (300, None, None), (513, None, None), (600, None, None), (1024, None, None),
                                     (100, 8, None), (100, 16, 1), (100, 32, 2), (400, 32, 2), (300, 16, 2),
                                     (300, 8, None), (700, 8, None)])
def test_refined_inversion_panel_layouts(ctx, monkeypatch, b, nb, rt):
    """Every layout of the blocked FP32 panel kernels against the oracle (the
    launch-per-panel form, which blocks above 512 take; QSI_GJ_PANELS selects
    it below): 32 columns with one row per thread (b <= 512), 16 with two (up
    to the largest block, 1024), forced widths and rows per thread
    (QSI_PANEL32_NB / _RT), ragged last panels and partial last warps."""
    from paper_2601_04904_gb300 import qsi

    monkeypatch.setenv("QSI_GJ_PANELS", "1")
    if nb is not None:
        monkeypatch.setenv("QSI_PANEL32_NB", str(nb))
    if rt is not None:
        monkeypatch.setenv("QSI_PANEL32_RT", str(rt))
    _, A, B = make_problem(2, b, 5, seed=17)
    f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.FP64_EMU)
    GR, GL = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    oR, oL = rgf.selquad(A, B)
    assert max_block_rel_err(qsi.to_host(GR), oR) < TOL
    assert max_block_rel_err(qsi.to_host(GL), oL) < TOL


@pytest.mark.parametrize("b", [1, 2, 31, 32, 33, 100, 255, 256, 257, 300, 480, 511, 512])
def test_cluster_gauss_jordan_matches_oracle_and_blocked_form(ctx, monkeypatch, b):
    """The one-launch cluster form of the FP32 Gauss-Jordan (ceil(b / 32) CTAs,
    the matrix resident in their shared memory) as the start of the Newton
    refinement: within 1e-10 of the oracle, and of the blocked launch-per-panel
    form; ragged last slabs, single-CTA clusters and the 16-CTA maximum."""
    from paper_2601_04904_gb300 import qsi

    _, A, B = make_problem(2, b, 5, seed=19)
    oR, oL = rgf.selquad(A, B)
    res = []
    for env in (None, "1"):
        if env:
            monkeypatch.setenv("QSI_GJ_PANELS", "1")
        f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.FP64_EMU)
        GR, GL = ctx.selquad(f)
        ctx.synchronize()
        f.close()
        res.append((qsi.to_host(GR), qsi.to_host(GL)))
    monkeypatch.delenv("QSI_GJ_PANELS")
    for GR, GL in res:
        assert max_block_rel_err(GR, oR) < TOL
        assert max_block_rel_err(GL, oL) < TOL
    assert max_block_rel_err(res[0][1], res[1][1]) < TOL


def test_cluster_gauss_jordan_batched_points(ctx):
    """Batched points run one cluster each (grid y): every point against the oracle."""
    from paper_2601_04904_gb300 import qsi

    n, b, a, nE = 3, 160, 40, 6
    h = inputs.hamiltonian(n, b, a, seed=inputs.BASE_SEED + 55)
    E, g = inputs.energy_grid(nE)
    Bs = [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 60 + k) for k in range(nE)]
    Bst = {k: np.stack([Bk[k] for Bk in Bs]) for k in qsi.KEYS}
    GR, GL = ctx.selquad_batched(qsi.to_device(h), E, 1e-3, g, qsi.to_device(Bst), precision=qsi.FP64_EMU)
    ctx.synchronize()
    for k in range(nE):
        oR, oL = rgf.selquad(rgf.assemble_a(h, E[k], 1e-3, g[k]), Bs[k])
        assert max_block_rel_err({key: GL[key][k].cpu().numpy() for key in qsi.KEYS}, oL) < TOL, k


def test_refined_inversion_matches_fp64_gauss_jordan(ctx, monkeypatch):
    """QSI_FP64_EMU with the refined inversion against the same mode with FP64
    Gauss-Jordan (QSI_NO_REFINED_INV): both within 1e-10 of the oracle and of
    each other; b = 200 spans several 32-column FP32 panels with a ragged one."""
    from paper_2601_04904_gb300 import qsi

    _, A, B = make_problem(3, 200, 72, seed=5)
    oR, oL = rgf.selquad(A, B)
    res = []
    for env in (None, "1"):
        if env:
            monkeypatch.setenv("QSI_NO_REFINED_INV", "1")
        c = qsi.Context(0)
        f = c.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.FP64_EMU)
        GR, GL = c.selquad(f)
        c.synchronize()
        f.close()
        res.append((qsi.to_host(GR), qsi.to_host(GL)))
        c.close()
    for GR, GL in res:
        assert max_block_rel_err(GR, oR) < TOL
        assert max_block_rel_err(GL, oL) < TOL
    assert max_block_rel_err(res[0][0], res[1][0]) < TOL


def test_bounded_wait_timeout_reported_and_context_usable(ctx):
    """The error model of the tensor-core kernels' bounded waits: a wait that
    runs out (here an mbarrier nothing arrives at, 2 ms limit) is reported by
    the next synchronize as QSI_ERR_TIMEOUT, the status word is cleared, and
    the context solves the next problem normally."""
    from paper_2601_04904_gb300 import qsi

    ctx.selftest_wait_timeout(2000)
    with pytest.raises(qsi.QsiError) as ei:
        ctx.synchronize()
    assert ei.value.status == qsi.ERR_TIMEOUT
    assert "bounded wait" in str(ei.value)
    ctx.synchronize()  # cleared
    with pytest.raises(qsi.QsiError) as ei:
        ctx.selftest_wait_timeout(0)
    assert ei.value.status == qsi.ERR_ARG
    _, A, B = make_problem(3, 40, 8)
    f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=qsi.FP64_EMU)
    GR, GL = ctx.selquad(f)
    ctx.synchronize()
    f.close()
    oR, oL = rgf.selquad(A, B)
    assert max_block_rel_err(qsi.to_host(GL), oL) < TOL


@pytest.mark.parametrize("prec", ["fp64_emu", "mixed"])
@pytest.mark.parametrize("n,b,a", [(2, 40, 8), (6, 100, 30), (9, 64, 0), (3, 600, 40)])
def test_shadow_sweep_starts(ctx, monkeypatch, prec, n, b, a):
    """The forward sweep's FP32 shadow (a third stream forming every block's
    Schur complement from FP32 starts and inverting it one step ahead; the
    main chain only refines): within 1e-12 of the same solve with the shadow
    off (QSI_NO_SHADOW: each block's own FP32 Gauss-Jordan start), and of the
    oracle at the precision's tolerance; cluster (b <= 512) and blocked
    (b = 600) Gauss-Jordan."""
    from paper_2601_04904_gb300 import qsi

    p = qsi.PRECISIONS[prec]
    tol = TOL if prec == "fp64_emu" else MIX_TOL
    _, A, B = make_problem(n, b, a, seed=7 + n)
    res = []
    for off in (False, True):
        if off:
            monkeypatch.setenv("QSI_NO_SHADOW", "1")
        f = ctx.factor(qsi.to_device(A), qsi.to_device(B), precision=p)
        GR, GL = ctx.selquad(f)
        ctx.synchronize()
        f.close()
        res.append((qsi.to_host(GR), qsi.to_host(GL)))
    oR, oL = rgf.selquad(A, B)
    for GR, GL in res:
        assert max_block_rel_err(GR, oR) < tol
        assert max_block_rel_err(GL, oL) < tol
    # the two starts refine to the same inverses up to the products' rounding
    # (FP64-level in FP64_EMU; 13-moduli products in mixed mode)
    close = 1e-12 if prec == "fp64_emu" else 1e-7
    assert max_block_rel_err(res[0][0], res[1][0]) < close
    assert max_block_rel_err(res[0][1], res[1][1]) < close
