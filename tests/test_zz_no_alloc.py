"""The allocation-free block inversion (qsi_block_inverse_noalloc).

This entry point exists for callers that cannot allocate device memory while
they run (their memory is reserved up front, or an allocation could stall a
time-critical loop).  Its inverse of one b x b block is checked against the
oracle (the selected inversion of a single-block matrix, n_blocks = 1 and
a = 0, where G^R = A^{-1}) and against the library's regular path.  The calls
share one scratch array whose status word must be reset on every call: a
block with a zero column reports info = 1 + that column, and the next call on
a regular block reports info = 0 with an accurate inverse.  Misaligned and
NULL pointers and oversized blocks are refused before anything is queued.
This file is collected last so that a failure here does not stop the other
GPU tests.
"""
import ctypes

import numpy as np
import pytest

from oracle import rgf

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _lib():
    from paper_2601_04904_gb300 import qsi

    f = qsi._lib.qsi_block_inverse_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    return qsi, f


def _block(b, seed):
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b))) / np.sqrt(b)
    return a + (0.3 + 1e-3j) * np.eye(b)


def _single_block(a):
    b = a.shape[0]
    z = np.zeros
    return {"diag": a[None].copy(), "upper": z((0, b, b), complex), "lower": z((0, b, b), complex),
            "arrow_r": z((1, b, 0), complex), "arrow_b": z((1, 0, b), complex), "tip": z((0, 0), complex)}


def _oracle_inverse(a):
    return rgf.selinv(_single_block(a))["diag"][0]


def _regular_inverse(qsi, ctx, a):
    f = ctx.factor(qsi.to_device(_single_block(a)))
    GR = ctx.selinv(f)
    ctx.synchronize()
    f.close()
    return GR["diag"][0].cpu().numpy()


def _call(inv, torch, a, info, out=None, offset=0):
    stream = torch.cuda.current_stream()
    A = torch.from_numpy(a).cuda()
    out = torch.empty_like(A) if out is None else out
    st = inv(ctypes.c_void_p(A.data_ptr() + offset), ctypes.c_void_p(out.data_ptr()), a.shape[0],
             ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(info.data_ptr()))
    torch.cuda.synchronize()
    return st, A, out


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qsi, inv = _lib()
    return torch, qsi, inv


@pytest.mark.parametrize("b", [40, 512])
def test_noalloc_inverse_matches_oracle_and_regular_path(env, b):
    """Two calls in a row on different blocks: each inverse within 1e-10 of the
    oracle and of the regular factor + selinv path; the input is untouched."""
    torch, qsi, inv = env
    ctx = qsi.Context(0)
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    for call, seed in enumerate((11, 12)):
        a = _block(b, seed + b)
        st, A, out = _call(inv, torch, a, info)
        assert st == qsi.OK, f"call {call}: status {st}"
        assert int(info.item()) == 0
        got = out.cpu().numpy()
        ref = _oracle_inverse(a)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL, call
        reg = _regular_inverse(qsi, ctx, a)
        assert np.linalg.norm(got - reg) / np.linalg.norm(reg) < TOL, call
        assert np.array_equal(A.cpu().numpy(), a)
    ctx.close()


@pytest.mark.parametrize("b,k", [(40, 0), (40, 17), (512, 3), (512, 300)])
def test_noalloc_singular_column_reported_then_status_reset(env, b, k):
    """A zero column k gives a zero pivot at step k (row operations keep the
    column zero): QSI_OK is returned and info = 1 + k (single-CTA kernel for
    b = 40, the cluster panel kernel for b = 512).  The next call, on a regular
    block, reports info = 0 and an accurate inverse: the shared status word
    was cleared."""
    torch, qsi, inv = env
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    a = _block(b, 5 + k)
    a[:, k] = 0.0
    st, _, _ = _call(inv, torch, a, info)
    assert st == qsi.OK
    assert int(info.item()) == k + 1
    good = _block(b, 6 + k)
    st, _, out = _call(inv, torch, good, info)
    assert st == qsi.OK
    assert int(info.item()) == 0
    ref = _oracle_inverse(good)
    assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) < TOL


def test_noalloc_in_place(env):
    torch, qsi, inv = env
    info = torch.zeros((1,), dtype=torch.int32, device="cuda")
    a = _block(96, 3)
    A = torch.from_numpy(a).cuda()
    st = inv(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()), 96,
             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.c_void_p(info.data_ptr()))
    torch.cuda.synchronize()
    assert st == qsi.OK and int(info.item()) == 0
    ref = _oracle_inverse(a)
    assert np.linalg.norm(A.cpu().numpy() - ref) / np.linalg.norm(ref) < TOL


def test_noalloc_rejects_oversize_misaligned_and_null(env):
    torch, qsi, inv = env
    info = torch.zeros((1,), dtype=torch.int32, device="cuda")
    A = torch.zeros((8, 8), dtype=torch.complex128, device="cuda")
    p = A.data_ptr()
    big = qsi.NOALLOC_MAX_B + 1
    assert inv(ctypes.c_void_p(p), ctypes.c_void_p(p), big, None, ctypes.c_void_p(info.data_ptr())) == qsi.ERR_ARG
    assert inv(ctypes.c_void_p(p), ctypes.c_void_p(p), 0, None, ctypes.c_void_p(info.data_ptr())) == qsi.ERR_ARG
    assert inv(None, ctypes.c_void_p(p), 4, None, ctypes.c_void_p(info.data_ptr())) == qsi.ERR_ARG
    assert inv(ctypes.c_void_p(p), ctypes.c_void_p(p), 4, None, None) == qsi.ERR_ARG
    # 8 bytes off a 16-byte boundary: refused before anything is queued
    assert inv(ctypes.c_void_p(p + 8), ctypes.c_void_p(p), 4, None, ctypes.c_void_p(info.data_ptr())) == qsi.ERR_ARG
    assert inv(ctypes.c_void_p(p), ctypes.c_void_p(p + 8), 4, None, ctypes.c_void_p(info.data_ptr())) == qsi.ERR_ARG
    torch.cuda.synchronize()
