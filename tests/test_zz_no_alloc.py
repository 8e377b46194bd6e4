"""The allocation-free block inversion, checked against the library's normal path.

qsi_block_inverse_noalloc exists for callers that cannot allocate device memory
while they run (their memory is reserved up front, or an allocation could stall
a time-critical loop).  It must give the same inverse as the regular path: here
the inverse of one b x b block computed by qsi_bta_factor + qsi_bta_selinv on a
single-block matrix (n_blocks = 1, a = 0, so G^R = A^{-1}).  Two calls in a row
(with different matrices) check that the shared scratch array is reset between
calls.  This file is collected last so that a failure here does not stop the
other GPU tests.
"""
import ctypes

import numpy as np
import pytest

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


def _reference_inverse(qsi, ctx, a):
    import torch

    A = {"diag": torch.from_numpy(a[None].copy()).cuda(), "upper": torch.zeros((0, a.shape[0], a.shape[0]),
         dtype=torch.complex128, device="cuda"), "lower": torch.zeros((0, a.shape[0], a.shape[0]),
         dtype=torch.complex128, device="cuda"), "arrow_r": torch.zeros((1, a.shape[0], 0), dtype=torch.complex128,
         device="cuda"), "arrow_b": torch.zeros((1, 0, a.shape[0]), dtype=torch.complex128, device="cuda"),
         "tip": torch.zeros((0, 0), dtype=torch.complex128, device="cuda")}
    f = ctx.factor(A)
    GR = ctx.selinv(f)
    ctx.synchronize()
    f.close()
    return GR["diag"][0].cpu().numpy()


@pytest.mark.parametrize("b", [40, 512])
def test_noalloc_inverse_matches_regular_path(b):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qsi, inv = _lib()
    ctx = qsi.Context(0)
    stream = torch.cuda.current_stream()
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    for call, seed in enumerate((11, 12)):
        a = _block(b, seed + b)
        A = torch.from_numpy(a).cuda()
        out = torch.empty_like(A)
        st = inv(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(out.data_ptr()), b,
                 ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(info.data_ptr()))
        assert st == qsi.OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        got = out.cpu().numpy()
        ref = _reference_inverse(qsi, ctx, a)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < TOL, f"call {call}: rel err {err:.3e}"
        # input untouched when output differs
        assert np.array_equal(A.cpu().numpy(), a)
    ctx.close()


def test_noalloc_rejects_oversize_and_bad_args():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qsi, inv = _lib()
    info = torch.zeros((1,), dtype=torch.int32, device="cuda")
    A = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    big = qsi.NOALLOC_MAX_B + 1
    assert inv(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()), big, None,
               ctypes.c_void_p(info.data_ptr())) == qsi.ERR_ARG
    assert inv(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()), 0, None,
               ctypes.c_void_p(info.data_ptr())) == qsi.ERR_ARG
    assert inv(None, ctypes.c_void_p(A.data_ptr()), 4, None, ctypes.c_void_p(info.data_ptr())) == qsi.ERR_ARG
