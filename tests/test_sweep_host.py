"""The library's sweep schedule (csrc/sweep.cu) built for the host, without a GPU.

tests/host_sweep/sweep_host.cpp compiles sweep.cu with no-op stream/event calls,
host allocations, and plain host loops in place of its two device primitives:
the grouped complex GEMM and the block inversion.  The result tests the
sweep's own logic against the oracle: every block it reads and writes, its
sizes, leading dimensions, offsets and operand transpositions.  Non-uniform
blocks (per-step b_i, b_{i+1}) and the uniform case (the same calls whether the
sizes arrive as a list or as one b) are both covered."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import rgf
from paper_2601_04904_gb300 import inputs
from paper_2601_04904_gb300.metrics import max_block_rel_err

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = inputs.KEYS
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = tmp_path_factory.mktemp("sweep_host") / "sweep_host.so"
    src = os.path.join(ROOT, "tests", "host_sweep", "sweep_host.cpp")
    subprocess.run([gxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-x", "c++", src, "-I", CUDA_INC, "-o", str(out)],
                   check=True)
    so = ctypes.CDLL(str(out))
    so.host_solve.restype = ctypes.c_int
    return so


def _ptrs(flat):
    arr = (ctypes.c_void_p * 6)()
    for k, key in enumerate(KEYS):
        arr[k] = flat[key].ctypes.data if flat[key].size else None
    return arr


def _solve(lib, sizes, a, A, B, uniform=False):
    fa, fb = inputs.pack_sizes(A), inputs.pack_sizes(B)
    fr = {k: np.zeros_like(v) for k, v in fa.items()}
    fl = {k: np.zeros_like(v) for k, v in fa.items()}
    bs = (ctypes.c_int * len(sizes))(*sizes)
    rc = lib.host_solve(len(sizes), bs, a, int(uniform), _ptrs(fa), _ptrs(fb), _ptrs(fr), _ptrs(fl))
    assert rc == 0
    return inputs.unpack_sizes(fr, sizes, a), inputs.unpack_sizes(fl, sizes, a)


@pytest.mark.parametrize("sizes,a", [([3, 5, 2, 4], 3), ([1, 4, 1], 0), ([6], 2), ([2, 3], 5),
                                     ([7, 3, 5, 2, 8, 4], 4), ([1, 1, 9, 1], 2), ([5, 4, 3, 2, 1], 0)])
def test_nonuniform_sweeps_match_oracle(lib, sizes, a):
    h = inputs.hamiltonian_sizes(sizes, a, seed=inputs.BASE_SEED + 70)
    B = inputs.lesser_rhs_sizes(sizes, a, seed=inputs.BASE_SEED + 71)
    A = rgf.assemble_a(h, 0.3, 1e-3, 0.5)
    R, L = _solve(lib, sizes, a, A, B)
    oR, oL = rgf.selquad(A, B)
    keys = KEYS if len(sizes) > 1 else ("diag", "arrow_r", "arrow_b", "tip")
    assert max_block_rel_err(R, oR, keys) < 1e-11
    assert max_block_rel_err(L, oL, keys) < 1e-11


def test_uniform_sizes_same_bits_either_way(lib):
    n, b, a = 5, 4, 3
    sizes = [b] * n
    h = inputs.hamiltonian_sizes(sizes, a, seed=inputs.BASE_SEED + 72)
    B = inputs.lesser_rhs_sizes(sizes, a, seed=inputs.BASE_SEED + 73)
    A = rgf.assemble_a(h, 0.3, 1e-3, 0.5)
    R1, L1 = _solve(lib, sizes, a, A, B, uniform=True)
    R2, L2 = _solve(lib, sizes, a, A, B, uniform=False)
    for k in KEYS:
        for X1, X2 in ((R1, R2), (L1, L2)):
            x1 = X1[k] if not isinstance(X1[k], list) else np.concatenate([v.ravel() for v in X1[k]])
            x2 = X2[k] if not isinstance(X2[k], list) else np.concatenate([v.ravel() for v in X2[k]])
            assert np.array_equal(x1, x2), k
    oR, oL = rgf.selquad(A, B)
    assert max_block_rel_err(R1, oR) < 1e-11 and max_block_rel_err(L1, oL) < 1e-11
