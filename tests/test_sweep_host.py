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
    so.host_partitioned.restype = ctypes.c_int
    so.host_partitioned_checked.restype = ctypes.c_int
    so.host_partitioned_checked.argtypes = [ctypes.c_int] * 5 + [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                                                  ctypes.c_void_p, ctypes.c_void_p]
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


@pytest.mark.parametrize("n,b,a,P,k", [(9, 3, 2, 3, 1), (17, 4, 3, 5, 2), (10, 2, 0, 3, 1), (12, 3, 2, 4, 0),
                                       (9, 3, 2, 2, 1), (16, 4, 0, 2, 2), (11, 2, 3, 2, 1)])
def test_partitioned_pipeline_with_library_sweeps(lib, n, b, a, P, k):
    """The partitioned solve end to end on the host: the library's move plan
    (run here in numpy), the library's own sweeps over the P partitions as
    batch entries with the partial flag (the schedule the GPU runs), and the
    oracle for the reduced system; the result against the oracle's
    unpartitioned solve."""
    from conftest import make_problem
    from test_partition_plan import K_IN, K_LOC, K_LOC_OUT, K_OUT, K_RED, K_RED_OUT, aid, blocks, reduced_dict, run_moves

    from paper_2601_04904_gb300 import qsi

    _, A, B = make_problem(n, b, a, seed=100 + n, eta=0.1)
    Bs = ([B] + [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 700 + r) for r in range(1, k)])[:k]
    moves, sizes, pe, (_, m, w, nr, sD, sR) = qsi.partition_plan(n, b, a, P, k)
    arrs = {i: np.zeros(max(1, int(sizes[i])), np.complex128) for i in range(qsi.PLAN_ARRAYS)}
    for f, M in enumerate([A] + Bs):
        for kk, key in enumerate(KEYS):
            if sizes[aid(K_IN, f, kk)]:
                arrs[aid(K_IN, f, kk)][:] = M[key].ravel()
    strides = (ctypes.c_longlong * 6)(sD, m * b * b, m * b * b, sR, sR, w * w)
    fam = (ctypes.c_void_p * (6 * (2 + 2 * k)))()
    for f in range(1 + k):
        for kk in range(6):
            fam[6 * f + kk] = arrs[aid(K_LOC, f, kk)].ctypes.data
            fam[6 * (1 + k + f) + kk] = arrs[aid(K_LOC_OUT, f, kk)].ctypes.data
    run_moves(arrs, moves, 0, pe[0])
    assert lib.host_sweep(0, m + 1, b, w, P, k, 1, fam, strides) == 0
    run_moves(arrs, moves, pe[0], pe[1])
    Ar = reduced_dict(arrs, K_RED, 0, nr, b, a)
    outs = [rgf.selinv(Ar)] + [rgf.selquad(Ar, reduced_dict(arrs, K_RED, f, nr, b, a))[1] for f in range(1, 1 + k)]
    for f, o in enumerate(outs):
        for kk, key in enumerate(KEYS):
            arrs[aid(K_RED_OUT, f, kk)][: o[key].size] = o[key].ravel()
    run_moves(arrs, moves, pe[1], pe[2])
    assert lib.host_sweep(1, m + 1, b, w, P, k, 1, fam, strides) == 0
    run_moves(arrs, moves, pe[2], pe[3])
    got = [{"diag": blocks(arrs[aid(K_OUT, f, 0)], n, b, b), "upper": blocks(arrs[aid(K_OUT, f, 1)], n - 1, b, b),
            "lower": blocks(arrs[aid(K_OUT, f, 2)], n - 1, b, b), "arrow_r": blocks(arrs[aid(K_OUT, f, 3)], n, b, a),
            "arrow_b": blocks(arrs[aid(K_OUT, f, 4)], n, a, b), "tip": arrs[aid(K_OUT, f, 5)][: a * a].reshape(a, a)}
           for f in range(1 + k)]
    assert max_block_rel_err(got[0], rgf.selinv(A)) < 1e-10
    for r in range(k):
        assert max_block_rel_err(got[1 + r], rgf.selquad(A, Bs[r])[1]) < 1e-10, r


@pytest.mark.parametrize("n,b,a,k", [(5, 3, 2, 2), (4, 4, 0, 3), (1, 5, 3, 2), (6, 2, 3, 1)])
def test_library_sweeps_multi_rhs_and_diagonal_only(lib, n, b, a, k):
    """The library's sweeps with k right-hand sides (one SQ recurrence each
    beside the one SI recurrence), full outputs and then diagonal-only outputs
    (upper / lower NULL: off-diagonal blocks in per-step scratch), against the
    oracle; the kept blocks bitwise equal between the two."""
    from conftest import make_problem

    _, A, _ = make_problem(n, b, a, seed=120 + n)
    Bs = [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 750 + r) for r in range(k)]
    z = lambda shape: np.zeros(shape, np.complex128)
    shapes = {"diag": (n, b, b), "upper": (max(n - 1, 0), b, b), "lower": (max(n - 1, 0), b, b),
              "arrow_r": (n, b, a), "arrow_b": (n, a, b), "tip": (a, a)}
    strides = (ctypes.c_longlong * 6)(0, 0, 0, 0, 0, 0)

    def run(diag_only):
        fac = [{key: np.ascontiguousarray(M[key]).copy() for key in KEYS} for M in [A] + Bs]
        outs = [{key: z(s) for key, s in shapes.items()} for _ in range(1 + k)]
        fam = (ctypes.c_void_p * (6 * (2 + 2 * k)))()
        for f, M in enumerate(fac + outs):
            for kk, key in enumerate(KEYS):
                skip = diag_only and f > k and key in ("upper", "lower")
                fam[6 * f + kk] = None if (skip or M[key].size == 0) else M[key].ctypes.data
        assert lib.host_sweep(0, n, b, a, 1, k, 0, fam, strides) == 0
        assert lib.host_sweep(1, n, b, a, 1, k, 0, fam, strides) == 0
        return outs

    full = run(False)
    oR = rgf.selinv(A)
    keys = KEYS if n > 1 else ("diag", "arrow_r", "arrow_b", "tip")
    assert max_block_rel_err(full[0], oR, keys) < 1e-11
    for r in range(k):
        assert max_block_rel_err(full[1 + r], rgf.selquad(A, Bs[r])[1], keys) < 1e-11, r
    diag = run(True)
    for f in range(1 + k):
        for key in ("diag", "arrow_r", "arrow_b", "tip"):
            assert np.array_equal(diag[f][key], full[f][key]), (f, key)


def test_library_sweeps_batched_points(lib):
    """Three independent problems as batch entries (per-point strides, the
    layout of the batched energy sweep), each against the oracle."""
    from conftest import make_problem

    n, b, a, nb_ = 4, 3, 2, 3
    probs = [make_problem(n, b, a, seed=140 + p) for p in range(nb_)]
    stack = lambda key, i: np.ascontiguousarray(np.stack([p[i][key] for p in probs]))
    fac = [{key: stack(key, 1) for key in KEYS}, {key: stack(key, 2) for key in KEYS}]
    outs = [{key: np.zeros_like(fac[0][key]) for key in KEYS} for _ in range(2)]
    per = {key: int(np.prod(fac[0][key].shape[1:])) for key in KEYS}
    strides = (ctypes.c_longlong * 6)(*[per[key] for key in KEYS])
    fam = (ctypes.c_void_p * 24)()
    for f, M in enumerate(fac + outs):
        for kk, key in enumerate(KEYS):
            fam[6 * f + kk] = M[key].ctypes.data
    assert lib.host_sweep(0, n, b, a, nb_, 1, 0, fam, strides) == 0
    assert lib.host_sweep(1, n, b, a, nb_, 1, 0, fam, strides) == 0
    for p, (_, A, B) in enumerate(probs):
        oR, oL = rgf.selquad(A, B)
        assert max_block_rel_err({key: outs[0][key][p] for key in KEYS}, oR) < 1e-11, p
        assert max_block_rel_err({key: outs[1][key][p] for key in KEYS}, oL) < 1e-11, p


@pytest.mark.parametrize("n,b,a,k", [(5, 3, 2, 2), (4, 4, 0, 1), (2, 3, 2, 3), (1, 4, 2, 1)])
def test_library_backward_split_same_bits(lib, n, b, a, k):
    """The backward sweep with the SQ chain split off onto the side stream
    (double-buffered U and P by step parity) computes the same products: the
    host run gives the same bits as the joint phases, for full and
    diagonal-only outputs."""
    from conftest import make_problem

    _, A, _ = make_problem(n, b, a, seed=160 + n)
    Bs = [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 770 + r) for r in range(k)]
    shapes = {"diag": (n, b, b), "upper": (max(n - 1, 0), b, b), "lower": (max(n - 1, 0), b, b),
              "arrow_r": (n, b, a), "arrow_b": (n, a, b), "tip": (a, a)}
    strides = (ctypes.c_longlong * 6)(0, 0, 0, 0, 0, 0)

    def run(split, diag_only):
        lib.host_set_split(int(split))
        try:
            fac = [{key: np.ascontiguousarray(M[key]).copy() for key in KEYS} for M in [A] + Bs]
            outs = [{key: np.zeros(s, np.complex128) for key, s in shapes.items()} for _ in range(1 + k)]
            fam = (ctypes.c_void_p * (6 * (2 + 2 * k)))()
            for f, M in enumerate(fac + outs):
                for kk, key in enumerate(KEYS):
                    skip = diag_only and f > k and key in ("upper", "lower")
                    fam[6 * f + kk] = None if (skip or M[key].size == 0) else M[key].ctypes.data
            assert lib.host_sweep(0, n, b, a, 1, k, 0, fam, strides) == 0
            assert lib.host_sweep(1, n, b, a, 1, k, 0, fam, strides) == 0
            return outs
        finally:
            lib.host_set_split(0)

    for diag_only in (False, True):
        x, y = run(False, diag_only), run(True, diag_only)
        for f in range(1 + k):
            for key in KEYS:
                assert np.array_equal(x[f][key], y[f][key]), (diag_only, f, key)
    oR, oL = rgf.selquad(A, Bs[0])
    keys = KEYS if n > 1 else ("diag", "arrow_r", "arrow_b", "tip")
    assert max_block_rel_err(y[1], oL, ("diag", "arrow_r", "arrow_b", "tip")) < 1e-11
    assert max_block_rel_err(run(True, False)[0], oR, keys) < 1e-11


def test_partitioned_pipeline_backward_split(lib):
    """The partitioned pipeline (partial sweeps over batched partitions) with the
    backward split: same result as the joint phases."""
    lib.host_set_split(1)
    try:
        test_partitioned_pipeline_with_library_sweeps(lib, 17, 4, 3, 5, 2)
    finally:
        lib.host_set_split(0)


def _ah(lib, on):
    lib.host_set_antihermitian(int(on))


@pytest.mark.parametrize("sizes,a", [([3, 5, 2, 4], 3), ([4, 4, 4, 4, 4], 2), ([6], 2), ([2, 3], 5),
                                     ([5, 4, 3, 2, 1], 0)])
def test_antihermitian_mirroring_matches_oracle(lib, sizes, a):
    """QSI_ASSUME_ANTIHERMITIAN_B: the forward arrow update B-hat_{t,i+1} and
    the backward Y21, Y_{R,i} are mirrored (-X^H) instead of multiplied.  With
    the recipe's anti-Hermitian B the sweeps still match the oracle, G^R is
    bitwise the unflagged one, and G^< is anti-Hermitian on the pattern by
    construction."""
    h = inputs.hamiltonian_sizes(sizes, a, seed=inputs.BASE_SEED + 80)
    B = inputs.lesser_rhs_sizes(sizes, a, seed=inputs.BASE_SEED + 81)
    A = rgf.assemble_a(h, 0.3, 1e-3, 0.5)
    uniform = len(set(sizes)) == 1
    R0, L0 = _solve(lib, sizes, a, A, B, uniform=uniform)
    _ah(lib, True)
    try:
        R1, L1 = _solve(lib, sizes, a, A, B, uniform=uniform)
    finally:
        _ah(lib, False)
    oR, oL = rgf.selquad(A, B)
    keys = KEYS if len(sizes) > 1 else ("diag", "arrow_r", "arrow_b", "tip")
    assert max_block_rel_err(L1, oL, keys) < 1e-11
    assert max_block_rel_err(L1, L0, keys) < 1e-11
    flat = lambda X: X if not isinstance(X, list) else np.concatenate([np.ravel(v) for v in X] or [np.zeros(0)])
    for k in KEYS:
        assert np.array_equal(flat(R0[k]), flat(R1[k])), k
    for i in range(len(sizes) - 1):
        assert np.array_equal(np.asarray(L1["lower"][i]), -np.conj(np.asarray(L1["upper"][i]).T))
    for i in range(len(sizes)):
        assert np.array_equal(np.asarray(L1["arrow_b"][i]), -np.conj(np.asarray(L1["arrow_r"][i]).T))


def test_antihermitian_mirroring_split_and_partitioned(lib):
    """The mirrored sweeps with the backward split and in the partitioned
    pipeline (partial sweeps over batched partitions, two right-hand sides)."""
    _ah(lib, True)
    lib.host_set_split(1)
    try:
        test_library_backward_split_same_bits(lib, 5, 3, 2, 2)
        test_partitioned_pipeline_with_library_sweeps(lib, 17, 4, 3, 5, 2)
    finally:
        lib.host_set_split(0)
        _ah(lib, False)
    _ah(lib, True)
    try:
        test_partitioned_pipeline_with_library_sweeps(lib, 9, 3, 2, 3, 1)
        # the twisted split: the reversed bottom half's B stays anti-Hermitian
        test_partitioned_pipeline_with_library_sweeps(lib, 9, 3, 2, 2, 1)
        test_partitioned_pipeline_with_library_sweeps(lib, 10, 4, 3, 2, 2)
    finally:
        _ah(lib, False)


@pytest.mark.parametrize("n,b,a", [(5, 4, 3), (3, 6, 0), (4, 2, 5), (1, 3, 2)])
def test_antihermitian_saving_matches_work_model(lib, n, b, a):
    """The complex multiply-adds the sweeps execute without and with mirroring
    differ by exactly what the work model subtracts for anti-Hermitian B."""
    from paper_2601_04904_gb300 import metrics

    lib.host_cmac.restype = ctypes.c_double
    sizes = [b] * n
    h = inputs.hamiltonian_sizes(sizes, a, seed=inputs.BASE_SEED + 82)
    B = inputs.lesser_rhs_sizes(sizes, a, seed=inputs.BASE_SEED + 83)
    A = rgf.assemble_a(h, 0.3, 1e-3, 0.5)
    done = []
    for on in (False, True):
        _ah(lib, on)
        try:
            lib.host_cmac(1)
            _solve(lib, sizes, a, A, B, uniform=True)
            done.append(lib.host_cmac(1))
        finally:
            _ah(lib, False)
    model = lambda ah: metrics.cmac_forward(n, b, a, True, ah) + metrics.cmac_backward(n, b, a, True, ah)
    assert done[0] - done[1] == model(False) - model(True)
    assert done[1] < done[0] or a == 0 and n == 1


def _run_partitioned(lib, A, Bs, P, fixed, host_io, diag_only=False):
    """qsi_partitioned_run itself (csrc/partition.cu) on host arrays: its plan,
    layout, block moves and host copies, with the library's sweeps."""
    n, b, a = rgf.shape_of(A)
    k = len(Bs)
    ins = [{key: np.ascontiguousarray(M[key], dtype=np.complex128) for key in KEYS} for M in [A] + Bs]
    outs = [{key: (None if diag_only and key in ("upper", "lower") else np.zeros_like(ins[0][key])) for key in KEYS}
            for _ in range(1 + k)]
    pin = (ctypes.c_void_p * (6 * (1 + k)))()
    pout = (ctypes.c_void_p * (6 * (1 + k)))()
    for f in range(1 + k):
        for kk, key in enumerate(KEYS):
            pin[6 * f + kk] = ins[f][key].ctypes.data if ins[f][key].size else None
            o = outs[f][key]
            pout[6 * f + kk] = o.ctypes.data if o is not None and o.size else None
    full = (ctypes.c_int * (1 + k))(*([0 if diag_only else 1] * (1 + k)))
    rc = lib.host_partitioned(n, b, a, P, k, int(fixed), int(host_io), pin, pout, full)
    assert rc == 0
    return outs


@pytest.mark.parametrize("n,b,a,P,k", [(9, 3, 2, 2, 1), (10, 4, 3, 2, 1), (9, 3, 2, 3, 1), (12, 2, 0, 4, 2),
                                       (7, 3, 2, 2, 0), (17, 4, 3, 5, 2)])
@pytest.mark.parametrize("fixed", [False, True])
def test_library_partitioned_run_matches_oracle(lib, n, b, a, P, k, fixed):
    """The library's partitioned run (plan, layout, block moves, partial sweeps
    of the partitions as batch entries, reduced system, boundary hand-off), in
    its own-allocation and fixed-memory forms, against the oracle's
    unpartitioned solve."""
    from conftest import make_problem

    _, A, B = make_problem(n, b, a, seed=300 + n, eta=0.1)
    Bs = ([B] + [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 710 + r) for r in range(1, k)])[:k]
    outs = _run_partitioned(lib, A, Bs, P, fixed, False)
    assert max_block_rel_err(outs[0], rgf.selinv(A)) < 1e-10
    for r in range(k):
        assert max_block_rel_err(outs[1 + r], rgf.selquad(A, Bs[r])[1]) < 1e-10, r


@pytest.mark.parametrize("n,b,a", [(9, 3, 2), (10, 4, 3), (3, 2, 1), (8, 2, 0)])
@pytest.mark.parametrize("k", [0, 1])
@pytest.mark.parametrize("diag_only", [False, True])
def test_library_twisted_host_io_same_bits(lib, n, b, a, k, diag_only):
    """The twisted split's host input / output form (blocks copied straight
    between the caller's arrays and the partition slots, the separator and
    tip through the staging area) gives the bits of the plan's device form,
    with and without B, full and diagonal-only outputs, odd and even n."""
    from conftest import make_problem

    _, A, B = make_problem(n, b, a, seed=320 + n, eta=0.1)
    Bs = [B][:k]
    dev = _run_partitioned(lib, A, Bs, 2, True, False, diag_only)
    host = _run_partitioned(lib, A, Bs, 2, True, True, diag_only)
    for f in range(1 + k):
        for key in KEYS:
            if dev[f][key] is None:
                assert host[f][key] is None
                continue
            assert np.array_equal(host[f][key], dev[f][key]), (f, key)
    keys = ("diag", "arrow_r", "arrow_b", "tip") if diag_only else KEYS
    assert max_block_rel_err(host[0], rgf.selinv(A), keys) < 1e-10
    if k:
        assert max_block_rel_err(host[1], rgf.selquad(A, B)[1], keys) < 1e-10


def test_library_twisted_host_io_antihermitian(lib):
    """Both flags' combination on the host: the twisted split's host form
    with the mirrored sweeps (the reversed bottom half's B stays
    anti-Hermitian)."""
    from conftest import make_problem

    n, b, a = 11, 3, 2
    _, A, B = make_problem(n, b, a, seed=340, eta=0.1)
    _ah(lib, True)
    try:
        outs = _run_partitioned(lib, A, [B], 2, True, True)
    finally:
        _ah(lib, False)
    assert max_block_rel_err(outs[0], rgf.selinv(A)) < 1e-10
    assert max_block_rel_err(outs[1], rgf.selquad(A, B)[1]) < 1e-10


@pytest.mark.parametrize("eta,P", [(2.0, 4), (1e-3, 4), (0.1, 3)])
def test_library_checked_partitioned_run(lib, eta, P):
    """The automatic partition count's two stages in the library's run: the
    partitions' forward sweeps form kappa_F = ||S||_F ||S^-1||_F of every pivot
    (the estimate equals the plan's pivots' kappa_F formed in numpy), and the
    rest runs only when it is within the limit: then the result matches the
    oracle, else the outputs stay untouched."""
    from conftest import make_problem
    from test_partition_plan import partition_pivot_kappa

    n, b, a = 16, 8, 4
    _, A, B = make_problem(n, b, a, seed=360, eta=eta)
    ref_kappa = partition_pivot_kappa(A, P, frobenius=True)
    limit = (1e-10 / 1e-13) ** 0.5
    for kappa_max in (limit, 1e300):
        ins = [{key: np.ascontiguousarray(M[key], dtype=np.complex128) for key in KEYS} for M in (A, B)]
        outs = [{key: np.zeros_like(ins[0][key]) for key in KEYS} for _ in range(2)]
        pin, pout = (ctypes.c_void_p * 12)(), (ctypes.c_void_p * 12)()
        for f in range(2):
            for kk, key in enumerate(KEYS):
                pin[6 * f + kk] = ins[f][key].ctypes.data
                pout[6 * f + kk] = outs[f][key].ctypes.data
        kap = ctypes.c_double(-1.0)
        full = (ctypes.c_int * 2)(1, 1)
        rc = lib.host_partitioned_checked(n, b, a, P, 1, kappa_max, ctypes.addressof(kap), pin, pout, full)
        assert rc == 0
        assert abs(kap.value - ref_kappa) <= 1e-9 * ref_kappa
        if ref_kappa <= kappa_max:
            assert max_block_rel_err(outs[0], rgf.selinv(A)) < 1e-13 * ref_kappa ** 2 + 1e-10
            assert max_block_rel_err(outs[1], rgf.selquad(A, B)[1]) < 1e-13 * ref_kappa ** 2 + 1e-10
        else:
            assert all(not np.any(outs[f][key]) for f in range(2) for key in KEYS)


def test_library_host_io_form_rejects_what_it_does_not_cover(lib):
    """The host input / output form covers the twisted split with at most one
    right-hand side: other partition counts or more right-hand sides are an
    argument error (cudaErrorInvalidValue) before anything runs."""
    from conftest import make_problem

    n, b, a = 9, 3, 2
    _, A, B = make_problem(n, b, a, seed=380, eta=0.1)
    for P, Bs in ((3, [B]), (2, [B, B])):
        k = len(Bs)
        ins = [{key: np.ascontiguousarray(M[key], dtype=np.complex128) for key in KEYS} for M in [A] + Bs]
        outs = [{key: np.zeros_like(ins[0][key]) for key in KEYS} for _ in range(1 + k)]
        pin, pout = (ctypes.c_void_p * (6 * (1 + k)))(), (ctypes.c_void_p * (6 * (1 + k)))()
        for f in range(1 + k):
            for kk, key in enumerate(KEYS):
                pin[6 * f + kk] = ins[f][key].ctypes.data
                pout[6 * f + kk] = outs[f][key].ctypes.data
        full = (ctypes.c_int * (1 + k))(*([1] * (1 + k)))
        assert lib.host_partitioned(n, b, a, P, k, 1, 1, pin, pout, full) == 1  # cudaErrorInvalidValue
        assert all(not np.any(outs[f][key]) for f in range(1 + k) for key in KEYS)


def test_library_partitioned_run_random_shapes(lib):
    """The library's partitioned run over random shapes, partition counts,
    right-hand sides and output forms (hypothesis): within the conditioning
    bound of the oracle, and for two partitions the host-I/O form bit for bit
    the device form."""
    pytest.importorskip("hypothesis")
    from hypothesis import given, settings
    from hypothesis import strategies as st

    from conftest import make_problem
    from test_partition_plan import partition_pivot_kappa

    shapes = st.integers(3, 16).flatmap(
        lambda n: st.tuples(st.just(n), st.integers(1, 4), st.integers(0, 3), st.integers(2, (n + 1) // 2),
                            st.integers(0, 2), st.booleans(), st.integers(0, 500)))

    @settings(max_examples=40, deadline=None)
    @given(shapes)
    def check(shape):
        n, b, a, P, k, diag, seed = shape
        _, A, B = make_problem(n, b, a, seed=seed, eta=0.1)
        Bs = ([B] + [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 950 + seed + r) for r in range(1, k)])[:k]
        outs = _run_partitioned(lib, A, Bs, P, True, False, diag)
        bound = 1e-13 * partition_pivot_kappa(A, P) ** 2 + 1e-10
        keys = ("diag", "arrow_r", "arrow_b", "tip") if diag else KEYS
        assert max_block_rel_err(outs[0], rgf.selinv(A), keys) < bound
        for r in range(k):
            assert max_block_rel_err(outs[1 + r], rgf.selquad(A, Bs[r])[1], keys) < bound
        if P == 2 and k <= 1:
            host = _run_partitioned(lib, A, Bs, 2, True, True, diag)
            for f in range(1 + k):
                for key in KEYS:
                    if outs[f][key] is not None:
                        assert np.array_equal(host[f][key], outs[f][key]), (f, key)

    check()


def test_library_sweeps_random_block_sizes(lib):
    """The library's sweeps over random non-uniform block sizes (hypothesis):
    1-7 blocks of 1-6, arrow 0-4, with and without the backward split and the
    anti-Hermitian mirroring, against the oracle."""
    pytest.importorskip("hypothesis")
    from hypothesis import given, settings
    from hypothesis import strategies as st

    cases = st.tuples(st.lists(st.integers(1, 6), min_size=1, max_size=7), st.integers(0, 4), st.booleans(),
                      st.booleans(), st.integers(0, 500))

    @settings(max_examples=40, deadline=None)
    @given(cases)
    def check(case):
        sizes, a, split, ah = case[0], case[1], case[2], case[3]
        seed = case[4]
        h = inputs.hamiltonian_sizes(sizes, a, seed=inputs.BASE_SEED + 1000 + seed)
        B = inputs.lesser_rhs_sizes(sizes, a, seed=inputs.BASE_SEED + 1600 + seed)
        A = rgf.assemble_a(h, 0.3, 0.1, 0.5)
        lib.host_set_split(int(split))
        _ah(lib, ah)
        try:
            R, L = _solve(lib, sizes, a, A, B)
        finally:
            lib.host_set_split(0)
            _ah(lib, False)
        oR, oL = rgf.selquad(A, B)
        keys = KEYS if len(sizes) > 1 else ("diag", "arrow_r", "arrow_b", "tip")
        assert max_block_rel_err(R, oR, keys) < 1e-10
        assert max_block_rel_err(L, oL, keys) < 1e-10

    check()
