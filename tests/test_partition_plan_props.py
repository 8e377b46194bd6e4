"""Property tests of the partitioned solve's move plan (qsi_partition_plan,
Sec. III-B on one GPU) over random shapes, partition counts, right-hand-side
counts and output forms (host only).

For every valid (n, b, a, P): the plan exists exactly when 2P - 1 <= n; within
a phase no element is written twice and none is read that the phase writes
(one launch may run a phase's moves in any order); phase 3 writes every
element of the caller's outputs exactly once; every element of the caller's
inputs is read; the reduced system is assembled in phase 1 alone.  Run in
numpy with the partial sweeps and the oracle for the reduced system, the plan
reproduces the oracle's unpartitioned solve within the conditioning bound
1e-13 kappa^2 of the partitions' pivots (plus 1e-10)."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from conftest import make_problem  # noqa: E402
from oracle import rgf  # noqa: E402
from paper_2601_04904_gb300 import inputs  # noqa: E402
from paper_2601_04904_gb300.metrics import max_block_rel_err  # noqa: E402
from test_partition_plan import (K_IN, K_OUT, K_RED, aid, partition_pivot_kappa,  # noqa: E402
                                 partitioned_solve, qsi)

# P up to one past the largest valid count (n + 1) / 2, so both sides of the limit are drawn
shapes = st.integers(1, 20).flatmap(
    lambda n: st.tuples(st.just(n), st.integers(1, 3), st.integers(0, 3), st.integers(2, max(2, (n + 1) // 2 + 1)),
                        st.integers(0, 2), st.booleans()))


@settings(max_examples=80, deadline=None)
@given(shapes)
def test_plan_structure(shape):
    n, b, a, P, k, diag = shape
    plan = qsi.partition_plan(n, b, a, P, k, diag)
    if 2 * P - 1 > n:
        assert plan is None
        return
    assert plan is not None
    moves, sizes, pe, meta = plan
    assert meta[0] == P and meta[3] == P - 1
    assert meta[2] == (a if P == 2 else b + a)
    assert list(pe) == sorted(pe) and pe[3] == len(moves)
    written, read_all = {}, set()
    lo = 0
    for ph, hi in enumerate(pe):
        w_ph, r_ph = set(), set()
        for x in moves[lo:hi]:
            for r in range(x.rows):
                for c in range(x.cols):
                    e = (x.dst, x.dst_off + r * x.ldd + c)
                    assert e not in w_ph, (ph, e)
                    w_ph.add(e)
                    written.setdefault(e, []).append(ph)
                    for s in range(3):
                        if x.src[s] >= 0:
                            for j in range(x.cnt[s]):
                                r_ph.add((x.src[s], x.off[s] + j * x.stride[s] + r * x.lds[s] + c))
        assert not (w_ph & r_ph), ph
        read_all |= r_ph
        lo = hi
    for f in range(1 + k):
        for kk in range(6):
            out_id, in_id, red = aid(K_OUT, f, kk), aid(K_IN, f, kk), aid(K_RED, f, kk)
            for e in range(int(sizes[out_id])):
                assert written.get((out_id, e)) == [3], (f, kk, e)
            for e in range(int(sizes[in_id])):
                assert (in_id, e) in read_all, (f, kk, e)
            for e in range(int(sizes[red])):
                assert written.get((red, e)) == [1], (f, kk, e)


@settings(max_examples=60, deadline=None)
@given(shapes, st.integers(0, 1000))
def test_plan_solves_like_the_oracle(shape, seed):
    n, b, a, P, k, diag = shape
    hyp.assume(2 * P - 1 <= n)
    _, A, B = make_problem(n, b, a, seed=seed, eta=0.1)
    Bs = ([B] + [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 900 + seed + r) for r in range(1, k)])[:k]
    res, _ = partitioned_solve(A, Bs, P, diag)
    bound = 1e-13 * partition_pivot_kappa(A, P) ** 2 + 1e-10
    keys = ("diag", "arrow_r", "arrow_b", "tip") if diag else rgf_keys()
    assert max_block_rel_err(res[0], rgf.selinv(A), keys) < bound
    for r in range(k):
        assert max_block_rel_err(res[1 + r], rgf.selquad(A, Bs[r])[1], keys) < bound, r
    assert all(np.all(np.isfinite(v)) for d in res for v in d.values())


def rgf_keys():
    return ("diag", "upper", "lower", "arrow_r", "arrow_b", "tip")
