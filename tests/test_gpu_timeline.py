"""qsi_stats_timeline: the per-launch event timeline of a timed solve."""
import numpy as np
import pytest

from conftest import make_problem

pytestmark = pytest.mark.gpu


def test_timeline_matches_timed_launches():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os

    from paper_2601_04904_gb300 import qsi

    n, b, a = 6, 64, 32
    _, A, B = make_problem(n, b, a, seed=21, eta=0.1)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    Ad, Bd = qsi.to_device(A), qsi.to_device(B)
    os.environ["QSI_NO_GRAPH"] = "1"
    try:
        ctx.stats_reset(True)
        ctx.solve(Ad, [Bd], precision=qsi.FP64_EMU)
        ctx.synchronize()
        tl = ctx.stats_timeline()
        st = ctx.stats()
    finally:
        del os.environ["QSI_NO_GRAPH"]
    k, s, t0, t1 = tl["kind"], tl["stream"], tl["start_ms"], tl["end_ms"]
    assert len(k) > 0 and len(k) <= st["launches"]
    assert set(k.tolist()) <= set(range(8)) and 2 in k.tolist() and 5 in k.tolist()  # products, FP32 Gauss-Jordan
    assert np.all(t1 >= t0) and t0.min() == 0.0
    assert len(set(s.tolist())) >= 2  # main and side (and shadow) streams
    # the per-family sums agree with qsi_stats_read
    tc_ms = float((t1 - t0)[k == 2].sum())
    assert abs(tc_ms - st["tc_ms"]) <= 1e-3 * max(1.0, st["tc_ms"])
    ctx.stats_reset(False)
    assert len(ctx.stats_timeline()["kind"]) == 0
    ctx.close()
