"""GPU tests of the continuous-batching server (qsi_serve_*): every request's
result is identical alone and in the mix, and matches the oracle."""
import time

import numpy as np
import pytest

from conftest import make_problem
from oracle import rgf
from paper_2601_04904_gb300.metrics import max_block_rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10

SHAPES = [(4, 40, 16, True), (3, 65, 0, True), (6, 32, 8, False), (2, 100, 50, True), (5, 48, 24, True),
          (1, 8, 3, True), (3, 80, 0, False), (4, 70, 33, True), (2, 128, 64, True), (7, 24, 12, True)]


def _wait(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        if time.time() - t0 > timeout:
            raise TimeoutError("server did not finish")
        time.sleep(0.001)
    return out


@pytest.fixture(scope="module")
def qsi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04904_gb300 import qsi as q

    return q


def _problems(qsi, precisions):
    probs = []
    for k, (n, b, a, quad) in enumerate(SHAPES):
        _, A, B = make_problem(n, b, a, seed=k)
        probs.append((A, B if quad else None, precisions[k % len(precisions)]))
    return probs


@pytest.mark.parametrize("precision", ["fp64", "fp64_emu", "fp64_emu+mixed"])
def test_mix_equals_alone_and_oracle(qsi, precision):
    """Requests alone and in the mix give the same bits; against the oracle
    within 1e-10 (FP64, FP64_EMU) or 1e-6 (mixed); "fp64_emu+mixed" alternates
    the two precisions of the serving stream within one server."""
    precs = [qsi.PRECISIONS[p] for p in precision.split("+")]
    probs = _problems(qsi, precs)
    # alone: one request at a time through the ordinary path
    ctx = qsi.Context(0)
    alone = []
    for A, B, p in probs:
        f = ctx.factor(qsi.to_device(A), qsi.to_device(B) if B is not None else None, p)
        if B is None:
            res = (qsi.to_host(ctx.selinv(f)), None)
        else:
            GR, GL = ctx.selquad(f)
            res = (qsi.to_host(GR), qsi.to_host(GL))
        ctx.synchronize()
        f.close()
        alone.append(res)
    ctx.close()
    # mix: all submitted at once to a 3-slot server
    srv = qsi.Server(0, slots=3)
    outs, tickets = [], []
    for A, B, p in probs:
        n, b, a = qsi.shape_of(A)
        GR = qsi.device_zeros(n, b, a)
        GL = qsi.device_zeros(n, b, a) if B is not None else None
        Ad = qsi.to_device(A)
        Bd = qsi.to_device(B) if B is not None else None
        tickets.append(srv.submit(Ad, Bd, GR, GL, p))
        outs.append((GR, GL))
    res = _wait(srv, tickets)
    srv.close()
    bad = {i: r for i, (t, r) in enumerate(sorted(res.items())) if r["status"] != qsi.OK}
    assert not bad, f"requests with errors (index: result): {bad}"
    assert len({r["slot"] for r in res.values()}) > 1  # work was spread over slots
    # requests' work overlapped on the device: some pair of device intervals intersects
    iv = sorted((r["device_start_ms"], r["device_end_ms"]) for r in res.values())
    assert all(e > s for s, e in iv)
    overlap = max(min(iv[i][1], iv[j][1]) - max(iv[i][0], iv[j][0])
                  for i in range(len(iv)) for j in range(i + 1, len(iv)))
    assert overlap > 0.0, iv
    for (A, B, p), (GR, GL), (aR, aL) in zip(probs, outs, alone):
        tol = 1e-6 if p == qsi.MIXED else TOL
        gr = qsi.to_host(GR)
        for k in qsi.KEYS:
            assert np.array_equal(gr[k], aR[k])
        if B is not None:
            gl = qsi.to_host(GL)
            for k in qsi.KEYS:
                assert np.array_equal(gl[k], aL[k])
            oR, oL = rgf.selquad(A, B)
            assert max_block_rel_err(gl, oL) < tol
        else:
            oR = rgf.selinv(A)
        assert max_block_rel_err(gr, oR) < tol


def test_budget_admission_and_rejection(qsi):
    n, b, a = 3, 64, 32
    need = qsi.request_bytes(n, b, a, True, qsi.FP64)
    # budget for exactly one request at a time: requests run one after another
    srv = qsi.Server(0, slots=4, hbm_budget=need + need // 2)
    probs = [make_problem(n, b, a, seed=40 + k)[1:] for k in range(4)]
    outs, tickets = [], []
    for A, B in probs:
        GR, GL = qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a)
        tickets.append(srv.submit(qsi.to_device(A), qsi.to_device(B), GR, GL))
        outs.append((GR, GL))
    res = _wait(srv, tickets)
    for (A, B), (GR, GL), t in zip(probs, outs, tickets):
        assert res[t]["status"] == qsi.OK
        oR, oL = rgf.selquad(A, B)
        assert max_block_rel_err(qsi.to_host(GL), oL) < TOL
    # queueing: later requests waited for the budget
    assert max(r["queue_ms"] for r in res.values()) > 0.0
    # a request larger than the whole budget is refused at submit
    big = make_problem(3, 200, 100, seed=9)
    with pytest.raises(qsi.QsiError) as ei:
        srv.submit(qsi.to_device(big[1]), qsi.to_device(big[2]), qsi.device_zeros(3, 200, 100),
                   qsi.device_zeros(3, 200, 100))
    assert ei.value.status == qsi.ERR_BUSY
    srv.close()
