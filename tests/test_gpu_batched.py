"""GPU parity of the batched energy sweep (qsi_bta_selquad_batched): every
point against the oracle, against the single-solve path, and independent of
how the points are split into waves."""
import numpy as np
import pytest

from oracle import rgf
from paper_2601_04904_gb300 import inputs
from paper_2601_04904_gb300.metrics import max_block_rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _setup(n, b, a, nE, seed=0):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04904_gb300 import qsi

    h = inputs.hamiltonian(n, b, a, seed=inputs.BASE_SEED + seed)
    E, g = inputs.energy_grid(nE, seed=inputs.BASE_SEED + 1 + seed)
    Bs = [inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 100 + k) for k in range(nE)]
    Bst = {k: np.ascontiguousarray(np.stack([Bk[k] for Bk in Bs])) for k in qsi.KEYS}
    return qsi, h, E, g, Bs, Bst


def _host(qsi, m, k):
    return {key: m[key][k].cpu().numpy() for key in qsi.KEYS}


@pytest.mark.parametrize("n,b,a,nE", [(4, 40, 16, 5), (3, 80, 0, 3), (2, 70, 33, 4), (1, 8, 3, 2)])
def test_batched_matches_oracle(n, b, a, nE):
    qsi, h, E, g, Bs, Bst = _setup(n, b, a, nE)
    ctx = qsi.Context(0)
    GR, GL = ctx.selquad_batched(qsi.to_device(h), E, 1e-3, g, qsi.to_device(Bst))
    ctx.synchronize()
    for k in range(nE):
        oR, oL = rgf.selquad(rgf.assemble_a(h, E[k], 1e-3, g[k]), Bs[k])
        assert max_block_rel_err(_host(qsi, GR, k), oR) < TOL, k
        assert max_block_rel_err(_host(qsi, GL, k), oL) < TOL, k
    ctx.close()


def test_batched_equals_single_solves_bitwise_and_waves(monkeypatch):
    """Batched points, single solves and a 2-point wave split give identical bits
    (every point runs the same tiles in the same order)."""
    n, b, a, nE = 3, 48, 24, 5
    qsi, h, E, g, Bs, Bst = _setup(n, b, a, nE, seed=3)
    ctx = qsi.Context(0)
    Hd, Bd = qsi.to_device(h), qsi.to_device(Bst)
    GR, GL = ctx.selquad_batched(Hd, E, 1e-3, g, Bd)
    ctx.synchronize()
    for k in range(nE):
        A = ctx.assemble(Hd, float(E[k]), 1e-3, float(g[k]))
        f = ctx.factor(A, qsi.to_device(Bs[k]))
        r1, l1 = ctx.selquad(f)
        ctx.synchronize()
        f.close()
        for key in qsi.KEYS:
            assert np.array_equal(r1[key].cpu().numpy(), GR[key][k].cpu().numpy()), (k, key)
            assert np.array_equal(l1[key].cpu().numpy(), GL[key][k].cpu().numpy()), (k, key)
    ctx.close()
    monkeypatch.setenv("QSI_MAX_WAVE", "2")
    ctx2 = qsi.Context(0)
    GR2, GL2 = ctx2.selquad_batched(Hd, E, 1e-3, g, Bd)
    ctx2.synchronize()
    for key in qsi.KEYS:
        assert np.array_equal(GR2[key].cpu().numpy(), GR[key].cpu().numpy()), key
        assert np.array_equal(GL2[key].cpu().numpy(), GL[key].cpu().numpy()), key
    ctx2.close()


def test_batched_graph_replay_matches_direct(monkeypatch):
    """On a capturable stream a single-wave batch is captured into a CUDA graph
    once and replayed; a replay with new energies gives the same bits as the
    direct (uncaptured) path."""
    torch = pytest.importorskip("torch")
    n, b, a, nE = 3, 48, 24, 4
    qsi, h, E, g, Bs, Bst = _setup(n, b, a, nE, seed=8)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    Hd, Bd = qsi.to_device(h), qsi.to_device(Bst)
    GR = qsi.batched_zeros(nE, n, b, a)
    GL = qsi.batched_zeros(nE, n, b, a)
    outs = []
    for E_k in (E, E[::-1].copy()):
        with torch.cuda.stream(stream):
            ctx.selquad_batched(Hd, E_k, 1e-3, 0.5 + 0.3 * E_k, Bd, GR, GL)
        ctx.synchronize()
        outs.append(({k: GR[k].cpu().numpy() for k in qsi.KEYS}, {k: GL[k].cpu().numpy() for k in qsi.KEYS}))
    monkeypatch.setenv("QSI_NO_GRAPH", "1")
    for (oR, oL), E_k in zip(outs, (E, E[::-1].copy())):
        with torch.cuda.stream(stream):
            ctx.selquad_batched(Hd, E_k, 1e-3, 0.5 + 0.3 * E_k, Bd, GR, GL)
        ctx.synchronize()
        for k in qsi.KEYS:
            assert np.array_equal(GR[k].cpu().numpy(), oR[k]), k
            assert np.array_equal(GL[k].cpu().numpy(), oL[k]), k
    # and the replayed (second) call is right against the oracle
    for k_pt in range(nE):
        Ek = E[::-1][k_pt]
        oR_, oL_ = rgf.selquad(rgf.assemble_a(h, Ek, 1e-3, 0.5 + 0.3 * Ek), Bs[k_pt])
        assert max_block_rel_err({kk: outs[1][1][kk][k_pt] for kk in qsi.KEYS}, oL_) < TOL
    ctx.close()


@pytest.mark.parametrize("prec_name", ["FP64_EMU", "MIXED"])
@pytest.mark.parametrize("mode", ["waves", "waves2", "lanes1", "lanes3"])
def test_batched_tensor_core_matches_single_solves(monkeypatch, mode, prec_name):
    """Tensor-core precisions batched: point-major waves (every launch covers
    all points of a wave; "waves2": two points per wave, so that a ragged last
    wave occurs), or single-point solves over concurrent lanes
    (QSI_BATCHED_LANES); every point bitwise equal to its own single solve, and
    in QSI_FP64_EMU within 1e-10 of the oracle."""
    torch = pytest.importorskip("torch")
    if mode.startswith("lanes"):
        monkeypatch.setenv("QSI_BATCHED_LANES", "1")
        monkeypatch.setenv("QSI_TC_LANES", mode[-1])
    elif mode == "waves2":
        monkeypatch.setenv("QSI_TC_WAVE", "2")
    n, b, a, nE = 3, 48, 24, 5
    qsi, h, E, g, Bs, Bst = _setup(n, b, a, nE, seed=12)
    ctx = qsi.Context(0)
    Hd, Bd = qsi.to_device(h), qsi.to_device(Bst)
    GR = qsi.batched_zeros(nE, n, b, a)
    GL = qsi.batched_zeros(nE, n, b, a)
    prec = getattr(qsi, prec_name)
    ctx.selquad_batched(Hd, E, 1e-3, g, Bd, GR, GL, prec)
    ctx.synchronize()
    for k in range(nE):
        A = ctx.assemble(Hd, float(E[k]), 1e-3, float(g[k]))
        f = ctx.factor(A, qsi.to_device(Bs[k]), precision=prec)
        sR, sL = ctx.selquad(f)
        ctx.synchronize()
        f.close()
        for key in qsi.KEYS:
            assert np.array_equal(GR[key][k].cpu().numpy(), sR[key].cpu().numpy()), (k, key)
            assert np.array_equal(GL[key][k].cpu().numpy(), sL[key].cpu().numpy()), (k, key)
        if prec != qsi.FP64_EMU:
            continue
        oR, oL = rgf.selquad(rgf.assemble_a(h, float(E[k]), 1e-3, float(g[k])), Bs[k])
        assert max_block_rel_err({kk: GR[kk][k].cpu().numpy() for kk in qsi.KEYS}, oR) < TOL
        assert max_block_rel_err({kk: GL[kk][k].cpu().numpy() for kk in qsi.KEYS}, oL) < TOL
    ctx.close()


@pytest.mark.parametrize("n,b,a,nE", [(2, 70, 33, 3), (3, 80, 0, 4), (2, 20, 90, 3), (1, 600, 40, 2)])
def test_batched_tensor_core_shapes_match_oracle(n, b, a, nE):
    """Point-major tensor-core waves on ragged shapes: arrow wider than the
    blocks (the tip inversion is the larger one), no arrow, a single block,
    and blocks past 512 (two panel rows per thread), against the oracle."""
    qsi, h, E, g, Bs, Bst = _setup(n, b, a, nE, seed=21)
    ctx = qsi.Context(0)
    GR, GL = ctx.selquad_batched(qsi.to_device(h), E, 1e-3, g, qsi.to_device(Bst), precision=qsi.FP64_EMU)
    ctx.synchronize()
    for k in range(nE):
        oR, oL = rgf.selquad(rgf.assemble_a(h, E[k], 1e-3, g[k]), Bs[k])
        assert max_block_rel_err(_host(qsi, GR, k), oR) < TOL, k
        assert max_block_rel_err(_host(qsi, GL, k), oL) < TOL, k
    ctx.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU", "MIXED"])
@pytest.mark.parametrize("wave", [None, "3"])
def test_batched_graph_every_precision(monkeypatch, prec_name, wave):
    """On a stream context a batch is one CUDA-graph launch in every precision,
    also with several waves (QSI_TC_WAVE / QSI_MAX_WAVE = 3 for 7 points): the
    first call runs directly and captures, later calls replay (also with a new
    energy grid of the same length); every replay is bitwise equal to the
    direct run on the legacy stream."""
    torch = pytest.importorskip("torch")
    if wave:
        monkeypatch.setenv("QSI_TC_WAVE", wave)
        monkeypatch.setenv("QSI_MAX_WAVE", wave)
    n, b, a, nE = 3, 40, 16, 7
    qsi, h, E, g, Bs, Bst = _setup(n, b, a, nE, seed=33)
    prec = getattr(qsi, prec_name)
    stream = torch.cuda.Stream()
    ctx = qsi.Context(0, stream=stream)
    ctx0 = qsi.Context(0)
    Hd, Bd = qsi.to_device(h), qsi.to_device(Bst)
    GR, GL = qsi.batched_zeros(nE, n, b, a), qsi.batched_zeros(nE, n, b, a)
    torch.cuda.synchronize()
    g0 = ctx.stats()["graph_launches"]
    for call in range(3):
        Ec = E if call < 2 else E[::-1].copy()
        gc = g if call < 2 else g[::-1].copy()
        ctx.selquad_batched(Hd, Ec, 1e-3, gc, Bd, GR, GL, prec)
        ctx.synchronize()
        R0, L0 = ctx0.selquad_batched(Hd, Ec, 1e-3, gc, Bd, precision=prec)
        ctx0.synchronize()
        for key in qsi.KEYS:
            assert np.array_equal(GR[key].cpu().numpy(), R0[key].cpu().numpy()), (call, key)
            assert np.array_equal(GL[key].cpu().numpy(), L0[key].cpu().numpy()), (call, key)
    # tensor-core precisions: the first call ran directly (measuring the
    # scratch) and captured; FP64 captured and launched the graph at once
    assert ctx.stats()["graph_launches"] - g0 == (3 if prec == qsi.FP64 else 2)
    if prec == qsi.FP64_EMU:
        for k in range(nE):
            oR, oL = rgf.selquad(rgf.assemble_a(h, E[::-1][k], 1e-3, g[::-1][k]), Bs[k])
            assert max_block_rel_err(_host(qsi, GL, k), oL) < TOL, k
    ctx.close()
    ctx0.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP64_EMU"])
def test_batched_autotuner_bitwise_and_cached(monkeypatch, tmp_path, prec_name):
    """QSI_AUTOTUNE_CACHE: the first batch of a key is tuned (points per wave,
    reconstruction outputs per thread, moduli-per-CTA overhead), the winner is
    appended to the cache file; a new context reads it back without tuning.
    Tuned results are bitwise the untuned ones, point by point, and match the
    oracle."""
    torch = pytest.importorskip("torch")
    n, b, a, nE = 2, 48, 24, 20
    qsi, h, E, g, Bs, Bst = _setup(n, b, a, nE, seed=44)
    prec = getattr(qsi, prec_name)
    Hd, Bd = qsi.to_device(h), qsi.to_device(Bst)
    plain = qsi.Context(0)
    R0, L0 = plain.selquad_batched(Hd, E, 1e-3, g, Bd, precision=prec)
    plain.synchronize()
    assert not plain.batched_config()["tuned"]
    plain.close()
    cache = str(tmp_path / "tune.txt")
    monkeypatch.setenv("QSI_AUTOTUNE_CACHE", cache)
    cfgs = []
    for rep in range(2):  # the second context finds the key in the file
        stream = torch.cuda.Stream()
        ctx = qsi.Context(0, stream=stream)
        GR, GL = qsi.batched_zeros(nE, n, b, a), qsi.batched_zeros(nE, n, b, a)
        torch.cuda.synchronize()
        for _ in range(2):
            ctx.selquad_batched(Hd, E, 1e-3, g, Bd, GR, GL, prec)
            ctx.synchronize()
        cfg = ctx.batched_config()
        cfgs.append(cfg)
        assert cfg["tuned"] and cfg["wave"] in (8, 16, nE)
        for key in qsi.KEYS:
            assert np.array_equal(GR[key].cpu().numpy(), R0[key].cpu().numpy()), (rep, key)
            assert np.array_equal(GL[key].cpu().numpy(), L0[key].cpu().numpy()), (rep, key)
        ctx.close()
    lines = [ln for ln in open(cache).read().splitlines() if ln.startswith("qsi-batched-tune")]
    assert len(lines) == 1  # tuned once, then read back
    assert cfgs[0] == cfgs[1]
    assert qsi.autotune_cache_lookup(cache, n, b, a, prec, nE)[0] == cfgs[0]["wave"]
    for k in range(nE):
        oR, oL = rgf.selquad(rgf.assemble_a(h, E[k], 1e-3, g[k]), Bs[k])
        assert max_block_rel_err(_host(qsi, R0, k), oR) < TOL, k
        assert max_block_rel_err(_host(qsi, L0, k), oL) < TOL, k
