#!/usr/bin/env python3
"""Benchmark of the fused SI+SQ solve (one energy point = one step).

Default workload: one BTA matrix with n_blocks=64, b=512, a=256 (complex128),
built by the synthetic recipe (E=0.3, eta=1e-3, contact gamma=0.5).  A step is
the whole hot path on one matrix: forward sweep (factor) + fused backward sweep
(selquad), inputs resident in HBM (2.1 GB > L2, so no L2 flush is needed).

Prints one JSON line (rank 0).  Multi-GPU (torchrun): every rank solves its own
energy point (replicas, no collectives on the data path); value = points of all
ranks / max-over-ranks time.

The default line (N=1) also carries the other workloads of the benchmark
suite, each measured on this GPU with its own clock record: "batched" (256
energy points sharing one H, n=32, b=256, a=128), "mixed_c3" (n=128, b=1024,
a=512 in the reduced-moduli mixed precision, its per-block error against the
FP64-accurate solve, and the FP64-accurate and 3-term-split timings beside it)
and "serve" (a prefix of the seeded Poisson request stream: p50/p99 latency and
throughput); --no-suite leaves them out.

--impl reference times the CPU oracle (complex128 numpy) on a bounded sample of
the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2601_04904_gb300 import inputs, metrics, replicas  # noqa: E402

METRIC = "fused SI+SQ energy-points/sec"
UNIT = "energy-points/s"
# FP64 (DFMA) peak derived from the chip's unit counts and clock: 152 SMs x
# 2 DFMA/clk/SM (1/64 of the FP32 lanes) x 2 flop x 2.07 GHz = 1.259 TFLOP/s;
# equals the nominal 1.25 TFLOP/s FP64 figure.  Used only where no measured
# FP64 figure is at hand; the default line measures cuBLAS DGEMM / ZGEMM on
# the same GPU ("fp64_peak") and takes the larger as the FP64 denominator.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
MODULI = {"fp64_emu": 17, "mixed": 13}  # CRT moduli of the tensor-core products (QSI_MIXED_MODULI overrides)

WORKLOADS = {
    "bta_n64_b512_a256": dict(n=64, b=512, a=256),
    "bta_n128_b1024_a512": dict(n=128, b=1024, a=512),
    "bta_n8_b32_a16": dict(n=8, b=32, a=16),
    "bta_n16_b256_a128": dict(n=16, b=256, a=128),
    "bta_n8_b512_a256": dict(n=8, b=512, a=256),  # the n64 block sizes on 8 blocks (launch-list captures)
    "bta_n32_b256_a128": dict(n=32, b=256, a=128),  # one energy point of the batched workload
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="bta_n64_b512_a256", choices=sorted(WORKLOADS))
    p.add_argument("--precision", default="fp64_emu",
                   help="fp64_emu (default: FP64-accurate products on the BF16 tensor cores), fp64 (IEEE FP64 "
                        "everywhere), mixed (13-moduli products, 1e-6 per block) or split3 (3-term BF16 split, "
                        "FP32 accumulation)")
    p.add_argument("--no-suite", action="store_true",
                   help="single mode: leave out the batched, mixed_c3 and serve keys of the default line")
    p.add_argument("--no-fp64-compare", action="store_true",
                   help="single mode, precision != fp64: skip the short IEEE-FP64 run of the same matrices")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--mode", default="single", choices=["single", "batched", "serve", "partitioned", "extras"],
                   help="single: one energy point per step (default); batched: 256 energy points sharing H "
                        "(n=32, b=256, a=128) per step; serve: Poisson request stream through qsi_serve_*; "
                        "partitioned: single-solve latency of small-b shapes, plain vs partitioned solves")
    p.add_argument("--points", type=int, default=256, help="energy points of the batched mode")
    p.add_argument("--requests", type=int, default=200, help="requests of the serve mode (prefix of the stream)")
    p.add_argument("--slots", type=int, default=4)
    p.add_argument("--serve-mix", default="fp64_emu,mixed",
                   help="the two precisions of the serving stream's 50/50 mix: complex128 requests at FP64 "
                        "accuracy (fp64_emu, or the IEEE path fp64) and mixed-mode requests (mixed)")
    p.add_argument("--part-shape", default=None,
                   help="partitioned mode: one shape n,b,a instead of the default list")
    p.add_argument("--part-p", default=None, help="partitioned mode: comma-separated partition counts")
    p.add_argument("--part-only", action="store_true",
                   help="partitioned mode: time only the partitioned solve, --warmup then --steps calls "
                        "(for a launch list under a profiler)")
    p.add_argument("--ref-precision", default=None,
                   help="also solve once with this precision and report the per-block error of the timed one")
    return p.parse_args()


dist_env = replicas.env
energy_of = replicas.energy_of


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(wl: dict, target_s: float = 12.0):
    """Time the oracle on a bounded sample: the workload's b and a with fewer
    blocks; throughput is scaled to the full workload by the flop ratio."""
    from oracle import rgf

    n, b, a = wl["n"], wl["b"], wl["a"]
    ns = min(n, 2)
    while True:
        h = inputs.hamiltonian(ns, b, a)
        B = inputs.lesser_rhs(ns, b, a)
        A = rgf.assemble_a(h, 0.3, 1e-3, 0.5)
        t0 = time.perf_counter()
        rgf.selquad(A, B)
        dt = time.perf_counter() - t0
        if dt * 2 > target_s or ns >= n:
            break
        ns = min(n, max(ns * 2, int(ns * target_s / max(dt, 1e-3) * 0.8)))
    flops_ratio = metrics.flops_selquad(ns, b, a) / metrics.flops_selquad(n, b, a)
    value = flops_ratio / dt  # full-workload solves per second
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)))
    sample = (f"oracle (numpy complex128) on n_blocks={ns} of the workload's b={b}, a={a} "
              f"({dt:.2f} s), scaled to n_blocks={n} by the flop ratio {flops_ratio:.4f}")
    return value, cores, sample, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    times = []
    # each step a bounded sample: the whole run stays within a few minutes
    target = max(2.0, min(8.0, 150.0 / max(1, args.warmup + args.steps)))
    for i in range(args.warmup + args.steps):
        v, cores, sample, dt = oracle_sample(wl, target_s=target)
        if i >= args.warmup:
            times.append(1.0 / v)
    ms = 1e3 * statistics.mean(times)
    value = 1e3 / ms
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, wl, impl="reference"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def config_of(args, wl, impl="ours"):
    n, b, a = wl["n"], wl["b"], wl["a"]
    inb = 2 * metrics.bytes_bta(n, b, a)
    if impl == "reference":
        return {"workload": args.workload, "n_blocks": n, "b": b, "a": a,
                "precision": "complex128 (numpy, IEEE double)", "E": 0.3, "eta": 1e-3, "gamma": 0.5,
                "call": "oracle.rgf.selquad (plain CPU sweep, threaded BLAS) on the host cores",
                "sample": "each step a bounded sample of the workload's blocks, scaled by the flop ratio"}
    return {"workload": args.workload, "n_blocks": n, "b": b, "a": a, "precision": args.precision,
            "E": 0.3, "eta": 1e-3, "gamma": 0.5, "call": "qsi_bta_solve (graph-cached on its stream)",
            "l2": f"inputs larger than L2 ({inb / 1e9:.2f} GB of A and B per step)" if inb > 129e6
            else "inputs smaller than L2: L2 not flushed (latency-bound case)"}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"qsi_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
def device_bta_hermitian(torch, n, b, a, gen, scale):
    """Seeded Hermitian BTA matrix generated on the device (benchmark inputs only)."""
    cplx = lambda *s: torch.complex(torch.randn(*s, generator=gen, device="cuda", dtype=torch.float64),
                                    torch.randn(*s, generator=gen, device="cuda", dtype=torch.float64)) * scale
    d = cplx(n, b, b)
    d = 0.5 * (d + d.transpose(-1, -2).conj())
    u = cplx(n - 1, b, b)
    r = cplx(n, b, a)
    t = cplx(a, a)
    return {"diag": d.contiguous(), "upper": u.contiguous(), "lower": u.transpose(-1, -2).conj().contiguous(),
            "arrow_r": r.contiguous(), "arrow_b": r.transpose(-1, -2).conj().contiguous(),
            "tip": (0.5 * (t + t.T.conj())).contiguous()}


def device_bta_antihermitian(torch, n, b, a, gen, lead=()):
    cplx = lambda *s: torch.complex(torch.randn(*s, generator=gen, device="cuda", dtype=torch.float64),
                                    torch.randn(*s, generator=gen, device="cuda", dtype=torch.float64))
    d = cplx(*lead, n, b, b)
    d = d - d.transpose(-1, -2).conj()
    u = cplx(*lead, n - 1, b, b)
    r = cplx(*lead, n, b, a)
    t = cplx(*lead, a, a)
    return {"diag": d.contiguous(), "upper": u.contiguous(), "lower": (-u.transpose(-1, -2).conj()).contiguous(),
            "arrow_r": r.contiguous(), "arrow_b": (-r.transpose(-1, -2).conj()).contiguous(),
            "tip": (t - t.transpose(-1, -2).conj()).contiguous()}


def run_extras(args):
    """Cost of the widened variants next to the plain solve, same GPU, same
    precision: G^< and G^> in one sweep (two right-hand sides) against one,
    diagonal-only outputs against full ones (c1 shape, graph replays), and a
    solve with non-uniform blocks against the uniform solve of the same total
    size (direct launches on the legacy default stream for both)."""
    import torch

    from paper_2601_04904_gb300 import qsi

    prec = qsi.PRECISIONS[args.precision]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = qsi.Context(0, stream=stream)

    def timed(fn, c, st, reps=3, warm=2):
        for _ in range(warm):
            fn()
        c.synchronize()
        torch.cuda.synchronize()
        if st is None:  # legacy default stream: host clock around the calls, device drained after each
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
                c.synchronize()
            return (time.perf_counter() - t0) * 1e3 / reps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        c.synchronize()
        return e0.elapsed_time(e1) / reps

    n, b, a = 64, 512, 256
    gen = torch.Generator(device="cuda").manual_seed(inputs.BASE_SEED + 5000)
    Ad = device_bta_hermitian(torch, n, b, a, gen, 1.0 / np.sqrt(b))
    ctx.assemble(Ad, 0.3, 1e-3, 0.5, out=Ad)
    B1, B2 = device_bta_antihermitian(torch, n, b, a, gen), device_bta_antihermitian(torch, n, b, a, gen)
    GR, G1, G2 = qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a)
    DR, D1 = qsi.device_zeros(n, b, a, off_diagonal=False), qsi.device_zeros(n, b, a, off_diagonal=False)
    torch.cuda.synchronize()
    one = timed(lambda: ctx.solve(Ad, [B1], GR, [G1], prec), ctx, stream)
    two = timed(lambda: ctx.solve(Ad, [B1, B2], GR, [G1, G2], prec), ctx, stream)
    diag = timed(lambda: ctx.solve(Ad, [B1], DR, [D1], prec), ctx, stream)
    del Ad, B1, B2, GR, G1, G2, DR, D1
    torch.cuda.empty_cache()

    # non-uniform blocks: n=32 blocks alternating 192 / 320 (mean 256), a=128,
    # against the uniform (32, 256, 128) solve; A = (E + i eta) I - H - i gamma I
    # on every diagonal (inputs only), B anti-Hermitian
    ctx0 = qsi.Context(0)
    nv, av = 32, 128
    sizes = [192 if i % 2 == 0 else 320 for i in range(nv)]
    g2 = torch.Generator(device="cuda").manual_seed(inputs.BASE_SEED + 5001)
    cn = lambda *s: torch.complex(torch.randn(*s, generator=g2, device="cuda", dtype=torch.float64),
                                  torch.randn(*s, generator=g2, device="cuda", dtype=torch.float64))
    sc = 1.0 / np.sqrt(max(sizes))
    z = complex(0.3, 1e-3) + 0.5j

    def ragged(hermitian):
        d = []
        for s_ in sizes:
            x = cn(s_, s_) * (sc if hermitian else 1.0)
            x = 0.5 * (x + x.conj().T) if hermitian else x - x.conj().T
            d.append(z * torch.eye(s_, dtype=torch.complex128, device="cuda") - x if hermitian else x)
        up = [cn(sizes[i], sizes[i + 1]) * (sc if hermitian else 1.0) for i in range(nv - 1)]
        lo = [(-u.conj().T if hermitian else -u.conj().T) for u in up]
        ar = [cn(s_, av) * (sc if hermitian else 1.0) for s_ in sizes]
        ab = [(-r.conj().T if hermitian else -r.conj().T) for r in ar]
        up = [-u if hermitian else u for u in up]
        ar = [-r if hermitian else r for r in ar]
        t = cn(av, av) * (sc if hermitian else 1.0)
        t = (z * torch.eye(av, dtype=torch.complex128, device="cuda") - 0.5 * (t + t.conj().T)) if hermitian \
            else t - t.conj().T
        flat = lambda xs: torch.cat([x.reshape(-1) for x in xs]).contiguous()
        return {"diag": flat(d), "upper": flat(up), "lower": flat(lo), "arrow_r": flat(ar), "arrow_b": flat(ab),
                "tip": t.reshape(-1).contiguous()}

    Av, Bv = ragged(True), ragged(False)
    VR, VX = qsi.flat_zeros(sizes, av), [qsi.flat_zeros(sizes, av)]
    torch.cuda.synchronize()
    l0 = ctx0.stats()["launches"]
    var_ms = timed(lambda: ctx0.solve_varsize(sizes, Av, [Bv], VR, VX, prec), ctx0, None)
    var_launches = (ctx0.stats()["launches"] - l0) / 5
    del Av, Bv, VR, VX
    gen3 = torch.Generator(device="cuda").manual_seed(inputs.BASE_SEED + 5002)
    Au = device_bta_hermitian(torch, nv, 256, av, gen3, 1.0 / np.sqrt(256))
    ctx0.assemble(Au, 0.3, 1e-3, 0.5, out=Au)
    Bu = device_bta_antihermitian(torch, nv, 256, av, gen3)
    UR, UX = qsi.device_zeros(nv, 256, av), [qsi.device_zeros(nv, 256, av)]
    torch.cuda.synchronize()
    l0 = ctx0.stats()["launches"]
    uni_ms = timed(lambda: ctx0.solve(Au, [Bu], UR, UX, prec), ctx0, None)
    uni_launches = (ctx0.stats()["launches"] - l0) / 5
    print(json.dumps({
        "metric": "widened variants, ms per solve", "mode": "extras", "unit": "ms", "higher_is_better": False,
        "n_gpus": 1, "precision": args.precision, "dtype": "f64", "data": "synthetic",
        "c1_one_rhs_ms": one, "c1_two_rhs_ms": two, "second_rhs_cost": two / one - 1.0,
        "c1_diag_only_ms": diag, "diag_only_saving": 1.0 - diag / one,
        "varsize_n32_192_320_a128_ms": var_ms, "uniform_n32_b256_a128_ms": uni_ms,
        "varsize_over_uniform": var_ms / uni_ms, "varsize_launches": var_launches, "uniform_launches": uni_launches,
        "config": {"workload": "c1 (n=64, b=512, a=256) for right-hand sides and diagonal-only outputs; "
                               "n=32 blocks of 192/320 vs 256, a=128 for non-uniform blocks",
                   "timing": "2 warm-up + 3 timed calls each; c1: CUDA events around graph replays; "
                             "non-uniform vs uniform: host clock per call to completion on the legacy stream"}}))
    ctx.close()
    ctx0.close()


def measure_batched(points=256, steps=2, warmup=1, precision="fp64_emu"):
    """256 energy points sharing one H (n=32, b=256, a=128): one
    qsi_bta_selquad_batched call per step in `precision` (every launch covers
    all points of a wave), against per-point single solves of the same points
    on the same GPU in FP64 and in `precision`.  Returns the measurement."""
    import torch

    from paper_2601_04904_gb300 import qsi

    n, b, a, nE = 32, 256, 128, points
    prec = qsi.PRECISIONS[precision]
    stream = torch.cuda.Stream()  # a capturable stream: the batch runs as one CUDA graph
    torch.cuda.set_stream(stream)
    # the library's autotuner (points per wave, tensor-core launch knobs): tuned
    # during the first warm-up call, cached in this file for later runs
    tune_cache = os.environ.setdefault("QSI_AUTOTUNE_CACHE", os.path.join("/tmp", "qsi_autotune_cache.txt"))
    ctx = qsi.Context(0, stream=stream)
    H = qsi.to_device(inputs.hamiltonian(n, b, a))
    E, g = inputs.energy_grid(nE)
    gen = torch.Generator(device="cuda").manual_seed(inputs.BASE_SEED + 2)
    Bst = device_bta_antihermitian(torch, n, b, a, gen, lead=(nE,))
    GR = qsi.batched_zeros(nE, n, b, a)
    GL = qsi.batched_zeros(nE, n, b, a)
    for _ in range(warmup):
        ctx.selquad_batched(H, E, 1e-3, g, Bst, GR, GL, prec)
    ctx.synchronize()
    tuned = ctx.batched_config()
    ctx.stats_reset(False)
    g0 = ctx.stats()["graph_launches"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            ctx.selquad_batched(H, E, 1e-3, g, Bst, GR, GL, prec)
        e1.record(stream)
        torch.cuda.synchronize()
    ctx.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = ctx.stats()
    graph_launches = st["graph_launches"] - g0
    # one more (untimed) batch with every launch bracketed by events: device
    # time per kernel family, as shares of that batch's time (launched
    # directly: a graph replay cannot bracket its kernels)
    ctx.stats_reset(True)
    os.environ["QSI_NO_GRAPH"] = "1"
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    ctx.selquad_batched(H, E, 1e-3, g, Bst, GR, GL, prec)
    t1e.record(stream)
    ctx.synchronize()
    del os.environ["QSI_NO_GRAPH"]
    stk, ms_k = ctx.stats(), t0e.elapsed_time(t1e)
    shares = {k: stk[v] / ms_k for k, v in (("zinv_panel", "panel_ms"), ("fp32_gauss_jordan", "panel32_ms"),
                                            ("zgemm_fp64", "gemm_ms"), ("tc_mma", "tc_ms"), ("tc_aux", "tc_aux_ms"),
                                            ("tc_aux_exp", "tc_exp_ms"), ("tc_aux_conv", "tc_conv_ms"),
                                            ("tc_aux_crt", "tc_crt_ms"))}
    shares["zinv_other"] = (stk["inv_ms"] - stk["panel_ms"] - stk["panel32_ms"]) / ms_k
    # per-point single solves of the first points (same GPU), FP64 and `precision`
    k_single = min(8, nE)
    Bk = {key: Bst[key][0].contiguous() for key in qsi.KEYS}
    GRk, GLk = qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a)

    def singles(p):
        A0 = ctx.assemble(H, float(E[0]), 1e-3, float(g[0]))
        f = ctx.factor(A0, Bk, p)
        ctx.selquad(f, GRk, GLk)
        f.close()
        ctx.synchronize()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(k_single):
            Ak = ctx.assemble(H, float(E[k]), 1e-3, float(g[k]))
            f = ctx.factor(Ak, Bk, p)
            ctx.selquad(f, GRk, GLk)
            f.close()
        ctx.synchronize()
        return k_single / (time.perf_counter() - t0)

    single = singles(qsi.FP64)
    single_tc = singles(prec) if prec != qsi.FP64 else single
    flops = nE * metrics.flops_selquad(n, b, a)
    out = {
        "value": nE / (ms / 1e3), "unit": UNIT, "ms_per_batch": ms, "steps": steps, "warmup": warmup,
        "workload": f"bta_n{n}_b{b}_a{a}_x{nE}E", "points": nE, "precision": precision,
        "call": "qsi_bta_selquad_batched (every wave in one CUDA graph, replayed)",
        "schedule": {"points_per_wave": tuned["wave"], "crt_outputs_per_thread": tuned["crt_v"] or 2,
                     "moduli_per_cta_overhead_ktiles": tuned["cta_fill"] if tuned["cta_fill"] >= 0 else 6.0,
                     "autotuned": tuned["tuned"], "tuning_cache": tune_cache,
                     "graph_launches_per_batch": graph_launches / steps},
        "l2": "inputs larger than L2",
        "tflops_algorithmic": flops / (ms / 1e3) / 1e12, "gpu_launches_per_batch": st["launches"] / steps,
        "kernel_shares": shares,
        "single_solve_points_per_s_fp64": single, "batched_over_single_fp64": nE / (ms / 1e3) / single,
        "single_solve_points_per_s_" + precision: single_tc,
        "batched_over_single_" + precision: nE / (ms / 1e3) / single_tc,
        "clocks": clk.summary()}
    ctx.close()
    del H, Bst, GR, GL
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    d = measure_batched(args.points, args.steps, args.warmup, args.precision)
    print(json.dumps({"metric": METRIC, "mode": "batched", "n_gpus": 1, "higher_is_better": True,
                      "dtype": "f64", "data": "synthetic", **d}))


def run_partitioned(args):
    """Latency of one solve (call to completion) of small-b shapes, where the
    sequential depth of the sweeps rather than the arithmetic sets the time:
    the plain solve (qsi_bta_solve, graph replay) against the partitioned
    solve (qsi_bta_solve_partitioned) at several partition counts, with the
    partitioned result's max block difference to the plain one."""
    import torch

    from paper_2601_04904_gb300 import qsi

    prec = qsi.PRECISIONS[args.precision]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = qsi.Context(0, stream=stream)
    shapes = [(8, 32, 16, (2, 3, 4)), (128, 128, 0, (2, 4, 8, 16, 32)), (64, 128, 128, (2, 4, 8, 16)),
              (128, 256, 128, (4, 8, 16))]
    if args.part_shape:
        n_, b_, a_ = (int(x) for x in args.part_shape.split(","))
        shapes = [(n_, b_, a_, tuple(int(x) for x in (args.part_p or "0").split(",")))]
    rows = []
    reps = args.steps if args.part_only else max(args.steps, 5)

    def lat(fn):
        for _ in range(args.warmup if args.part_only else max(args.warmup, 3)):
            fn()
        stream.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            stream.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(ts)

    for n, b, a, Ps in shapes:
        gen = torch.Generator(device="cuda").manual_seed(inputs.BASE_SEED + 3000 + n + b + a)
        Ad = device_bta_hermitian(torch, n, b, a, gen, 1.0 / np.sqrt(b))
        Bd = device_bta_antihermitian(torch, n, b, a, gen)
        ctx.assemble(Ad, 0.3, 1e-3, 0.5, out=Ad)
        GR, GX = qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)]
        torch.cuda.synchronize()
        plain_ms, ref = None, None
        if not args.part_only:
            plain_ms = lat(lambda: ctx.solve(Ad, [Bd], GR, GX, prec))
            ref = ({k: v.clone() for k, v in GR.items()}, {k: v.clone() for k, v in GX[0].items()})
        row = {"shape": [n, b, a], "plain_ms": plain_ms, "partitioned": []}
        for P in Ps:
            if 2 * P - 1 > n:
                continue
            PR, PX = qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)]
            l0 = ctx.stats()["launches"]
            ms = lat(lambda: ctx.solve_partitioned(Ad, [Bd], P, PR, PX, prec))
            ent = {"P": P, "ms": ms, "launches_per_call": (ctx.stats()["launches"] - l0) / max(1, reps + args.warmup)}
            if ref is not None:
                ent["speedup"] = plain_ms / ms
                ent["max_block_diff_vs_plain"] = max(
                    metrics.max_block_rel_err(qsi.to_host(PR), qsi.to_host(ref[0])),
                    metrics.max_block_rel_err(qsi.to_host(PX[0]), qsi.to_host(ref[1])))
            row["partitioned"].append(ent)
        if not args.part_only:
            # partitions = 0 (the twisted split) and -1 (round(sqrt(n)) general
            # partitions if the device conditioning estimate of their pivots
            # allows, else the twisted split)
            QR, QX = qsi.device_zeros(n, b, a), [qsi.device_zeros(n, b, a)]
            ms0 = lat(lambda: ctx.solve_partitioned(Ad, [Bd], 0, QR, QX, prec))
            d0 = max(metrics.max_block_rel_err(qsi.to_host(QR), qsi.to_host(ref[0])),
                     metrics.max_block_rel_err(qsi.to_host(QX[0]), qsi.to_host(ref[1])))
            row["twisted"] = {"ms": ms0, "vs_plain": plain_ms / ms0, "max_block_diff_vs_plain": d0}
            f0 = ctx.stats()["partition_fallbacks"]
            ms = lat(lambda: ctx.solve_partitioned(Ad, [Bd], -1, QR, QX, prec))
            st = ctx.stats()
            row["checked"] = {"ms": ms, "kappa_F": st["partition_kappa"],
                              "chosen": "twisted" if st["partition_fallbacks"] > f0 else "general",
                              "vs_plain": plain_ms / ms}
        rows.append(row)
    # a speed-up counts only where the partitioned result is within 1e-10 of the plain one
    best = {f"{r['shape'][0]}x{r['shape'][1]}x{r['shape'][2]}": max(
        (p["speedup"] for p in r["partitioned"] if p.get("max_block_diff_vs_plain", 1.0) < 1e-10), default=None)
        for r in rows}
    print(json.dumps({"metric": "single-solve latency, plain vs partitioned", "mode": "partitioned",
                      "unit": "ms", "higher_is_better": False, "n_gpus": 1, "precision": args.precision,
                      "dtype": "f64", "data": "synthetic", "reps": reps, "rows": rows,
                      "best_speedup_within_1e-10": best,
                      "config": {"workload": "small-b shapes (c0 and small c4 requests)", "eta": 1e-3,
                                 "timing": "host wall clock per call to stream completion, median"}}))
    ctx.close()


def measure_serve(requests=200, slots=4, serve_mix="fp64_emu,mixed"):
    """Poisson request stream (seeded) of SI+SQ solves of mixed sizes through the
    continuous-batching server: saturated throughput, then arrivals at 0.8x that
    rate (timed, with its clock record).  Returns the measurement."""
    import torch

    from paper_2601_04904_gb300 import qsi

    rng = np.random.default_rng(inputs.BASE_SEED + 2)
    R = requests
    p_a, p_b = serve_mix.split(",")
    shapes = [(int(rng.integers(16, 129)), int(rng.choice([128, 256, 512, 768])), int(rng.choice([0, 128, 256, 512])),
               p_a if rng.random() < 0.5 else p_b) for _ in range(2000)][:R]
    gap = rng.exponential(1.0, size=2000)[:R]

    def make(k):
        n, b, a, p = shapes[k]
        gen = torch.Generator(device="cuda").manual_seed(inputs.BASE_SEED + 1000 + k)
        Hd = device_bta_hermitian(torch, n, b, a, gen, 1.0 / np.sqrt(b))
        Bd = device_bta_antihermitian(torch, n, b, a, gen)
        ctx_tmp.assemble(Hd, 0.3, 1e-3, 0.5, out=Hd)  # A in place of H
        ctx_tmp.synchronize()
        return Hd, Bd, qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a), qsi.PRECISIONS[p]

    ctx_tmp = qsi.Context(0)
    flops = [metrics.flops_selquad(n, b, a) for n, b, a, _ in shapes]
    # device memory split between the clients' request buffers (A, B, G^R, G^<
    # of every submitted, unfinished request) and the server's admissions
    # (factor + sweep temporaries): a client holds a new request back until
    # its buffers fit, as a caller with finite memory would
    free0 = torch.cuda.mem_get_info()[0]
    client_budget, server_budget = int(free0 * 0.42), int(free0 * 0.45)
    req_bytes = lambda n, b, a: 4 * 16 * ((3 * n - 2) * b * b + 2 * n * b * a + a * a)

    def run_stream(rate):
        srv = qsi.Server(0, slots=slots, hbm_budget=server_budget)
        tickets, results, live = [], {}, {}
        held = [0]

        def drain():
            for t in list(live):
                r = srv.poll(t)
                if r is not None:
                    results[t] = r
                    held[0] -= live.pop(t)[-1]

        t_start = time.perf_counter()
        t_next = t_start
        for k in range(R):
            if rate:
                t_next += gap[k] / rate
                while time.perf_counter() < t_next:
                    drain()
                    time.sleep(0.0005)
            need = req_bytes(*shapes[k][:3])
            while live and held[0] + need > client_budget:
                drain()
                time.sleep(0.0005)
            if torch.cuda.memory_reserved() + need > client_budget:
                torch.cuda.empty_cache()
            Ad, Bd, GR, GL, p = make(k)
            t = srv.submit(Ad, Bd, GR, GL, p)
            tickets.append(t)
            live[t] = (Ad, Bd, GR, GL, need)
            held[0] += need
        while live:
            drain()
            time.sleep(0.0005)
        wall = time.perf_counter() - t_start
        srv.close()
        lat = sorted(results[t]["latency_ms"] for t in tickets)
        ok = all(results[t]["status"] == qsi.OK for t in tickets)
        return wall, lat, ok

    wall_sat, _, ok1 = run_stream(None)
    sat = R / wall_sat
    with ClockSampler(0) as clk:
        wall, lat, ok2 = run_stream(0.8 * sat)
    pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    out = {
        "value": R / wall, "unit": UNIT, "saturated_points_per_s": sat, "arrival_rate": 0.8 * sat,
        "p50_latency_ms": pct(0.5), "p99_latency_ms": pct(0.99), "requests": R,
        "requests_note": f"the first {R} of the seeded 2000-request stream" if R < 2000 else "the whole stream",
        "all_ok": ok1 and ok2, "slots": slots, "wall_s": wall,
        "tflops_algorithmic": sum(flops) / wall / 1e12,
        "workload": "serve_poisson_2000" if R >= 2000 else f"serve_poisson_2000_prefix{R}",
        "mix": "n U{16..128}, b in {128,256,512,768}, a in {0,128,256,512}, " + f"{p_a} / {p_b} 50/50",
        "rate": "0.8 x measured saturated throughput",
        "memory": "request buffers <= 0.42 x free HBM (a client waits for completions), "
                  "server admissions <= 0.45 x free HBM",
        "clocks": clk.summary()}
    ctx_tmp.close()
    torch.cuda.empty_cache()
    return out


def run_serve(args):
    d = measure_serve(args.requests, args.slots, args.serve_mix)
    print(json.dumps({"metric": METRIC, "mode": "serve", "n_gpus": 1, "higher_is_better": True, "dtype": "f64",
                      "data": "synthetic", **d}))


def fmax_nan(a: float, b: float) -> float:
    """max(a, b) with a NaN taken as inf (Python's max would drop it)."""
    return float("inf") if not (np.isfinite(a) and np.isfinite(b)) else max(a, b)


def block_err_device(torch, X: dict, R: dict, keys) -> float:
    """Max over pattern blocks of ||X - R||_F / ||R||_F (absolute below 1e-300), on the device;
    inf when any block's error is not finite."""
    w = 0.0
    with torch.no_grad():
        for k in keys:
            if R[k].numel() == 0:
                continue
            xs, rs = X[k].reshape(-1, *X[k].shape[-2:]), R[k].reshape(-1, *R[k].shape[-2:])
            num = torch.linalg.matrix_norm(xs - rs)
            den = torch.linalg.matrix_norm(rs)
            e = float(torch.where(den >= 1e-300, num / den.clamp_min(1e-300), num).max())
            if not np.isfinite(e):  # max() would drop a NaN
                return float("inf")
            w = max(w, e)
    return w


def measure_fp64_peak():
    """FP64 throughput of the library GEMMs on this GPU (burst): cuBLAS DGEMM
    (torch.matmul float64, 4096^3) and ZGEMM (complex128, 2048^3, 8 real flop
    per complex multiply-add), best of 5 after a warm-up."""
    import torch

    out = {}
    for name, dt, N, fl in (("dgemm", torch.float64, 4096, 2.0), ("zgemm", torch.complex128, 2048, 8.0)):
        a = torch.randn(N, N, dtype=dt, device="cuda")
        b_ = torch.randn(N, N, dtype=dt, device="cuda")
        c = torch.matmul(a, b_)
        torch.cuda.synchronize()
        best = None
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b_, out=c)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[name + "_tflops"] = fl * N ** 3 / (best / 1e3) / 1e12
        del a, b_, c
    out["peak_tflops"] = max(out["dgemm_tflops"], out["zgemm_tflops"])
    out["how"] = ("cuBLAS through torch.matmul: DGEMM 4096^3 (2 flop per multiply-add), ZGEMM 2048^3 "
                  "(8 real flop per complex multiply-add); best of 5 CUDA-event timings after a warm-up")
    out["derived_dfma_tflops"] = FP64_PEAK_TFLOPS
    torch.cuda.empty_cache()
    return out


def measure_c3(steps=3, warmup=2):
    """The precision workload (n=128, b=1024, a=512; A and B generated on the
    device with the synthetic recipe) in QSI_MIXED: ms per solve, and every
    output block's relative error against the FP64-accurate tensor-core solve
    of the same matrices on the same GPU (FP64_EMU, itself within 1e-10 of the
    oracle), with the FP64_EMU and 3-term-split (QSI_SPLIT3) timings beside it."""
    import torch

    from paper_2601_04904_gb300 import qsi

    n, b, a = 128, 1024, 512
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = qsi.Context(0, stream=stream)
    gen = torch.Generator(device="cuda").manual_seed(inputs.BASE_SEED + 6000)
    A = device_bta_hermitian(torch, n, b, a, gen, 1.0 / np.sqrt(b))
    ctx.assemble(A, 0.3, 1e-3, 0.5, out=A)
    B = device_bta_antihermitian(torch, n, b, a, gen)
    GR, GL = qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a)
    torch.cuda.synchronize()

    def timed(prec, k, w):
        for _ in range(w):
            ctx.solve(A, [B], GR, [GL], prec)
        ctx.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            ctx.solve(A, [B], GR, [GL], prec)
        e1.record(stream)
        ctx.synchronize()
        return e0.elapsed_time(e1) / k

    with ClockSampler(0) as clk:
        ms_emu = timed(qsi.FP64_EMU, 2, 1)
    RR = {k: v.clone() for k, v in GR.items()}
    RL = {k: v.clone() for k, v in GL.items()}
    with ClockSampler(0) as clk_mixed:
        ms_mixed = timed(qsi.MIXED, steps, warmup)
    err_mixed = {"G^R": block_err_device(torch, GR, RR, qsi.KEYS), "G^<": block_err_device(torch, GL, RL, qsi.KEYS)}
    ms_split = timed(qsi.SPLIT3, 1, 1)
    err_split = {"G^R": block_err_device(torch, GR, RR, qsi.KEYS), "G^<": block_err_device(torch, GL, RL, qsi.KEYS)}
    flops = metrics.flops_selquad(n, b, a)
    nm = int(os.environ.get("QSI_MIXED_MODULI", MODULI["mixed"]))
    out = {"workload": "bta_n128_b1024_a512", "precision": "mixed", "moduli": nm, "ms_per_solve": ms_mixed,
           "value": 1e3 / ms_mixed, "unit": UNIT, "steps": steps, "warmup": warmup,
           "tflops_algorithmic": flops / (ms_mixed / 1e3) / 1e12,
           "max_block_rel_err_vs_fp64_emu": err_mixed, "tolerance": 1e-6,
           "meets_tolerance": max(err_mixed.values()) < 1e-6,
           "fp64_emu_ms_per_solve": ms_emu, "speedup_over_fp64_emu": ms_emu / ms_mixed,
           "split3_ms_per_solve": ms_split, "split3_max_block_rel_err_vs_fp64_emu": err_split,
           "call": "qsi_bta_solve (graph-cached on its stream)", "clocks": clk_mixed.summary(),
           "clocks_fp64_emu": clk.summary()}
    ctx.close()
    del A, B, GR, GL, RR, RL
    torch.cuda.empty_cache()
    return out


# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# the kernels the roofline may name, keyed (kernel, precision), from one capture
# of the kernel as it is now (cold caches: ncu flushes them between passes);
# absent = not captured since the kernel last changed.
TRAFFIC_PER_LAUNCH = {("tc_mma_kernel", "fp64_emu"): 1.188e8}
TRAFFIC_SOURCE = {("tc_mma_kernel", "fp64_emu"):
                  "ncu dram__bytes_read.sum + dram__bytes_write.sum, average over the 121 tc_mma launches of one "
                  "step of the same block sizes on 8 blocks (caches flushed; "
                  "profiles/tc_mma_kernel_dram_bta_n8_b512_a256_fp64emu.md)"}


def measured_peaks():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def roofline_of(st, ms_total, precision, wl, fp64_peak=None):
    """Roofline of the kernel with the largest summed device time in one step
    (every launch bracketed by CUDA events).  achieved = the method's
    algorithmic flops that the kernel carries (8 per complex multiply-add of the
    work model) / its summed event time.

    Tensor-core products: the block products of the sweeps (the work model
    minus the block inversions; the Newton refinement's products are extra work
    of the inversion, not counted) against the measured sustained BF16 peak, the
    pipe they run on; pipe_util beside it counts the BF16 work the emulation
    executes for them (4 real products per complex product and modulus, 17
    moduli for the FP64-accurate products, 13 for the mixed ones, 6 split pairs
    for the 3-term split; Newton products included).  IEEE FP64 kernels: against
    the measured cuBLAS FP64 GEMM peak of this GPU, else the derived DFMA peak."""
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained")
    n, b, a = wl["n"], wl["b"], wl["a"]
    prod_flops = metrics.flops_products(n, b, a)
    if fp64_peak:
        p64, p64_src = fp64_peak, "of measured: cuBLAS DGEMM/ZGEMM on this GPU (bench fp64_peak)"
    else:
        p64, p64_src = FP64_PEAK_TFLOPS, "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz"
    cands = []
    if st["panel_ms"] > 0:
        cands.append(dict(kernel="zinv_panel_kernel", what="cluster-of-8 Gauss-Jordan panel elimination, DFMA",
                          ms=st["panel_ms"], launches=st["panel_launches"], flops=st["panel_flops"], bound="alu",
                          peak=p64, peak_source=p64_src))
    if st["panel32_ms"] > 0:
        # blocks up to 512: one cluster launch per block; above (or QSI_GJ_PANELS) panels of columns
        cluster = b <= 512 and not os.environ.get("QSI_GJ_PANELS")
        cands.append(dict(kernel="gj32_cluster_kernel" if cluster else "panel32_kernel",
                          what=("FP32 Gauss-Jordan of the refined inversion, one 16-CTA cluster per block, FFMA"
                                if cluster else "FP32 Gauss-Jordan panel of the refined inversion, FFMA"),
                          ms=st["panel32_ms"], launches=st["panel32_launches"], flops=st["panel32_flops"], bound="alu",
                          peak=FP32_PEAK_TFLOPS, peak_source="derived: 152 SMs x 256 FP32 flop/clk x 2.07 GHz"))
    if st["gemm_ms"] > 0:
        cands.append(dict(kernel="zgemm_fp64_kernel", what="grouped complex GEMM, DFMA", ms=st["gemm_ms"],
                          launches=st["gemm_launches"], flops=st["gemm_flops"], bound="alu", peak=p64,
                          peak_source=p64_src))
    if st["tc_ms"] > 0 and bf16:
        nm = int(os.environ.get("QSI_MIXED_MODULI", MODULI["mixed"])) if precision == "mixed" else 17
        sweep = min(prod_flops, st["tc_flops"])
        newton = st["tc_flops"] - sweep
        if precision == "split3":
            bf16_work = 6.0 * sweep + 17.0 * newton
        else:
            bf16_work = nm * sweep + 17.0 * newton
        cands.append(dict(kernel="tc_mma_kernel", what="tcgen05 BF16 products of the FP64-emulated block products",
                          ms=st["tc_ms"], launches=st["tc_launches"], flops=sweep, bound="tensor",
                          peak=bf16, peak_source="of measured: bf16_tflops_sustained in MEASURED_PEAKS.json",
                          pipe_util=bf16_work / (st["tc_ms"] / 1e3) / 1e12 / bf16,
                          newton_flops=newton))
    if not cands:
        return None
    k = max(cands, key=lambda c: c["ms"])
    achieved = k["flops"] / (k["ms"] / 1e3) / 1e12
    others = [{"kernel": c["kernel"], "bound": c["bound"], "share_of_step": c["ms"] / ms_total if ms_total else None,
               "frac": (c["flops"] / (c["ms"] / 1e3) / 1e12) / c["peak"] if c["peak"] else None}
              for c in sorted(cands, key=lambda c: -c["ms"])]
    out = {"kernel": k["kernel"] + " (" + k["what"] + ")", "bound": k["bound"], "achieved": achieved,
           "peak": k["peak"], "unit": "TFLOP/s", "frac": achieved / k["peak"],
           "traffic": TRAFFIC_PER_LAUNCH.get((k["kernel"], precision)), "peak_source": k["peak_source"],
           "launches": int(k["launches"]), "avg_launch_ms": k["ms"] / max(1, k["launches"]),
           "share_of_step": k["ms"] / ms_total if ms_total else None, "all_kernels": others,
           "achieved_counts": "algorithmic flops of the method carried by this kernel (work model, 8 per "
                              "complex multiply-add)"}
    if "pipe_util" in k:
        out["pipe_util"] = k["pipe_util"]
        out["newton_flops_excluded"] = k["newton_flops"]
    if out["traffic"] is not None:
        out["traffic_source"] = TRAFFIC_SOURCE.get((k["kernel"], precision))
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "partitioned":
        return run_partitioned(args)
    if args.mode == "extras":
        return run_extras(args)
    import torch

    from paper_2601_04904_gb300 import qsi

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.workload]
    n, b, a = wl["n"], wl["b"], wl["a"]
    prec = qsi.PRECISIONS[args.precision]
    E, eta, gamma = energy_of(rank), 1e-3, 0.5

    h_np = inputs.hamiltonian(n, b, a)
    bl_np = inputs.lesser_rhs(n, b, a, seed=replicas.rhs_seed(rank))
    # a non-default stream: qsi_bta_solve captures the solve once as a CUDA
    # graph and replays it (same buffers every step)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # torch's own work (buffers, checks) is ordered with the solves
    H = qsi.to_device(h_np)
    B = qsi.to_device(bl_np)
    GR = qsi.device_zeros(n, b, a)
    GL = qsi.device_zeros(n, b, a)
    torch.cuda.synchronize()
    ctx = qsi.Context(local, stream=stream)
    A = ctx.assemble(H, E, eta, gamma)
    ctx.synchronize()
    del H

    def step():
        ctx.solve(A, [B], GR, [GL], prec)

    for _ in range(args.warmup):
        step()
    ctx.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # timed steps: launch counters only (no per-launch events inside the timed region)
    ctx.stats_reset(time_kernels=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]  # step boundaries
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        ev[0].record(stream)
        for k in range(args.steps):
            step()
            ev[k + 1].record(stream)
        e1.record(stream)
        barrier()
    ctx.synchronize()
    ms_total = replicas.max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    per_step = np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)])
    launches_timed = ctx.stats()["launches"]
    ms_step = ms_total / args.steps
    value = replicas.job_rate(world, args.steps, ms_total / 1e3)
    # end to end through the C ABI from pinned host buffers, right after the
    # timed region (before the longer IEEE-FP64 comparison run heats the GPU)
    def host_e2e(path):
        """The metric through qsi_bta_selquad_host from pinned host buffers:
        per call the H2D of A and B, the solve and the D2H of G^R and G^<."""
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        A_h = {k: A[k].cpu().pin_memory() for k in qsi.KEYS}
        B_h = {k: pin(bl_np[k]) for k in qsi.KEYS}
        GR_h = {k: torch.empty_like(A_h[k]).pin_memory() for k in qsi.KEYS}
        GL_h = {k: torch.empty_like(A_h[k]).pin_memory() for k in qsi.KEYS}
        for _ in range(3):  # first call solves and captures, the others replay
            ctx.selquad_host(A_h, B_h, GR_h, GL_h, prec)
        k_e2e = 6
        if dist is not None:
            dist.barrier()
        with ClockSampler(local) as clk_e2e:
            t0 = time.perf_counter()
            calls = []
            for _ in range(k_e2e):
                tc = time.perf_counter()
                ctx.selquad_host(A_h, B_h, GR_h, GL_h, prec)
                calls.append((time.perf_counter() - tc) * 1e3)
            dt = replicas.max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        bytes_in = 2 * metrics.bytes_bta(n, b, a)
        res = {"value": replicas.job_rate(world, k_e2e, dt), "unit": UNIT, "h2d_bytes_per_step": bytes_in,
               "d2h_bytes_per_step": bytes_in, "steps": k_e2e, "call_ms": calls,
               "median_call_ms": statistics.median(calls), "clocks": clk_e2e.summary(), "path": path}
        return res, GR_h, GL_h

    # end to end through the C ABI from pinned host buffers, right after the
    # timed region (before the longer IEEE-FP64 comparison run heats the GPU)
    e2e = None
    if not args.no_e2e:
        e2e, _, _ = host_e2e("qsi_bta_selquad_host (pinned host A, B -> device -> host G^R, G^<)")

    # one more (untimed) step with every launch bracketed by events: device time
    # per kernel family (shares of that step, roofline of the dominant kernel)
    # (a graph replay cannot bracket its kernels: this step launches directly)
    ctx.stats_reset(time_kernels=True)
    k0e, k1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0e.record(stream)
    f = ctx.factor(A, B, prec)
    ctx.selquad(f, GR, GL)
    f.close()
    k1e.record(stream)
    ctx.synchronize()
    st = ctx.stats()
    ms_kstep = k0e.elapsed_time(k1e)

    # verification on sampled blocks: (A G^R)_ii = I and (A G^<)_ii = (B G^R^H)_ii
    chk = {}
    with torch.no_grad():
        worst_r, worst_l = 0.0, 0.0
        for i in sorted({0, n // 2, n - 1}):
            ag = A["diag"][i] @ GR["diag"][i] + A["arrow_r"][i] @ GR["arrow_b"][i]
            ax = A["diag"][i] @ GL["diag"][i] + A["arrow_r"][i] @ GL["arrow_b"][i]
            bg = B["diag"][i] @ GR["diag"][i].conj().T + B["arrow_r"][i] @ GR["arrow_r"][i].conj().T
            if i > 0:
                ag += A["lower"][i - 1] @ GR["upper"][i - 1]
                ax += A["lower"][i - 1] @ GL["upper"][i - 1]
                bg += B["lower"][i - 1] @ GR["lower"][i - 1].conj().T
            if i < n - 1:
                ag += A["upper"][i] @ GR["lower"][i]
                ax += A["upper"][i] @ GL["lower"][i]
                bg += B["upper"][i] @ GR["upper"][i].conj().T
            eye = torch.eye(b, dtype=ag.dtype, device=ag.device)
            worst_r = fmax_nan(worst_r, float(torch.linalg.norm(ag - eye) / b ** 0.5))
            worst_l = fmax_nan(worst_l, float(torch.linalg.norm(ax - bg) / torch.linalg.norm(bg)))
        chk = {"blocks": sorted({0, n // 2, n - 1}), "AG_minus_I_rel": worst_r, "AX_minus_BGH_rel": worst_l}

    # FP64 peak of this GPU (cuBLAS DGEMM / ZGEMM): the FP64 denominator
    fp64_peak = measure_fp64_peak() if world == 1 else None
    p64 = fp64_peak["peak_tflops"] if fp64_peak else FP64_PEAK_TFLOPS

    # the same matrices in IEEE FP64 on the same GPU: throughput beside the
    # timed precision, and the per-block error of the timed result against it
    fp64_cmp = None
    if args.precision != "fp64" and not args.no_fp64_compare and world == 1:
        if not args.ref_precision:
            args.ref_precision = "fp64"
        wR, wL = qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a)
        torch.cuda.synchronize()
        for _ in range(1):
            f = ctx.factor(A, B, qsi.FP64)
            ctx.selquad(f, wR, wL)
            f.close()
        ctx.synchronize()
        k64 = 2
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tR, tL = qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a)
        torch.cuda.synchronize()
        c0.record(stream)
        for _ in range(k64):
            f = ctx.factor(A, B, qsi.FP64)
            ctx.selquad(f, tR, tL)
            f.close()
        c1.record(stream)
        ctx.synchronize()
        ms64 = c0.elapsed_time(c1) / k64
        del tR, tL
        fp64_cmp = {"value": 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64, "steps": k64,
                    "pct_fp64_peak": 100.0 * metrics.flops_selquad(n, b, a) / (ms64 / 1e3) / 1e12 / p64,
                    "fp64_peak_tflops": p64,
                    "fp64_peak_source": "measured cuBLAS FP64 GEMM (fp64_peak)" if fp64_peak else "derived",
                    "speedup_of_timed_precision": ms64 / ms_step}

    # the same workload with QSI_ASSUME_ANTIHERMITIAN_B (B is anti-Hermitian
    # here, as Sigma^< is): mirrored blocks instead of a fifth of the products
    ah = None
    if world == 1 and not args.no_suite:
        ctx.set_flags(qsi.ASSUME_ANTIHERMITIAN_B)
        hR, hL = qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a)
        torch.cuda.synchronize()
        for _ in range(2):  # solve + capture, replay
            ctx.solve(A, [B], hR, [hL], prec)
        ctx.synchronize()
        k_ah = 5
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk_ah:
            torch.cuda.synchronize()
            h0.record(stream)
            for _ in range(k_ah):
                ctx.solve(A, [B], hR, [hL], prec)
            h1.record(stream)
            ctx.synchronize()
        ms_ah = h0.elapsed_time(h1) / k_ah
        ctx.set_flags(0)
        fl_ah = metrics.flops_selquad(n, b, a, antihermitian=True)
        ah = {"value": 1e3 / ms_ah, "unit": UNIT, "ms_per_step": ms_ah, "steps": k_ah,
              "speedup_over_unflagged": ms_step / ms_ah,
              "tflops_algorithmic": fl_ah / (ms_ah / 1e3) / 1e12,
              "flops_per_step": fl_ah, "flops_per_step_unflagged": metrics.flops_selquad(n, b, a),
              "max_block_rel_err_vs_unflagged": {"G^R": block_err_device(torch, hR, GR, qsi.KEYS),
                                                 "G^<": block_err_device(torch, hL, GL, qsi.KEYS)},
              "call": "qsi_set_flags(QSI_ASSUME_ANTIHERMITIAN_B) + qsi_bta_solve (graph-cached)",
              "clocks": clk_ah.summary()}
        del hR, hL

    # the same workload through the twisted two-way split (qsi_bta_solve_partitioned
    # with partitions = 0: the top half from block 0 down, the bottom half from
    # block n-1 up; the plain sweep's pivots), device-resident, graph-cached
    tw = None
    if world == 1 and not args.no_suite and n >= 3:
        wR, wL = qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a)
        torch.cuda.synchronize()
        for _ in range(2):  # solve + capture, replay
            ctx.solve_partitioned(A, [B], 0, wR, [wL], prec)
        ctx.synchronize()
        k_tw = 5
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk_tw:
            torch.cuda.synchronize()
            w0.record(stream)
            for _ in range(k_tw):
                ctx.solve_partitioned(A, [B], 0, wR, [wL], prec)
            w1.record(stream)
            ctx.synchronize()
        ms_tw = w0.elapsed_time(w1) / k_tw
        tw = {"value": 1e3 / ms_tw, "unit": UNIT, "ms_per_step": ms_tw, "steps": k_tw,
              "speedup_over_plain": ms_step / ms_tw,
              "max_block_rel_err_vs_plain": {"G^R": block_err_device(torch, wR, GR, qsi.KEYS),
                                             "G^<": block_err_device(torch, wL, GL, qsi.KEYS)},
              "call": "qsi_bta_solve_partitioned(partitions = 0: the twisted two-way split, graph-cached)",
              "clocks": clk_tw.summary()}
        del wR, wL
        if not args.no_e2e:
            # end to end through the twisted split: partition blocks copied
            # straight into their slots and back, beside the sweeps
            ctx.set_flags(qsi.TWISTED_SPLIT)
            tw_e2e, hR, hL = host_e2e("qsi_set_flags(QSI_TWISTED_SPLIT) + qsi_bta_selquad_host (pinned host buffers)")
            ctx.set_flags(0)
            tw_e2e["max_block_rel_err_vs_plain"] = {
                "G^R": block_err_device(torch, {k: v.cuda() for k, v in hR.items()}, GR, qsi.KEYS),
                "G^<": block_err_device(torch, {k: v.cuda() for k, v in hL.items()}, GL, qsi.KEYS)}
            tw["e2e"] = tw_e2e
            del hR, hL

    if args.ref_precision:
        # per-block relative Frobenius error against a reference solve on the same GPU
        rR, rL = qsi.device_zeros(n, b, a), qsi.device_zeros(n, b, a)
        torch.cuda.synchronize()  # zero-filled on torch's stream, written on the context's
        f = ctx.factor(A, B, qsi.PRECISIONS[args.ref_precision])
        ctx.selquad(f, rR, rL)
        f.close()
        ctx.synchronize()
        worst = {name: block_err_device(torch, X, R, qsi.KEYS) for name, X, R in (("G^R", GR, rR), ("G^<", GL, rL))}
        chk["max_block_rel_err_vs_" + args.ref_precision] = worst
        del rR, rL
    tc_achieved = st["tc_flops"] / (st["tc_ms"] / 1e3) / 1e12 if st["tc_ms"] > 0 else None
    flops_step = metrics.flops_selquad(n, b, a)
    roof = roofline_of(st, ms_kstep, args.precision, wl, p64 if fp64_peak else None)
    tflops_alg = flops_step / (ms_step / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(args, wl),
        "parallelism": "replicas" if world > 1 else "single",
        "tflops_algorithmic": tflops_alg,
        "gpu_launches": int(launches_timed),
        "roofline": roof,
        "kernel_shares": {k: v / ms_kstep for k, v in (("zinv_panel", st["panel_ms"]), ("fp32_gauss_jordan", st["panel32_ms"]),
                                                       ("zgemm_fp64", st["gemm_ms"]), ("tc_mma", st["tc_ms"]),
                                                       ("tc_aux", st["tc_aux_ms"]),
                                                       ("tc_aux_exp", st["tc_exp_ms"]),
                                                       ("tc_aux_conv", st["tc_conv_ms"]),
                                                       ("tc_aux_crt", st["tc_crt_ms"]),
                                                       ("zinv_other",
                                                        st["inv_ms"] - st["panel_ms"] - st["panel32_ms"]))},
        "step_ms": {"median": float(np.median(per_step)), "mean": float(per_step.mean()),
                    "ci95_half_width": (float(1.96 * per_step.std(ddof=1) / np.sqrt(len(per_step)))
                                        if len(per_step) > 1 else None), "n": int(len(per_step))},
        "kernel_times_step_ms": ms_kstep,
        "inversion_ms_per_step": st["inv_ms"],
        "tensor_core_products": {"launches": int(st["tc_launches"]), "ms_per_step": st["tc_ms"],
                                 "fp64_equiv_tflops": tc_achieved},
        "check": chk,
        "ieee_fp64_same_gpu": fp64_cmp,
        "fp64_peak": fp64_peak,
        "antihermitian_b": ah,
        "twisted": tw,
        "clocks": clk.summary(),
    }
    if args.precision == "fp64":
        out["pct_fp64_peak"] = 100.0 * tflops_alg / p64
    else:
        # tensor-core precisions: the method's FP64-equivalent rate as a
        # multiple of the FP64 pipe's measured peak (not a roofline fraction)
        out["algorithmic_over_fp64_peak"] = tflops_alg / p64

    # the other workloads of the suite (N=1, default workload only)
    if world == 1 and not args.no_suite and args.workload == "bta_n64_b512_a256":
        del A, B, GR, GL
        ctx.close()
        ctx = None
        torch.cuda.empty_cache()
        out["mixed_c3"] = measure_c3()
        out["batched"] = measure_batched(256, 2, 1, "fp64_emu")
        out["serve"] = measure_serve(200, 4, "fp64_emu,mixed")

    if e2e is not None:
        out["e2e"] = e2e

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = oracle_sample(wl)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if ctx is not None:
        ctx.close()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
