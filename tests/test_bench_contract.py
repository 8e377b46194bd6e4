"""The reference arm of bench.py (the oracle on the host cores) prints one JSON
line with the keys and units of the benchmark line; no GPU needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "bta_n8_b32_a16"],
                         capture_output=True, text=True, cwd=ROOT, timeout=600, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "bta_n8_b32_a16"
    # the reference line names what it times: the numpy oracle, not the library call
    assert "oracle" in line["config"]["call"] and "qsi_" not in line["config"]["call"]
    assert "complex128" in line["config"]["precision"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def _stats(**kw):
    st = {k: 0 for k in ("panel_ms", "panel_launches", "panel_flops", "panel32_ms", "panel32_launches",
                         "panel32_flops", "gemm_ms", "gemm_launches", "gemm_flops", "tc_ms", "tc_launches",
                         "tc_flops")}
    st.update(kw)
    return st


def test_roofline_names_and_measures_the_dominant_kernel():
    """roofline_of (host arithmetic only): the kernel family with the largest
    summed event time is reported, the FP32 Gauss-Jordan under the kernel that
    runs at that block size, achieved = its flops / its time, frac against its peak."""
    sys.path.insert(0, ROOT)
    import bench

    wl = {"n": 64, "b": 512, "a": 256}
    st = _stats(panel32_ms=60.0, panel32_launches=64, panel32_flops=64 * 8 * 512.0 ** 3,
                tc_ms=50.0, tc_launches=900, tc_flops=3.0e12)
    r = bench.roofline_of(st, 100.0, "fp64_emu", wl)
    assert r["kernel"].startswith("gj32_cluster_kernel") and r["bound"] == "alu"
    assert abs(r["achieved"] - 64 * 8 * 512.0 ** 3 / 60e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / bench.FP32_PEAK_TFLOPS) < 1e-12
    assert [k["kernel"] for k in r["all_kernels"]][0] == "gj32_cluster_kernel"
    r = bench.roofline_of(st, 100.0, "fp64_emu", {"n": 8, "b": 1024, "a": 512})
    assert r["kernel"].startswith("panel32_kernel")
    st = _stats(panel32_ms=10.0, panel32_launches=64, panel32_flops=1e10, tc_ms=50.0, tc_launches=900,
                tc_flops=3.0e12)
    r = bench.roofline_of(st, 100.0, "fp64_emu", wl)
    if r is not None and bench.measured_peaks().get("bf16_tflops_sustained"):
        assert r["kernel"].startswith("tc_mma_kernel") and r["bound"] == "tensor"
        assert r["achieved"] <= 3.0e12 / 50e-3 / 1e12 + 1e-9
