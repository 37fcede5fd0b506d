"""bench.py's output contract on CPU: the reference arm's JSON line (the FP64
oracle timed on host cores) and the roofline bookkeeping of the GPU line,
exercised on fixed stage times."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--ref-slices", "2", "--ref-targets", "64"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["higher_is_better"] is True
    assert "workload" in rec["config"]
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == rec["value"] and cb["sample"]
    assert rec["e2e"] == {"value": rec["value"], "unit": rec["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


class _Obj:
    pass


def _mnist_like(proj="bf16x3", pair=True):
    import bench

    prob = _Obj()
    prob.N = prob.M = 60000
    prob.P, prob.d, prob.window, prob.n_ft, prob.kernel = 2048, 784, 8, 1024, "laplace"
    plan = _Obj()
    plan.G, plan.proj = 2048, proj
    plan.variant = lambda: "momentwin32"
    plan.gemm_pair = lambda: pair
    return bench, prob, plan


def test_roofline_takes_the_kernel_with_the_largest_time_per_step():
    bench, prob, plan = _mnist_like()
    stages = {"prep_x": 0.066, "project_x": 0.34, "spread_filter": 0.43, "prep_y": 0.27, "project_y": 0.31,
              "interp": 0.36, "reduce": 0.01}
    roof, per_stage = bench.roofline(prob, plan, stages, {"sm_mhz": 2070.0},
                                     {"bf16_tflops": 1890.0, "hbm_gbs": 6686.1}, "measured", 152)
    # the GEMM's two launches (0.65 ms) outweigh the spread's one (0.43 ms)
    assert roof["kernel"] == "tc_project_pair<BF16x3>" and roof["launches"] == 2
    flop = 6.0 * 60000 * 2048 * 784
    assert roof["achieved"] == pytest.approx(2 * flop / 0.65e-3 / 1e12, rel=1e-9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 1890.0, rel=1e-12)
    assert roof["traffic"] == pytest.approx(0.5 * (bench.TRAFFIC_MNIST["project_x"] +
                                                   bench.TRAFFIC_MNIST["project_y"]))
    sp = per_stage["spread_filter"]
    assert sp["hbm_bytes"] == 4.0 * 60000 * 2048 + 4.0 * 60000 + 4.0 * 2048 * 2048
    assert sp["hbm_frac"] == pytest.approx(sp["hbm_bytes"] / 0.43e-3 / 1e9 / 6686.1)


def test_traffic_is_null_outside_the_captured_configuration():
    bench, prob, plan = _mnist_like(pair=False)
    stages = {"project_x": 0.4, "project_y": 0.4, "spread_filter": 0.43, "interp": 0.36}
    roof, per_stage = bench.roofline(prob, plan, stages, {"sm_mhz": 2070.0},
                                     {"bf16_tflops": 1890.0, "hbm_gbs": 6686.1}, "measured", 152)
    assert roof["kernel"] == "tc_project_persistent<BF16x3>" and roof["traffic"] is None
    assert per_stage["interp"]["traffic"] == bench.TRAFFIC_MNIST["interp"]
    prob.N = prob.M = 1000
    roof, _ = bench.roofline(prob, plan, stages, {"sm_mhz": 2070.0}, {"bf16_tflops": 1890.0, "hbm_gbs": 6686.1},
                             "measured", 152)
    assert roof["traffic"] is None
