"""bench.py's host side without a GPU: the reference arm (the FP64 oracle on the
host cores) prints one JSON line with the contract's keys, only rank 0 of a
multi-rank launch prints it, and the roofline block's arithmetic."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0"}, "--workload", "2d_n20_256sq", "--steps", "2", "--warmup", "1")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference"
    assert out["steps"] == 2 and out["warmup"] == 1 and out["n_gpus"] == 1
    assert out["higher_is_better"] is True and out["dtype"] == "f64"
    assert out["value"] > 0 and out["cpu_baseline"]["value"] == out["value"]
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert out["config"]["workload"] == "2d_n20_256sq"
    # a step is one complete FP64 evaluation, timed as it ran; the APD rate divides
    # by the evaluations one APD takes
    assert out["ms_per_step"] == pytest.approx(1000.0 * out["evaluation_s"], rel=1e-9)
    assert out["value"] == pytest.approx(1.0 / (out["evaluation_s"] * out["evals_per_apd"]), rel=1e-9)
    assert out["pair_evals_per_s"] == pytest.approx(65536 * 20 / out["evaluation_s"], rel=1e-9)


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--workload", "2d_n20_256sq", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_roofline_arithmetic():
    # FP32 form: achieved = evaluated pairs x the executed flops per pair / time,
    # peak = SMs x 128 FP32 lanes x 2 flops x the max SM clock, frac = achieved / peak;
    # the algorithmic and dense-equivalent figures are rates beside it.
    # Tensor-core form: 2 x 32 tensor flops per scored pair against the operand type's peak.
    import bench
    peaks, _ = bench.load_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    form = {"precision": "fp32", "pair_rate": 6.0e12, "scored_pair_rate": 3.0e11, "pruned": True,
            "launch_ms": 0.6, "launches": 10}
    rb = bench.roofline_block(form, 3, 152, "3d_n1000_256cube_lloyd5")
    peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    assert rb["bound"] == "alu" and rb["unit"] == "TFLOP/s"
    assert rb["peak"] == pytest.approx(peak)
    assert rb["achieved"] == pytest.approx(3.0e11 * bench.FLOPS_PER_PAIR[3] / 1e12)
    assert rb["frac"] == pytest.approx(rb["achieved"] / peak)
    assert rb["algorithmic_tflops_evaluated"] == pytest.approx(3.0e11 * 20 / 1e12)
    assert rb["dense_equivalent_rate_tflops"] == pytest.approx(6.0e12 * 20 / 1e12)
    rb2 = bench.roofline_block(dict(form, precision="tc_tf32"), 2, 152, "2d_n2000_1024sq")
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    assert rb2["bound"] == "tensor" and rb2["peak"] == pytest.approx(bf16 * 1.1 / 2.25)
    assert rb2["achieved"] == pytest.approx(3.0e11 * 64 / 1e12)
    assert rb2["frac"] == pytest.approx(rb2["achieved"] / rb2["peak"])


def test_counters_follow_the_kernel_code(tmp_path, monkeypatch):
    # the ncu counters are used only while the kernel's code hash matches the capture
    import bench
    f = tmp_path / "c.txt"
    h = bench.kernel_source_hash("tc")
    f.write_text(f"# kernel workload form hash dram_bytes warp_instructions pairs\n"
                 f"assign_tc_kernel<3,0> 3d_n1000_256cube_lloyd5 pruned {h} 1000 2000 4000\n"
                 f"assign_tc_kernel<3,0> 3d_n1000_256cube_lloyd5 dense 0123456789abcdef 1 2 3\n")
    monkeypatch.setattr(bench, "COUNTERS_FILE", str(f))
    assert bench.ncu_counters("assign_tc_kernel<3,0>", "3d_n1000_256cube_lloyd5", True, "tc") == \
        {"dram_bytes": 1000, "warp_instructions": 2000, "pairs": 4000}
    assert bench.ncu_counters("assign_tc_kernel<3,0>", "3d_n1000_256cube_lloyd5", False, "tc") is None
    # scaled to the timed region's mean launch by its N x J pairs (here twice the captured launch's)
    form = {"precision": "tc_tf32", "pair_rate": 8.0e6, "scored_pair_rate": 1.0e6, "pruned": True,
            "launch_ms": 1.0, "launches": 3}
    rb = bench.roofline_block(form, 3, 152, "3d_n1000_256cube_lloyd5")
    assert rb["traffic"] == 2000 and rb["warp_instructions_per_launch"] == 4000
    peaks, _ = bench.load_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    assert rb["issue_frac"] == pytest.approx(4000 / 1e-3 / (4 * 152 * mhz * 1e6))
