"""Host-side arithmetic of bench.py: algorithmic bytes and flops behind the roofline fields."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_algorithmic_bytes_per_update():
    # complex64: read H (K x N), write W (N x K); WB also reads and writes G and X (K x K each)
    assert bench.algorithmic_bytes_per_update(256, 32, "full") == 8 * 2 * 256 * 32
    assert bench.algorithmic_bytes_per_update(256, 32, "wb") == 8 * 2 * 256 * 32 + 8 * 4 * 32 * 32
    # the batched workload's launch: 1024 instances, 160 KiB each
    assert 1024 * bench.algorithmic_bytes_per_update(256, 32, "wb") == 167772160


def test_lowrank_flops_counts_the_sketch_widths_of_algorithm_1():
    # K = 8, k_init = 2, p = 1: widths 3, 5, 8 (capped at K)
    def it(K, d):
        return 16.0 * K * K * d + 24.0 * K * d * d
    assert bench.lowrank_flops(8, 2, 1, 1) == it(8, 3)
    assert bench.lowrank_flops(8, 2, 1, 3) == it(8, 3) + it(8, 5) + it(8, 8)
    assert bench.lowrank_flops(8, 2, 1, 1.5) == it(8, 3) + 0.5 * it(8, 5)
    assert bench.lowrank_flops(8, 2, 1, 0) == 0.0


def test_blocked_roofline_takes_the_dominant_stage():
    st = {"gram": 0.1, "lowrank": 6.0, "woodbury": 0.02, "inverse": 1.2, "precoder": 0.2,
          "total": 7.52}
    f = bench.lowrank_flops(512, 2, 8, 6)
    r = bench.blocked_roofline(st, 1, 4096, 512, f)
    assert r["kernel"] == "blocked engine stage 'lowrank'"
    assert r["achieved"] == pytest.approx(f / 6.0e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP32_FMA_TFLOPS)
    st2 = dict(st, lowrank=0.05)
    r2 = bench.blocked_roofline(st2, 4, 4096, 512)
    assert r2["kernel"] == "blocked engine stage 'inverse'" and r2["achieved"] is None
    st3 = dict(st2, precoder=2.0)
    r3 = bench.blocked_roofline(st3, 4, 4096, 512)
    assert r3["achieved"] == pytest.approx(4 * (8.0 * 4096 * 512 ** 2 + 8.0 * 512 ** 3) / 2e-3 / 1e12)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on host cores (no GPU) and prints one
    JSON line with the metric, unit and config of the default workload, the oracle as its
    cpu_baseline and an e2e object with zero copy bytes."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                         timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC
    assert d["unit"] == "updates/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("batched_256x32")
