"""The benchmark's reference arm (the FP64 oracle on the host cores) runs without a GPU and
prints one JSON line with the contract's keys; the FLOP and byte models the roofline uses
match hand counts."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("workload", ["batch", "paper_scale"])
def test_reference_arm_json(workload):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--workload", workload], capture_output=True, text=True, check=True,
                         timeout=600).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert "workload" in d["config"]


def test_flop_model_hand_counts():
    import bench
    assert bench.fft_flops(1024) == 5 * 1024 * 10
    # FAM at Np=256, P=1024: frames 1024 x (2*256 + 5*256*8 + 6*256), pairs 65536 x (6*1024 + 5*1024*10)
    assert bench.fam_flops(256, 1024) == 1024 * (512 + 10240 + 1536) + 65536 * (6144 + 51200)
    # SSCA at Np=256, N=2^20: per point 2 + 5*8 + 12 per channel, per channel 5 N log2 N
    N = 1 << 20
    assert bench.ssca_flops(256, N) == N * (512 + 10240 + 3072) + 256 * 5 * N * 20
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9     # 152 SMs at 2.07 GHz
    assert abs(bench.fp32_peak_tflops(148, 1965.0) - 148 * 128 * 2 * 1.965e-3) < 1e-9
