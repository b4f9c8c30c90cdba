"""Autotuner: scd_ssca_tune / scd_batch_tune time the schedules (and the persistent one's sizing
candidates, keep the fastest, record it (in-process and in the SCD_TUNE_CACHE JSON file), and
the tuned runs still match the FP64 oracle."""
import json
import os

import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import binding, signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    binding.load()
    return t


def _entries(path):
    return {e["key"]: e for e in json.load(open(path))["entries"]}


def test_ssca_tune_records_choice_and_auto_stays_exact(torch, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("SCD_TUNE_CACHE", str(cache))
    N, Np = 1 << 14, 64
    x = signals.modulated("qpsk", N, 4, 0.1, 5.0, seed=9100)
    a = orc.hamming_window(Np)
    xd, ad = torch.from_numpy(x).cuda(), torch.from_numpy(a).cuda()
    binding.scd_ssca_tune(xd, Np, window=ad, reps=2)
    e = [v for k, v in _entries(cache).items() if f"|ssca|N={N}|Np={Np}|p=0" in k]
    assert len(e) == 1 and e[0]["schedule"] in (1, 2, 3) and e[0]["ms"] > 0   # stages, persistent, fused
    got = binding.scd_ssca(xd, Np, window=ad, schedule="auto").cpu().numpy()
    binding.scd_check_device()
    ref = orc.ssca(x, a, Np)
    assert float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))) <= 1e-5


@pytest.mark.parametrize("estimator,Np,L", [("fam", 64, 16), ("ssca", 128, 1)])
def test_batch_tune_keeps_results_exact(torch, tmp_path, monkeypatch, estimator, Np, L):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("SCD_TUNE_CACHE", str(cache))
    lengths = [4096, 9000, 20000, 5000]
    sigs = [signals.batch_signal(300 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan(estimator, lengths, Np, L, "fp32")
    x = torch.from_numpy(np.concatenate(sigs)).cuda()
    out = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.tune(x, out, ws, stream=s, reps=1)
        out.zero_()
        plan.run(x, out, ws, stream=s)
    s.synchronize()
    binding.scd_check_device(s)
    assert any("|batch|" in k for k in _entries(cache))
    a = orc.hamming_window(Np)
    for i, sig in enumerate(sigs):
        if estimator == "fam":
            ref = orc.fam(sig, a, Np, L, plan.sizes[i])
        else:
            ref = orc.ssca(sig[:plan.sizes[i]], a, Np)
        got = plan.output(out, i).cpu().numpy()
        assert float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))) <= 1e-5
    plan.close()
