"""Failure detection on the GPU without a GPU fault: a batch run whose first task never
publishes its completion (SCD_FAULT_INJECT=batch_drop:0) makes the dependent tasks give up
their bounded waits (2 s of device time); the host reads SCD_ERR_TIMEOUT from
scd_check_device, the context stays usable, and the next run without the injection is
correct."""
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


@pytest.mark.parametrize("estimator,Np,L", [("ssca", 32, 1), ("fam", 32, 8)])
def test_dropped_task_times_out_and_recovers(torch, monkeypatch, estimator, Np, L):
    lengths = [4096, 5000]
    sigs = [signals.batch_signal(500 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan(estimator, lengths, Np, L)
    if estimator == "ssca":
        plan.set_schedule("persistent")                      # the schedule with device-side waits
    x = torch.from_numpy(np.concatenate(sigs)).cuda()
    out = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    binding.scd_check_device()                               # clean start
    monkeypatch.setenv("SCD_FAULT_INJECT", "batch_drop:0")
    plan.run(x, out, ws, stream=stream)
    with pytest.raises(binding.ScdError) as e:
        binding.scd_check_device()
    assert e.value.status == binding.SCD_ERR_TIMEOUT
    monkeypatch.delenv("SCD_FAULT_INJECT")
    plan.run(x, out, ws, stream=stream)
    binding.scd_check_device()                               # no error: the context is usable
    a = orc.hamming_window(Np)
    for i, xs in enumerate(sigs):
        n = plan.sizes[i]
        ref = orc.fam(xs, a, Np, L, n) if estimator == "fam" else orc.ssca(xs[:n].copy(), a, Np)
        got = plan.output(out, i).cpu().numpy()
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5
    plan.close()
