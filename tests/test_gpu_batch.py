"""Batched form: uneven-length signals through one persistent (graph-captured) launch per
estimator; every signal's estimate is compared with the FP64 oracle on the same input."""
import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import binding, signals

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split": 1e-3}


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    binding.load()
    return t


def _arena(torch, sigs):
    return torch.from_numpy(np.concatenate(sigs)).cuda()


def _run(torch, plan, sigs, stream=None):
    x = _arena(torch, sigs)
    out = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    plan.run(x, out, ws, stream=stream)
    binding.scd_check_device(stream)
    return x, out, ws


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_fam_batch_every_signal(torch, precision):
    Np, L = 64, 16
    lengths = [4096, 5000, 1100, 8300, 4200, 2200, 17000, 3000]
    sigs = [signals.batch_signal(i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("fam", lengths, Np, L, precision)
    assert plan.sizes == [128, 256, 64, 512, 256, 128, 1024, 128]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _, out, _ = _run(torch, plan, sigs, s)
    s.synchronize()
    a = orc.hamming_window(Np)
    for i, x in enumerate(sigs):
        P = plan.sizes[i]
        ref = orc.fam(x, a, Np, L, P)
        got = plan.output(out, i).cpu().numpy()
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert err <= TOL[precision], (i, err)
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_ssca_batch_every_signal(torch, precision):
    Np = 128
    lengths = [4096, 6000, 16384, 9000, 40000, 4500]
    sigs = [signals.batch_signal(100 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("ssca", lengths, Np, 1, precision)
    assert plan.sizes == [4096, 4096, 16384, 8192, 32768, 4096]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _, out, _ = _run(torch, plan, sigs, s)
    s.synchronize()
    a = orc.hamming_window(Np)
    for i, x in enumerate(sigs):
        N = plan.sizes[i]
        ref = orc.ssca(x[:N], a, Np)
        got = plan.output(out, i).cpu().numpy()
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert err <= TOL[precision], (i, err)
    plan.close()


def test_batch_graph_replay_is_bitwise_deterministic(torch):
    Np, L = 64, 16
    lengths = [5000, 9000, 4100, 20000]
    sigs = [signals.batch_signal(200 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("fam", lengths, Np, L, "fp32")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x, out, ws = _run(torch, plan, sigs, s)
        first = out.clone()
        for _ in range(3):                                    # graph replays
            out.zero_()
            plan.run(x, out, ws, stream=s)
    s.synchronize()
    binding.scd_check_device(s)
    assert torch.equal(out, first)
    plan.close()


def test_batch_rejects_too_short_signal(torch):
    with pytest.raises(binding.ScdError):
        binding.BatchPlan("ssca", [5000, 1000], 128)


def test_batch_512_signals_subset(torch):
    """The 512-signal mixed workload (lengths log-uniform in [2^12, 2^18]), SSCA at Np=128:
    all signals in one launch; the 4 shortest and 2 longest checked against the oracle."""
    Np = 128
    lengths = signals.batch_lengths()
    sigs = [signals.batch_signal(i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("ssca", lengths, Np, 1, "fp32")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _, out, _ = _run(torch, plan, sigs, s)
    s.synchronize()
    a = orc.hamming_window(Np)
    order = np.argsort(lengths)
    for i in list(order[:4]) + list(order[-2:]):
        N = plan.sizes[i]
        ch = np.array([0, 77, 127])
        ref = orc.ssca(sigs[i][:N], a, Np, channels=ch)
        got = plan.output(out, i)[torch.from_numpy(ch).cuda()].cpu().numpy()
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert err <= TOL["fp32"], (i, err)
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_ssca_batch_staged_schedule(torch, precision):
    """The staged schedule (one launch per stage and size class) against the FP64 oracle for
    every signal, and bit for bit against the persistent schedule (same tile arithmetic)."""
    Np = 64
    lengths = [4096, 70000, 9000, 4200, 150000, 33000, 8192]
    sigs = [signals.batch_signal(300 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("ssca", lengths, Np, 1, precision)
    plan.set_schedule("persistent")
    _, out_p, _ = _run(torch, plan, sigs)
    plan.set_schedule("stages")
    _, out_s, _ = _run(torch, plan, sigs)
    assert torch.equal(out_p, out_s)
    a = orc.hamming_window(Np)
    for i, x in enumerate(sigs):
        N = plan.sizes[i]
        ref = orc.ssca(x[:N].copy(), a, Np)
        got = plan.output(out_s, i).cpu().numpy()
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert err <= TOL[precision], (i, err)
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_fam_batch_staged_schedule(torch, precision):
    """FAM staged schedule (the channelisers, then one launch per size class P) against the
    FP64 oracle for every signal, and bit for bit against the persistent schedule."""
    Np, L = 64, 16
    lengths = [4096, 5000, 1100, 8300, 70000, 2200, 17000, 3000, 140000]
    sigs = [signals.batch_signal(400 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("fam", lengths, Np, L, precision)
    plan.set_schedule("persistent")
    _, out_p, _ = _run(torch, plan, sigs)
    plan.set_schedule("stages")
    _, out_s, _ = _run(torch, plan, sigs)
    assert torch.equal(out_p, out_s)
    a = orc.hamming_window(Np)
    for i, x in enumerate(sigs):
        P = plan.sizes[i]
        ref = orc.fam(x, a, Np, L, P)
        got = plan.output(out_s, i).cpu().numpy()
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert err <= TOL[precision], (i, err)
    plan.close()


@pytest.mark.parametrize("estimator,Np,L", [("fam", 64, 16), ("ssca", 64, 1)])
def test_batch_profile_output_both_schedules(torch, estimator, Np, L):
    """Alpha-profile output: the staged schedule's profiles equal the persistent schedule's bit
    for bit (maxima do not depend on the order of the reductions)."""
    lengths = [4096, 70000, 9000, 33000]
    sigs = [signals.batch_signal(500 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan(estimator, lengths, Np, L)
    plan.set_output("profile")
    x = _arena(torch, sigs)
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    outs = []
    for sched in ("persistent", "stages"):
        plan.set_schedule(sched)
        out = torch.empty(plan.out_offsets[-1], dtype=torch.float32, device="cuda")
        plan.run(x, out, ws)
        binding.scd_check_device()
        outs.append(out)
    assert torch.equal(outs[0], outs[1])
    assert float(outs[1].max()) > 0
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_fam_batch_exact_lengths(torch, precision):
    """Exact-length FAM plan: P_i = (len_i - Np)//L + 1 (powers of two and not), every signal
    against the FP64 oracle."""
    Np, L = 32, 8
    lengths = [1000, 1048, 824, 2000, 300]
    sigs = [signals.batch_signal(600 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("fam", lengths, Np, L, precision, exact=True)
    assert plan.sizes == [(n - Np) // L + 1 for n in lengths]
    _, out, _ = _run(torch, plan, sigs)
    a = orc.hamming_window(Np)
    for i, x in enumerate(sigs):
        ref = orc.fam(x, a, Np, L, plan.sizes[i])
        got = plan.output(out, i).cpu().numpy()
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert err <= TOL[precision], (i, err)
    with pytest.raises(binding.ScdError):
        plan.set_output("profile")
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_ssca_batch_exact_lengths(torch, precision):
    """Exact-length SSCA plan: N_i = len_i (powers of two and not), every signal against the
    FP64 oracle."""
    Np = 32
    lengths = [5000, 8192, 4500, 12289]
    sigs = [signals.batch_signal(700 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("ssca", lengths, Np, 1, precision, exact=True)
    assert plan.sizes == lengths
    _, out, _ = _run(torch, plan, sigs)
    a = orc.hamming_window(Np)
    for i, x in enumerate(sigs):
        ref = orc.ssca(x, a, Np)
        got = plan.output(out, i).cpu().numpy()
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert err <= TOL[precision], (i, err)
    plan.close()
