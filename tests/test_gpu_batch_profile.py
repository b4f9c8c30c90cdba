"""Alpha-profile output of the batched and streaming plans (scd_batch_plan_set_output):
each signal's profile, reduced inside the persistent kernel without writing the estimate,
against the FP64 oracle's profile of the same signal, and bit for bit against the
standalone profile kernels applied to the same plan's full estimates."""
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


def _both_modes(torch, plan, x, power):
    """Runs the plan in estimate mode, then in profile mode, on the same inputs."""
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    full = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device="cuda")
    plan.run(x, full, ws)
    est = [plan.output(full, i).clone() for i in range(plan.nsig)]
    plan.set_output("profile", power)
    prof = torch.full((plan.out_offsets[-1],), -1.0, dtype=torch.float32, device="cuda")   # run zeroes it
    plan.run(x, prof, ws)
    plan.run(x, prof, ws)                                   # a second run gives the same maxima
    binding.scd_check_device()
    return est, [plan.output(prof, i) for i in range(plan.nsig)]


@pytest.mark.parametrize("precision,power", [("fp32", 1), ("fp32", 2), ("split", 1)])
def test_fam_batch_profiles(torch, precision, power):
    Np, L = 32, 8
    lengths = [1200, 4100, 2500, 9000, 300, 16000]
    sigs = [signals.batch_signal(200 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("fam", lengths, Np, L, precision)
    x = torch.from_numpy(np.concatenate(sigs)).cuda()
    est, prof = _both_modes(torch, plan, x, power)
    a = orc.hamming_window(Np)
    for i, xs in enumerate(sigs):
        P = plan.sizes[i]
        assert prof[i].numel() == 2 * P * L
        same = binding.scd_fam_alpha_profile(est[i], Np, L, P, power=power)
        assert torch.equal(prof[i], same), i
        ref = orc.fam_alpha_profile(orc.fam(xs, a, Np, L, P), Np, L, P, power=power)
        got = prof[i].cpu().numpy()
        assert np.max(np.abs(got - ref)) / np.max(ref) <= TOL[precision] * power, i
    plan.close()


@pytest.mark.parametrize("precision,power", [("fp32", 1), ("fp32", 2), ("split", 1)])
def test_ssca_batch_profiles(torch, precision, power):
    Np = 64
    lengths = [4096, 7000, 16384, 5000, 33000]
    sigs = [signals.batch_signal(300 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("ssca", lengths, Np, 1, precision)
    x = torch.from_numpy(np.concatenate(sigs)).cuda()
    est, prof = _both_modes(torch, plan, x, power)
    a = orc.hamming_window(Np)
    for i, xs in enumerate(sigs):
        N = plan.sizes[i]
        assert prof[i].numel() == 2 * N
        same = binding.scd_ssca_alpha_profile(est[i], N, Np, power=power)
        assert torch.equal(prof[i], same), i
        ref = orc.ssca_alpha_profile(orc.ssca(xs[:N].copy(), a, Np), N, Np, power=power)
        got = prof[i].cpu().numpy()
        assert np.max(np.abs(got - ref)) / np.max(ref) <= TOL[precision] * power, i
    plan.close()


def test_stream_plan_profiles(torch):
    Np, W, hop, nwin = 32, 4096, 2048, 6
    plan = binding.StreamPlan("ssca", W, hop, nwin, Np)
    xs = signals.modulated("bpsk", plan.span, 8, 0.05, 10.0, seed=9000, pulse="rect")
    x = torch.from_numpy(xs).cuda()
    est, prof = _both_modes(torch, plan, x, 1)
    for i in range(nwin):
        assert torch.equal(prof[i], binding.scd_ssca_alpha_profile(est[i], W, Np)), i
    plan.close()


def test_profile_mode_validation(torch):
    plan = binding.BatchPlan("fam", [4096], 32, 20)          # 2 L > Np: the map band does not tile alpha
    with pytest.raises(binding.ScdError):
        plan.set_output("profile")
    plan.close()
