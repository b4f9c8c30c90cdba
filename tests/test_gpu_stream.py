"""GPU parity of the streaming form (successive, overlapping or gapped windows of one
continuous signal through a persistent plan, scd_stream_plan_create / scd_stream_advance):
every window of three consecutive groups against the FP64 oracle on the same stream slice.
Gate: max|dS|/max|S| <= 1e-5 per window (FP32 form)."""
import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import binding, signals

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    binding.load()
    return t


def _rel(gpu, ref):
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


def _run_stream(torch, plan, stream_x, groups, host):
    """Yields (global window index, estimate) for `groups` groups of the plan."""
    nwin, hop, W = plan.nsig, plan.hop, plan.window_len
    keep = max(W - hop, 0)
    x_arena = torch.from_numpy(stream_x[:plan.span].copy()).cuda()
    out = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(groups):
        if k > 0:
            a = k * nwin * hop + keep
            chunk = torch.from_numpy(stream_x[a:a + nwin * hop].copy())
            plan.advance(x_arena, chunk.pin_memory() if host else chunk.cuda(), stream=stream)
        plan.run(x_arena, out, ws, stream=stream)
        binding.scd_check_device()
        for i in range(nwin):
            yield k * nwin + i, plan.output(out, i).cpu().numpy()


@pytest.mark.parametrize("W,hop,nwin,host", [(5000, 2048, 4, True), (4096, 4096, 3, False), (4100, 6000, 2, True)])
def test_ssca_stream_windows_match_oracle(torch, W, hop, nwin, host):
    Np = 32
    plan = binding.StreamPlan("ssca", W, hop, nwin, Np)
    groups = 3
    total = (groups * nwin - 1) * hop + W + nwin * hop
    x = signals.modulated("qpsk", total, 4, 0.1, 8.0, seed=7000 + W)
    a = orc.hamming_window(Np)
    N = plan.sizes[0]
    for w, got in _run_stream(torch, plan, x, groups, host):
        ref = orc.ssca(x[w * hop:w * hop + N].copy(), a, Np)
        assert _rel(got, ref) <= TOL, w
    plan.close()


@pytest.mark.parametrize("hop,nwin,host", [(300, 5, False), (2000, 3, True)])
def test_fam_stream_windows_match_oracle(torch, hop, nwin, host):
    Np, L, P = 32, 8, 128
    W = (P - 1) * L + Np + 5
    plan = binding.StreamPlan("fam", W, hop, nwin, Np, L)
    assert plan.sizes[0] == P
    groups = 3
    total = (groups * nwin - 1) * hop + W + nwin * hop
    x = signals.modulated("bpsk", total, 8, 0.05, 10.0, seed=7100 + hop, pulse="rect")
    a = orc.hamming_window(Np)
    for w, got in _run_stream(torch, plan, x, groups, host):
        ref = orc.fam(x[w * hop:w * hop + W].copy(), a, Np, L, P)
        assert _rel(got, ref) <= TOL, w
    plan.close()
