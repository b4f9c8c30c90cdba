"""GPU parity of the fused SSCA schedule (channeliser + channel-data product + the strip
transform's first pass in one tile, the second pass in another): against the FP64 oracle,
element by element, at every tile shape the schedule has, and against the three-stage
schedule; the cross, conjugate and normalised variants; sizes the fused tiles do not fit run
the three-stage kernels."""
import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import binding, signals

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    binding.load()
    return t


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(gpu, ref):
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


# (N, Np): every (Np, M1, Q) tile shape (Q CTAs per cluster) and every second-pass size M2 in
# 64 .. 2048
FULL = [(1 << 12, 64), (1 << 13, 128), (1 << 14, 128), (1 << 14, 256), (1 << 15, 128), (1 << 15, 64)]
SAMPLED = [(1 << 16, 128), (1 << 16, 256), (1 << 17, 128), (1 << 17, 64), (1 << 17, 256), (1 << 18, 128),
           (1 << 18, 64), (1 << 19, 128)]


@pytest.mark.parametrize("N,Np", FULL)
def test_fused_matches_oracle_full(torch, N, Np):
    x = signals.modulated("qpsk", N, 4, 0.1, 5.0, seed=2100 + Np + N % 977)
    a = orc.hamming_window(Np)
    ref = orc.ssca(x, a, Np)
    got = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), schedule="fused").cpu().numpy()
    binding.scd_check_device()
    assert _rel(got, ref) <= FP32_TOL


@pytest.mark.parametrize("N,Np", SAMPLED)
def test_fused_matches_oracle_sampled_channels(torch, N, Np):
    """Full channel rows at the band edges, the centre and the boundaries between the
    cluster's channel blocks, recomputed by the oracle; every channel against the three-stage
    schedule."""
    x = signals.modulated("8psk", N, 8, -0.07, 3.0, seed=2200 + Np + N % 991)
    a = orc.hamming_window(Np)
    xd, ad = _dev(torch, x), _dev(torch, a)
    got_t = binding.scd_ssca(xd, Np, window=ad, schedule="fused")
    binding.scd_check_device()
    ch = np.array(sorted({0, 1, Np // 4 - 1, Np // 4, Np // 2 - 1, Np // 2, Np // 2 + 1, 3 * Np // 4 - 1,
                          3 * Np // 4, Np - 2, Np - 1}))
    ref = orc.ssca(x, a, Np, channels=ch, chunk=1 << 15)
    got = got_t[torch.from_numpy(ch).cuda()].cpu().numpy()
    smax = got_t.abs().max().item()
    assert float(np.max(np.abs(got - ref))) / smax <= FP32_TOL
    stages = binding.scd_ssca(xd, Np, window=ad, schedule="stages")
    assert (got_t - stages).abs().max().item() / smax <= FP32_TOL
    del got_t, stages
    torch.cuda.empty_cache()


@pytest.mark.parametrize("variant", ["cross", "conjugate", "normalise", "default_window"])
def test_fused_variants(torch, variant):
    N, Np = 1 << 14, 128
    x = signals.modulated("bpsk", N, 4, 0.11, 6.0, seed=2300)
    y = signals.modulated("qpsk", N, 8, -0.05, 2.0, seed=2301)
    a = orc.hamming_window(Np)
    kw, okw = {}, {}
    if variant == "cross":
        kw, okw = {"y": _dev(torch, y)}, {"y": y}
    elif variant == "conjugate":
        kw, okw = {"conjugate": True}, {"conjugate": True}
    elif variant == "normalise":
        kw, okw = {"normalise": 1}, {"normalise": 1}
    window = None if variant == "default_window" else _dev(torch, a)
    ref = orc.ssca(x, a, Np, **okw)
    got = binding.scd_ssca(_dev(torch, x), Np, window=window, schedule="fused", **kw).cpu().numpy()
    binding.scd_check_device()
    assert _rel(got, ref) <= FP32_TOL


@pytest.mark.parametrize("N,Np", [(1 << 12, 32), (1 << 20, 128), (1 << 12, 128), (1 << 19, 256)])
def test_fused_outside_its_tiles_runs_the_stages(torch, N, Np):
    x = signals.modulated("qpsk", N, 4, 0.02, 5.0, seed=2400 + Np)
    xd = _dev(torch, x)
    f = binding.scd_ssca(xd, Np, schedule="fused")
    s = binding.scd_ssca(xd, Np, schedule="stages")
    binding.scd_check_device()
    assert torch.equal(f, s)
    del f, s
    torch.cuda.empty_cache()
