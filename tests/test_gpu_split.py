"""Split-precision form (radix DFTs as bf16 hi/lo tensor-core GEMMs, FP32 accumulation)
against the FP64 oracle.  Gate: max |S_gpu - S_oracle| / max |S_oracle| <= 1e-3 (the stated
target for this form); the measured error is printed for the record."""
import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import binding, signals

pytestmark = pytest.mark.gpu

SPLIT_TOL = 1e-3


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    binding.load()
    return t


def _rel(gpu, ref):
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("Np,L,P", [
    (32, 8, 32), (16, 4, 2), (16, 4, 8), (64, 16, 64), (64, 16, 128), (128, 32, 256), (256, 64, 512),
    (16, 4, 2048), (16, 4, 4096), (16, 8, 8192), (16, 2, 16384),
])
def test_fam_split_matches_oracle(torch, Np, L, P):
    N = (P - 1) * L + Np + 1
    x = signals.modulated("qpsk", N, 8, 0.05, 10.0, seed=5000 + Np + P)
    a = orc.hamming_window(Np)
    ref = orc.fam(x, a, Np, L, P)
    got = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), precision="split").cpu().numpy()
    binding.scd_check_device()
    err = _rel(got, ref)
    print(f"FAM split Np={Np} L={L} P={P}: max err / max|S| = {err:.3e}")
    assert err <= SPLIT_TOL


def test_fam_split_paper_scale_sampled(torch):
    w = signals.fam_qam16_paper_scale()
    x, Np, L, P = w["x"], w["Np"], w["L"], w["P"]
    a = orc.hamming_window(Np)
    got_t = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), precision="split")
    binding.scd_check_device()
    g = np.random.default_rng(8)
    kh, lh = g.integers(0, Np, 64), g.integers(0, Np, 64)
    ref = orc.fam_pairs(x, a, Np, L, P, kh, lh)
    got = got_t[torch.from_numpy(kh).cuda(), torch.from_numpy(lh).cuda()].cpu().numpy()
    err = float(np.max(np.abs(got - ref))) / got_t.abs().max().item()
    print(f"FAM split paper scale: sampled max err / max|S| = {err:.3e}")
    assert err <= SPLIT_TOL


@pytest.mark.parametrize("schedule", ["auto", "stages"])
@pytest.mark.parametrize("N,Np", [(1 << 12, 16), (1 << 12, 256), (1 << 13, 32), (1 << 14, 64), (1 << 15, 128)])
def test_ssca_split_matches_oracle(torch, N, Np, schedule):
    x = signals.modulated("qpsk", N, 4, 0.1, 5.0, seed=6000 + Np)
    a = orc.hamming_window(Np)
    ref = orc.ssca(x, a, Np)
    got = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), precision="split",
                           schedule=schedule).cpu().numpy()
    binding.scd_check_device()
    err = _rel(got, ref)
    print(f"SSCA split N={N} Np={Np}: max err / max|S| = {err:.3e}")
    assert err <= SPLIT_TOL


def test_ssca_split_1m_sampled(torch):
    w = signals.ssca_mixture_1m()
    x, Np = w["x"], w["Np"]
    a = orc.hamming_window(Np)
    got_t = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), precision="split")
    binding.scd_check_device()
    ch = np.array([3, 128, 250])
    ref = orc.ssca(x, a, Np, channels=ch, chunk=1 << 16)
    got = got_t[torch.from_numpy(ch).cuda()].cpu().numpy()
    err = float(np.max(np.abs(got - ref))) / got_t.abs().max().item()
    print(f"SSCA split N=2^20: sampled max err / max|S| = {err:.3e}")
    assert err <= SPLIT_TOL
    del got_t
    torch.cuda.empty_cache()
