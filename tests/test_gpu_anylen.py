"""GPU parity of the any-length transforms (Bluestein's identity on the power-of-two FFTs):
FAM with a number of blocks P and SSCA with a signal length N that are not powers of two,
through the C ABI, against the FP64 oracle on the same seeded inputs.  Gates: FP32 form
max|dS|/max|S| <= 1e-5, split form <= 1e-3 (the stated targets).  Sizes span one to many
tiles, odd and even lengths, the smallest and the largest transform each path takes."""
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


def _rel(gpu, ref):
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ----------------------------------------------------------------------------- FAM, any P
@pytest.mark.parametrize("precision", ["fp32", "split"])
@pytest.mark.parametrize("Np,L,P,extra", [
    (16, 4, 3, 0),           # smallest transform (8 points, single pass)
    (16, 4, 5, 2),
    (32, 8, 7, 0),
    (32, 8, 24, 1),
    (64, 16, 100, 0),
    (16, 4, 1000, 3),        # 2048-point transforms, two per CTA
    (128, 32, 257, 0),       # just above a power of two: 1024-point transforms
    (16, 2, 5000, 0),        # 16384-point transforms (512 threads, one per CTA)
    (16, 1, 8191, 0),        # the largest P that is not a power of two
])
def test_fam_any_p_matches_oracle(torch, Np, L, P, extra, precision):
    N = (P - 1) * L + Np + extra
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=7000 + Np + P, pulse="rect")
    a = orc.hamming_window(Np)
    ref = orc.fam(x, a, Np, L, P)
    got = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), precision=precision).cpu().numpy()
    assert _rel(got, ref) <= TOL[precision]


@pytest.mark.parametrize("cross,conjugate", [(True, False), (False, True)])
def test_fam_any_p_variants(torch, cross, conjugate):
    Np, L, P = 32, 8, 77
    N = (P - 1) * L + Np
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=7100, pulse="rect")
    y = signals.modulated("qpsk", N, 4, -0.11, 5.0, seed=7101)
    a = orc.hamming_window(Np)
    ref = orc.fam(x, a, Np, L, P, y=y if cross else None, conjugate=conjugate)
    got = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), y=_dev(torch, y) if cross else None,
                          conjugate=conjugate).cpu().numpy()
    assert _rel(got, ref) <= TOL["fp32"]


def test_fam_any_p_paper_scale_sampled_pairs(torch):
    """Np=256, L=64 with P=1000 (N = 64,192): 48 sampled pairs recomputed by the oracle, and
    the exact symmetry S(l, k, -q) = conj S(k, l, q) over the whole estimate (for even P the
    bin -q sits at (P - qh) mod P)."""
    Np, L, P = 256, 64, 1000
    N = (P - 1) * L + Np
    x = signals.modulated("16qam", N, 8, 0.03, 12.0, seed=7200)
    a = orc.hamming_window(Np)
    got_t = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a))
    g = np.random.default_rng(72)
    kh = np.concatenate([g.integers(0, Np, 44), [0, 255, 128, 0]])
    lh = np.concatenate([g.integers(0, Np, 44), [0, 255, 128, 255]])
    ref = orc.fam_pairs(x, a, Np, L, P, kh, lh)
    got = got_t[torch.from_numpy(kh).cuda(), torch.from_numpy(lh).cuda()].cpu().numpy()
    smax = got_t.abs().max().item()
    assert float(np.max(np.abs(got - ref))) / smax <= TOL["fp32"]
    qh = torch.remainder(P - torch.arange(P, device="cuda"), P)
    err = (got_t.transpose(0, 1)[:, :, qh] - got_t.conj()).abs().max().item()
    assert err / smax <= TOL["fp32"]
    del got_t
    torch.cuda.empty_cache()


# ----------------------------------------------------------------------------- SSCA, any N
@pytest.mark.parametrize("precision", ["fp32", "split"])
@pytest.mark.parametrize("N,Np", [
    (4097, 16),              # smallest: 8192-point cyclic transforms
    (5000, 256),
    (6001, 32),
    (12345, 64),
    (3 * (1 << 13), 128),    # 24,576 = 3 * 2^13
    (100003, 16),            # prime length
])
def test_ssca_any_n_matches_oracle(torch, N, Np, precision):
    x = signals.modulated("qpsk", N, 4, 0.1, 5.0, seed=7300 + Np)
    a = orc.hamming_window(Np)
    ref = orc.ssca(x, a, Np)
    got = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), precision=precision).cpu().numpy()
    binding.scd_check_device()
    assert _rel(got, ref) <= TOL[precision]


@pytest.mark.parametrize("cross,conjugate,normalise", [(True, False, None), (False, True, None),
                                                       (True, True, None), (False, False, "power")])
def test_ssca_any_n_variants(torch, cross, conjugate, normalise):
    N, Np = 7777, 64
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=7400, pulse="rect")
    y = signals.modulated("qpsk", N, 4, -0.11, 5.0, seed=7401)
    a = orc.hamming_window(Np)
    ref = orc.ssca(x, a, Np, y=y if cross else None, conjugate=conjugate,
                   normalise={None: 0, "power": 1}[normalise])
    got = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), y=_dev(torch, y) if cross else None,
                           conjugate=conjugate, normalise=normalise).cpu().numpy()
    assert _rel(got, ref) <= TOL["fp32"]


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_ssca_any_n_largest_sampled_channels(torch, precision):
    """N = 2^19 - 1 (the largest length that is not a power of two: 2^20-point cyclic
    transforms) at Np = 256: 4 full channel rows recomputed by the oracle."""
    N, Np = (1 << 19) - 1, 256
    x = signals.modulated("bpsk", N, 4, -0.12, 3.0, seed=7500)
    a = orc.hamming_window(Np)
    got_t = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), precision=precision)
    binding.scd_check_device()
    ch = np.array([0, 101, 128, 255])
    ref = orc.ssca(x, a, Np, channels=ch, chunk=1 << 16)
    got = got_t[torch.from_numpy(ch).cuda()].cpu().numpy()
    smax = got_t.abs().max().item()
    assert float(np.max(np.abs(got - ref))) / smax <= TOL[precision]
    del got_t
    torch.cuda.empty_cache()


def test_ssca_any_n_rejects_persistent_schedule(torch):
    x = torch.zeros(5000, dtype=torch.complex64, device="cuda")
    with pytest.raises(binding.ScdError):
        binding.scd_ssca(x, 32, schedule="persistent")
