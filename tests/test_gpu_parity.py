"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by
element on the same seeded inputs.  Gate for the FP32 form: max |S_gpu - S_oracle| /
max |S_oracle| <= 1e-5 (the stated FP32 accuracy target)."""
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


def _rel(gpu, ref):
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ----------------------------------------------------------------------------- FAM
@pytest.mark.parametrize("Np,L,P,extra", [
    (32, 8, 32, 0),          # the N=280 BPSK configuration
    (16, 4, 2, 3),
    (16, 1, 8, 0),
    (16, 4, 16, 1),
    (64, 16, 64, 7),         # ragged tail ignored
    (64, 16, 128, 0),
    (128, 32, 256, 5),
    (256, 64, 64, 0),
    (16, 4, 2048, 0),
    (16, 4, 4096, 2),
    (16, 8, 8192, 0),
    (16, 2, 16384, 0),
])
def test_fam_matches_oracle(torch, Np, L, P, extra):
    N = (P - 1) * L + Np + extra
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=1000 + Np + P, pulse="rect")
    a = orc.hamming_window(Np)
    ref = orc.fam(x, a, Np, L, P)
    got = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a)).cpu().numpy()
    assert _rel(got, ref) <= FP32_TOL


def test_fam_small_config_and_default_window(torch):
    w = signals.fam_small_bpsk()
    x, Np, L, P = w["x"], w["Np"], w["L"], w["P"]
    ref = orc.fam(x, orc.hamming_window(Np), Np, L, P, mode="direct")
    got = binding.scd_fam(_dev(torch, x), Np, L, P).cpu().numpy()        # window = NULL
    assert _rel(got, ref) <= FP32_TOL


def test_fam_paper_scale_sampled_pairs(torch):
    """Np=256, L=64, P=1024 (N=65,728), 16-QAM: every output is computed on the GPU; the
    oracle recomputes 96 sampled channel pairs exactly, and the full output is checked
    for exact conjugate symmetry S(l,k,-q) = conj S(k,l,q) up to rounding."""
    w = signals.fam_qam16_paper_scale()
    x, Np, L, P = w["x"], w["Np"], w["L"], w["P"]
    a = orc.hamming_window(Np)
    got_t = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a))
    g = np.random.default_rng(5)
    kh = np.concatenate([g.integers(0, Np, 90), [0, 255, 128, 0, 255, 7]])
    lh = np.concatenate([g.integers(0, Np, 90), [0, 255, 128, 255, 0, 7]])
    ref = orc.fam_pairs(x, a, Np, L, P, kh, lh)
    got = got_t[torch.from_numpy(kh).cuda(), torch.from_numpy(lh).cuda()].cpu().numpy()
    smax = float(np.max(np.abs(got_t[torch.arange(Np), torch.arange(Np), P // 2].cpu().numpy())))
    assert float(np.max(np.abs(got - ref))) / smax <= FP32_TOL
    qh = torch.remainder(P - torch.arange(P, device="cuda"), P)
    flipped = got_t.transpose(0, 1)[:, :, qh]
    err = (flipped - got_t.conj()).abs().max().item()
    assert err / got_t.abs().max().item() <= FP32_TOL


# ----------------------------------------------------------------------------- SSCA
@pytest.mark.parametrize("schedule", ["auto", "stages"])
@pytest.mark.parametrize("N,Np", [
    (1 << 12, 16), (1 << 12, 256), (1 << 13, 32), (1 << 14, 64), (1 << 15, 128), (1 << 17, 32),
])
def test_ssca_matches_oracle(torch, N, Np, schedule):
    x = signals.modulated("qpsk", N, 4, 0.1, 5.0, seed=2000 + Np)
    a = orc.hamming_window(Np)
    ref = orc.ssca(x, a, Np)
    got = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), schedule=schedule).cpu().numpy()
    binding.scd_check_device()
    assert _rel(got, ref) <= FP32_TOL


def test_ssca_64k_config_full(torch):
    """N=2^16, Np=256, QPSK RRC 0.35 at 5 dB: full element-wise comparison."""
    w = signals.ssca_qpsk_64k()
    x, Np = w["x"], w["Np"]
    a = orc.hamming_window(Np)
    ref = orc.ssca(x, a, Np)
    got = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a)).cpu().numpy()
    assert _rel(got, ref) <= FP32_TOL


@pytest.mark.parametrize("schedule", ["auto", "stages"])
def test_ssca_1m_config_sampled_channels(torch, schedule):
    """N=2^20, Np=256, BPSK+QPSK mixture at 0 dB: every channel is computed on the GPU;
    the oracle recomputes 5 full channel rows (2^20 bins each)."""
    w = signals.ssca_mixture_1m()
    x, Np = w["x"], w["Np"]
    N = x.shape[0]
    a = orc.hamming_window(Np)
    got_t = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), schedule=schedule)
    binding.scd_check_device()
    ch = np.array([0, 97, 128, 200, 255])
    ref = orc.ssca(x, a, Np, channels=ch, chunk=1 << 16)
    got = got_t[torch.from_numpy(ch).cuda()].cpu().numpy()
    smax = got_t.abs().max().item()
    assert float(np.max(np.abs(got - ref))) / smax <= FP32_TOL
    assert abs(np.max(np.abs(ref)) - np.max(np.abs(got))) / smax <= FP32_TOL
    del got_t
    torch.cuda.empty_cache()


# ----------------------------------------------------------------------------- maps
@pytest.mark.parametrize("Np,L,P,power", [(32, 8, 32, 1), (64, 16, 128, 2), (16, 2, 64, 1)])
def test_fam_map_matches_oracle(torch, Np, L, P, power):
    N = (P - 1) * L + Np
    x = signals.modulated("qpsk", N, 4, -0.1, 8.0, seed=3000 + P)
    a = orc.hamming_window(Np)
    S = orc.fam(x, a, Np, L, P)
    S_dev = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a))
    got = binding.scd_fam_map(S_dev, Np, L, P, power=power).cpu().numpy()
    ref = orc.fam_map(S, Np, L, P, power=power)
    assert _rel(got, ref) <= FP32_TOL * power
    assert np.array_equal(got == 0, ref == 0)


@pytest.mark.parametrize("N,Np,power", [(1 << 12, 32, 1), (1 << 13, 16, 2)])
def test_ssca_map_matches_oracle(torch, N, Np, power):
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=4000 + N, pulse="rect")
    a = orc.hamming_window(Np)
    S = orc.ssca(x, a, Np)
    S_dev = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a))
    got = binding.scd_ssca_map(S_dev, N, Np, power=power).cpu().numpy()
    ref = orc.ssca_map(S, N, Np, power=power)
    assert _rel(got, ref) <= FP32_TOL * power
    assert np.array_equal(got == 0, ref == 0)


def test_map_of_exact_oracle_input_is_exact(torch):
    """Feeding the oracle's own S (rounded to complex64) to the GPU map: the map is a pure
    index permutation plus |.|, so it matches the oracle's map of the same complex64 data
    to float32 rounding, and the zero pattern is identical."""
    Np, L, P = 16, 4, 32
    x = signals.awgn((P - 1) * L + Np, seed=77)
    S = orc.fam(x, orc.hamming_window(Np), Np, L, P).astype(np.complex64)
    got = binding.scd_fam_map(_dev(torch, S), Np, L, P).cpu().numpy()
    ref = orc.fam_map(S.astype(np.complex128), Np, L, P)
    assert _rel(got, ref) < 1e-6
    assert np.array_equal(got == 0, ref == 0)


# ----------------------------------------------------------------------------- maximum sizes
@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_fam_maximum_size_sampled_pairs(torch, precision):
    """The largest FAM the ABI takes at the largest Np: Np=256, P=16384 (L=64, N = 1,048,768;
    an 8.6 GB estimate): 12 sampled channel pairs recomputed by the oracle."""
    Np, L, P = 256, 64, 16384
    N = (P - 1) * L + Np
    x = signals.modulated("qpsk", N, 4, 0.07, 10.0, seed=9100)
    a = orc.hamming_window(Np)
    got_t = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), precision=precision)
    kh = np.array([0, 255, 128, 17, 200, 64, 3, 250, 128, 90, 0, 255])
    lh = np.array([0, 255, 128, 230, 5, 64, 3, 6, 127, 91, 255, 0])
    ref = orc.fam_pairs(x, a, Np, L, P, kh, lh)
    got = got_t[torch.from_numpy(kh).cuda(), torch.from_numpy(lh).cuda()].cpu().numpy()
    smax = float(np.max(np.abs(got_t[torch.arange(Np), torch.arange(Np), P // 2].cpu().numpy())))
    tol = FP32_TOL if precision == "fp32" else 1e-3
    assert float(np.max(np.abs(got - ref))) / smax <= tol
    del got_t
    torch.cuda.empty_cache()


@pytest.mark.parametrize("Np", [16, 64])
def test_ssca_maximum_length_small_np(torch, Np):
    """N = 2^20 with the smallest channel counts (single-pass 16-point channeliser at Np=16):
    4 full channel rows recomputed by the oracle."""
    N = 1 << 20
    x = signals.modulated("bpsk", N, 4, -0.12, 3.0, seed=9200 + Np)
    a = orc.hamming_window(Np)
    got_t = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a))
    binding.scd_check_device()
    ch = np.array([0, Np // 2 - 1, Np // 2, Np - 1])
    ref = orc.ssca(x, a, Np, channels=ch, chunk=1 << 16)
    got = got_t[torch.from_numpy(ch).cuda()].cpu().numpy()
    smax = got_t.abs().max().item()
    assert float(np.max(np.abs(got - ref))) / smax <= FP32_TOL
    del got_t
    torch.cuda.empty_cache()


@pytest.mark.parametrize("schedule", ["stages", "persistent"])
@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_ssca_2p19_both_schedules(torch, schedule, precision):
    """N = 2^19 (strip transform split 512 x 1024, the one size where the column pass is the
    shorter one): 4 full channel rows of both schedules and both forms against the oracle."""
    N, Np = 1 << 19, 64
    x = signals.modulated("qpsk", N, 4, 0.1, 5.0, seed=9300)
    a = orc.hamming_window(Np)
    got_t = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), schedule=schedule, precision=precision)
    binding.scd_check_device()
    ch = np.array([0, 17, Np // 2, Np - 1])
    ref = orc.ssca(x, a, Np, channels=ch, chunk=1 << 16)
    got = got_t[torch.from_numpy(ch).cuda()].cpu().numpy()
    smax = got_t.abs().max().item()
    tol = FP32_TOL if precision == "fp32" else 1e-3
    assert float(np.max(np.abs(got - ref))) / smax <= tol
    del got_t
    torch.cuda.empty_cache()


def test_fam_paper_match_dsss(torch):
    """The paper's own FAM configuration (Sec. IV: N = 2048 samples of DSSS BPSK at 10 dB,
    Np = 256, L = 64, P = 32; the 2048 samples zero-padded to (P - 1) L + Np = 2240): every
    cell against the oracle."""
    Np, L, P = 256, 64, 32
    x = np.zeros((P - 1) * L + Np, dtype=np.complex64)
    x[:2048] = signals.dsss_bpsk(2048, 10.0, seed=9400)
    a = orc.hamming_window(Np)
    got = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a)).cpu().numpy()
    ref = orc.fam(x, a, Np, L, P)
    assert _rel(got, ref) <= FP32_TOL
