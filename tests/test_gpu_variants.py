"""GPU parity of the cross and conjugate estimates, the conjugate FAM map and the alpha
profiles, through the C ABI, against the FP64 oracle on the same seeded inputs.
Gates: FP32 form max|dS|/max|S| <= 1e-5, split form <= 1e-3 (the stated targets)."""
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


def _pair(N, seed):
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=seed, pulse="rect")
    y = signals.modulated("qpsk", N, 4, -0.11, 5.0, seed=seed + 1)
    return x, y


# ----------------------------------------------------------------------------- FAM
@pytest.mark.parametrize("precision", ["fp32", "split"])
@pytest.mark.parametrize("cross,conjugate", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("Np,L,P,extra", [(32, 8, 32, 0), (16, 4, 256, 3), (64, 16, 128, 0), (256, 64, 16, 1)])
def test_fam_variants_match_oracle(torch, Np, L, P, extra, cross, conjugate, precision):
    N = (P - 1) * L + Np + extra
    x, y = _pair(N, 5000 + Np + P)
    a = orc.hamming_window(Np)
    ref = orc.fam(x, a, Np, L, P, y=y if cross else None, conjugate=conjugate)
    got = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), precision=precision,
                          y=_dev(torch, y) if cross else None, conjugate=conjugate).cpu().numpy()
    assert _rel(got, ref) <= TOL[precision]


def test_fam_conjugate_paper_scale_sampled_pairs(torch):
    """Np=256, L=64, P=1024, 16-QAM against a QPSK partner, conjugate cross estimate: the
    oracle recomputes 64 sampled channel pairs."""
    w = signals.fam_qam16_paper_scale()
    x, Np, L, P = w["x"], w["Np"], w["L"], w["P"]
    y = signals.modulated("qpsk", x.shape[0], 4, 0.1, 10.0, seed=5100)
    a = orc.hamming_window(Np)
    got_t = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), y=_dev(torch, y), conjugate=True)
    g = np.random.default_rng(6)
    kh = np.concatenate([g.integers(0, Np, 60), [0, 255, 128, 0]])
    lh = np.concatenate([g.integers(0, Np, 60), [0, 255, 128, 255]])
    ref = orc.fam_pairs(x, a, Np, L, P, kh, lh, y=y, conjugate=True)
    got = got_t[torch.from_numpy(kh).cuda(), torch.from_numpy(lh).cuda()].cpu().numpy()
    smax = got_t.abs().max().item()
    assert float(np.max(np.abs(got - ref))) / smax <= TOL["fp32"]


# ----------------------------------------------------------------------------- SSCA
@pytest.mark.parametrize("schedule", ["stages", "persistent"])
@pytest.mark.parametrize("cross,conjugate", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("N,Np", [(1 << 12, 32), (1 << 13, 128), (1 << 15, 16)])
def test_ssca_variants_match_oracle(torch, N, Np, cross, conjugate, schedule):
    x, y = _pair(N, 6000 + Np)
    a = orc.hamming_window(Np)
    ref = orc.ssca(x, a, Np, y=y if cross else None, conjugate=conjugate)
    got = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), schedule=schedule,
                           y=_dev(torch, y) if cross else None, conjugate=conjugate).cpu().numpy()
    binding.scd_check_device()
    assert _rel(got, ref) <= TOL["fp32"]


@pytest.mark.parametrize("cross,conjugate", [(True, False), (False, True)])
def test_ssca_variants_split(torch, cross, conjugate):
    N, Np = 1 << 14, 64
    x, y = _pair(N, 6100)
    a = orc.hamming_window(Np)
    ref = orc.ssca(x, a, Np, y=y if cross else None, conjugate=conjugate)
    got = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), precision="split",
                           y=_dev(torch, y) if cross else None, conjugate=conjugate).cpu().numpy()
    assert _rel(got, ref) <= TOL["split"]


def test_ssca_cross_1m_sampled_channels(torch):
    """N=2^20, Np=256 cross estimate (mixture against a QPSK partner): 3 full channel rows
    recomputed by the oracle."""
    w = signals.ssca_mixture_1m()
    x, Np = w["x"], w["Np"]
    N = x.shape[0]
    y = signals.modulated("qpsk", N, 4, 0.05, 5.0, seed=6200)
    a = orc.hamming_window(Np)
    got_t = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), y=_dev(torch, y))
    binding.scd_check_device()
    ch = np.array([0, 130, 255])
    ref = orc.ssca(x, a, Np, channels=ch, chunk=1 << 16, y=y)
    got = got_t[torch.from_numpy(ch).cuda()].cpu().numpy()
    smax = got_t.abs().max().item()
    assert float(np.max(np.abs(got - ref))) / smax <= TOL["fp32"]
    del got_t
    torch.cuda.empty_cache()


# ----------------------------------------------------------------------------- maps, profiles
@pytest.mark.parametrize("Np,L,P,power", [(32, 8, 32, 1), (64, 16, 128, 2), (16, 2, 64, 1)])
def test_fam_conjugate_map_matches_oracle(torch, Np, L, P, power):
    N = (P - 1) * L + Np
    x = signals.modulated("bpsk", N, 8, 0.1, 10.0, seed=6300 + P, pulse="rect")
    a = orc.hamming_window(Np)
    S = orc.fam(x, a, Np, L, P, conjugate=True)
    S_dev = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), conjugate=True)
    got = binding.scd_fam_map(S_dev, Np, L, P, power=power, conjugate=True).cpu().numpy()
    ref = orc.fam_map(S, Np, L, P, power=power, conjugate=True)
    assert _rel(got, ref) <= TOL["fp32"] * power
    assert np.array_equal(got == 0, ref == 0)


@pytest.mark.parametrize("conjugate", [False, True])
@pytest.mark.parametrize("Np,L,P,power", [(32, 8, 32, 1), (16, 4, 256, 2), (64, 16, 64, 1), (16, 1, 64, 1)])
def test_fam_alpha_profile_matches_oracle(torch, Np, L, P, power, conjugate):
    N = (P - 1) * L + Np
    x = signals.modulated("bpsk", N, 8, 0.07, 10.0, seed=6400 + P, pulse="rect")
    a = orc.hamming_window(Np)
    S = orc.fam(x, a, Np, L, P, conjugate=conjugate)
    S_dev = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), conjugate=conjugate)
    got = binding.scd_fam_alpha_profile(S_dev, Np, L, P, power=power, conjugate=conjugate).cpu().numpy()
    ref = orc.fam_alpha_profile(S, Np, L, P, power=power, conjugate=conjugate)
    assert _rel(got, ref) <= TOL["fp32"] * power
    assert np.array_equal(got == 0, ref == 0)


@pytest.mark.parametrize("N,Np,power", [(1 << 12, 32, 1), (1 << 13, 16, 2), (1 << 12, 256, 1)])
def test_ssca_alpha_profile_matches_oracle(torch, N, Np, power):
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=6500 + N + Np, pulse="rect")
    a = orc.hamming_window(Np)
    S = orc.ssca(x, a, Np)
    S_dev = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a))
    got = binding.scd_ssca_alpha_profile(S_dev, N, Np, power=power).cpu().numpy()
    ref = orc.ssca_alpha_profile(S, N, Np, power=power)
    assert _rel(got, ref) <= TOL["fp32"] * power
    assert np.array_equal(got == 0, ref == 0)


def test_profiles_of_exact_input_are_exact(torch):
    """On the oracle's own S rounded to complex64, the profile is a max of |.|, so it matches
    the oracle's profile of the same complex64 data to float32 rounding."""
    Np, L, P = 16, 4, 32
    x = signals.awgn((P - 1) * L + Np, seed=78)
    for conj in (False, True):
        S = orc.fam(x, orc.hamming_window(Np), Np, L, P, conjugate=conj).astype(np.complex64)
        got = binding.scd_fam_alpha_profile(_dev(torch, S), Np, L, P, conjugate=conj).cpu().numpy()
        ref = orc.fam_alpha_profile(S.astype(np.complex128), Np, L, P, conjugate=conj)
        assert _rel(got, ref) < 1e-6
    N = 1 << 12
    xs = signals.awgn(N, seed=79)
    S = orc.ssca(xs, orc.hamming_window(32), 32).astype(np.complex64)
    got = binding.scd_ssca_alpha_profile(_dev(torch, S), N, 32).cpu().numpy()
    assert _rel(got, orc.ssca_alpha_profile(S.astype(np.complex128), N, 32)) < 1e-6


def test_profiles_equal_map_column_maxima_at_full_size(torch):
    """Paper-scale sizes (FAM Np=256 L=64 P=1024; SSCA N=2^20 Np=256): every profile value
    equals the largest value of its map column (both from this library's kernels)."""
    w = signals.fam_qam16_paper_scale()
    x, Np, L, P = w["x"], w["Np"], w["L"], w["P"]
    S = binding.scd_fam(_dev(torch, x), Np, L, P, conjugate=False)
    for conj in (False, True):
        if conj:
            S = binding.scd_fam(_dev(torch, x), Np, L, P, out=S, conjugate=True)
        M = binding.scd_fam_map(S, Np, L, P, conjugate=conj)
        prof = binding.scd_fam_alpha_profile(S, Np, L, P, conjugate=conj)
        assert torch.equal(prof, M.amax(dim=0))
        del M
    del S
    m = signals.ssca_mixture_1m()
    N = m["x"].shape[0]
    S = binding.scd_ssca(_dev(torch, m["x"]), m["Np"])
    M = binding.scd_ssca_map(S, N, m["Np"])
    prof = binding.scd_ssca_alpha_profile(S, N, m["Np"])
    assert torch.equal(prof, M.amax(dim=0))
    del S, M
    torch.cuda.empty_cache()


# ----------------------------------------------------------------------------- input normalisation
@pytest.mark.parametrize("precision", ["fp32", "split"])
@pytest.mark.parametrize("normalise,mode", [("power", 1), ("peak", 2)])
def test_fam_normalised_matches_oracle(torch, normalise, mode, precision):
    Np, L, P = 32, 8, 64
    N = (P - 1) * L + Np + 11                                 # the tail beyond the consumed samples
    x = (signals.modulated("qpsk", N, 4, 0.08, 6.0, seed=6600) * np.complex64(7.5)).astype(np.complex64)
    a = orc.hamming_window(Np)
    ref = orc.fam(x, a, Np, L, P, normalise=mode)
    got = binding.scd_fam(_dev(torch, x), Np, L, P, window=_dev(torch, a), precision=precision,
                          normalise=normalise).cpu().numpy()
    assert _rel(got, ref) <= TOL[precision]


@pytest.mark.parametrize("schedule", ["stages", "persistent"])
@pytest.mark.parametrize("normalise,mode", [("power", 1), ("peak", 2)])
def test_ssca_normalised_matches_oracle(torch, normalise, mode, schedule):
    N, Np = 1 << 13, 64
    x = (signals.modulated("bpsk", N, 8, -0.05, 6.0, seed=6700, pulse="rect") * np.complex64(0.03)).astype(np.complex64)
    a = orc.hamming_window(Np)
    ref = orc.ssca(x, a, Np, normalise=mode)
    got = binding.scd_ssca(_dev(torch, x), Np, window=_dev(torch, a), schedule=schedule,
                           normalise=normalise).cpu().numpy()
    binding.scd_check_device()
    assert _rel(got, ref) <= TOL["fp32"]
