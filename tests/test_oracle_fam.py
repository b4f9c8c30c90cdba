"""Pins of the FAM oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper (Sec. II-B, Eq. II.B-complex_demodulate_final,
Eq. II.B-SCD_function_FAM, Algorithm 1) or the mathematical identity it relies on.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import signals


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _bruteforce_fam(x, a, Np, L, P):
    """Triple sum straight from Eq. II.B-complex_demodulate_final and
    Eq. II.B-SCD_function_FAM, with angles computed in floating point (no integer
    reduction), pure Python loops:
        S(k,l,q) = sum_p sum_n sum_n' a[n] a[n'] x[pL+n] conj(x[pL+n'])
                   * exp(-i 2 pi (k (pL+n) - l (pL+n')) / Np) * exp(-i 2 pi q p / P)
    """
    xs = [complex(v) for v in x]
    av = [float(v) for v in a]
    out = np.zeros((Np, Np, P), dtype=np.complex128)
    for kh in range(Np):
        k = kh - Np // 2
        for lh in range(Np):
            l = lh - Np // 2
            z = []
            for p in range(P):
                acc = 0j
                for n in range(Np):
                    for n2 in range(Np):
                        acc += (av[n] * av[n2] * xs[p * L + n] * xs[p * L + n2].conjugate()
                                * cmath.exp(-2j * math.pi * (k * (p * L + n) - l * (p * L + n2)) / Np))
                z.append(acc)
            for qh in range(P):
                q = qh - P // 2
                out[kh, lh, qh] = sum(z[p] * cmath.exp(-2j * math.pi * q * p / P) for p in range(P))
    return out


@pytest.mark.parametrize("Np,L,P", [(4, 1, 8), (8, 2, 16), (4, 1, 5), (4, 2, 6), (8, 2, 7)])
def test_fam_bruteforce_tiny(Np, L, P):
    N = (P - 1) * L + Np
    x = signals.awgn(N, seed=11 + Np)
    a = orc.hamming_window(Np)
    ref = _bruteforce_fam(x, a, Np, L, P)
    for mode in ("direct", "fft"):
        assert _rel(orc.fam(x, a, Np, L, P, mode=mode), ref) < 1e-12


@pytest.mark.parametrize("Np,L,P", [(16, 4, 32), (32, 8, 64), (64, 16, 16), (16, 4, 33), (32, 8, 100)])
def test_fam_direct_matches_fft(Np, L, P):
    N = (P - 1) * L + Np + 5
    x = signals.modulated("qpsk", N, 4, 0.07, 10.0, seed=3)
    a = orc.hamming_window(Np)
    assert _rel(orc.fam(x, a, Np, L, P, "direct"), orc.fam(x, a, Np, L, P, "fft")) < 1e-12


def test_fam_pairs_match_full():
    Np, L, P = 32, 8, 32
    x = signals.fam_small_bpsk()["x"]
    a = orc.hamming_window(Np)
    S = orc.fam(x, a, Np, L, P)
    kh = np.array([0, 5, 31, 17])
    lh = np.array([3, 5, 0, 30])
    assert _rel(orc.fam_pairs(x, a, Np, L, P, kh, lh), S[kh, lh]) < 1e-14


def test_fam_alpha0_is_averaged_periodogram():
    """At alpha = 0 (k = l, q = 0) the down-conversion phases cancel and the FAM value is
    sum_p |DFT_Np(a x_p)[k]|^2, the unnormalised averaged periodogram."""
    Np, L, P = 32, 8, 32
    x = signals.fam_small_bpsk()["x"]
    a = orc.hamming_window(Np)
    S = orc.fam(x, a, Np, L, P)
    blocks = np.stack([x[p * L:p * L + Np].astype(np.complex128) * a for p in range(P)])
    pgram = np.sum(np.abs(np.fft.fft(blocks, axis=1)) ** 2, axis=0)      # natural order
    k = np.arange(-Np // 2, Np // 2)
    diag = np.array([S[kh, kh, P // 2] for kh in range(Np)])
    assert np.max(np.abs(diag.imag)) < 1e-12 * np.max(np.abs(diag))
    assert _rel(diag.real, pgram[np.mod(k, Np)]) < 1e-13


@pytest.mark.parametrize("P", [64, 50, 45])
def test_fam_alpha0_matches_scipy_welch(P):
    """Welch's PSD estimate (scipy) with the same window, segment length Np, hop L and
    P segments, scaled back to a raw sum: S(k,k,0) = welch * P * sum(a^2).  The zero bin
    is stored at floor(P/2) for any P."""
    signal = pytest.importorskip("scipy.signal")
    Np, L = 64, 16
    N = (P - 1) * L + Np
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=5, pulse="rect")
    a = orc.hamming_window(Np)
    S = orc.fam(x, a, Np, L, P)
    f, pxx = signal.welch(x.astype(np.complex128), fs=1.0, window=a.astype(np.float64), nperseg=Np,
                          noverlap=Np - L, detrend=False, return_onesided=False, scaling="density")
    ref = pxx * P * float(np.sum(a.astype(np.float64) ** 2))
    k = np.arange(-Np // 2, Np // 2)
    diag = np.array([S[kh, kh, P // 2].real for kh in range(Np)])
    assert _rel(diag, ref[np.mod(k, Np)]) < 1e-12


@pytest.mark.parametrize("P", [32, 31, 24])
def test_fam_conjugate_symmetry_exact(P):
    """S(l, k, -q) = conj(S(k, l, q)): swapping the pair conjugates z(p).  Bin q is stored
    at q + floor(P/2), so -q sits at 2 floor(P/2) - qh (mod P): P - qh for even P and
    P - 1 - qh for odd P, which pins where the zero bin of an odd size is stored."""
    Np, L = 32, 8
    x = signals.awgn((P - 1) * L + Np, seed=40 + P)
    S = orc.fam(x, orc.hamming_window(Np), Np, L, P)
    qh = np.arange(P)
    flipped = S.transpose(1, 0, 2)[:, :, np.mod(2 * (P // 2) - qh, P)]
    assert _rel(flipped, np.conj(S)) < 1e-14


def test_fam_channel_shift_invariance():
    """x'[n] = x[n] exp(i 2 pi j n / Np) moves every channel by j: S'(k,l,q) = S(k-j,l-j,q)
    (cyclically).  This only holds with the down-conversion factor of
    Eq. II.B-complex_demodulate_final in place."""
    Np, L, P, j = 32, 8, 32, 5
    x = signals.fam_small_bpsk()["x"]
    n = np.arange(x.shape[0])
    xs = (x.astype(np.complex128) * np.exp(2j * np.pi * j * n / Np)).astype(np.complex64)
    a = orc.hamming_window(Np)
    S = orc.fam(x, a, Np, L, P)
    S2 = orc.fam(xs, a, Np, L, P)
    idx = np.mod(np.arange(Np) - j, Np)
    # complex64 rounding of the shifted input is the only difference
    assert _rel(S2, S[idx][:, idx]) < 1e-6


def test_fam_scaling():
    Np, L, P = 16, 4, 16
    x = signals.awgn((P - 1) * L + Np, seed=9)
    c = np.complex64(0.5 - 2.0j)
    a = orc.hamming_window(Np)
    S = orc.fam(x, a, Np, L, P)
    S2 = orc.fam((x * c).astype(np.complex64), a, Np, L, P)
    assert _rel(S2, abs(complex(c)) ** 2 * S) < 1e-6


@pytest.mark.parametrize("Np,L,P", [(16, 4, 16), (32, 8, 32), (16, 2, 64), (16, 4, 12), (16, 16, 9)])
def test_fam_tones_closed_form(Np, L, P):
    """Closed form for x = sum_i A_i exp(i 2 pi c_i n / Np) (channel-centred tones):
    X(p,k) = sum_i A_i W_Np^{(k - c_i) p L} Ahat(k - c_i), Ahat(m) = sum_n a[n] W_Np^{m n},
    hence S(k,l,q) = P * sum_{i,j} A_i conj(A_j) Ahat(k-c_i) conj(Ahat(l-c_j)) whenever
    ((k-c_i) - (l-c_j)) P L / Np + q = 0 (mod P), and 0 otherwise."""
    cs = [3, -5, 0]
    amps = [1.0, 0.5 - 0.25j, 0.3j]
    N = (P - 1) * L + Np
    x = signals.tones(N, [c / Np for c in cs], amps)
    a = orc.hamming_window(Np).astype(np.float64)
    nn = np.arange(Np)

    def ahat(m):
        return np.sum(a * np.exp(-2j * np.pi * m * nn / Np))

    ref = np.zeros((Np, Np, P), dtype=np.complex128)
    for kh in range(Np):
        k = kh - Np // 2
        for lh in range(Np):
            l = lh - Np // 2
            for ci, Ai in zip(cs, amps):
                for cj, Aj in zip(cs, amps):
                    m = ((k - ci) - (l - cj)) * P * L // Np
                    q = (-m) % P                       # q = -m (mod P), in natural order
                    qs = q - P if q >= P - P // 2 else q   # signed: [-floor(P/2), P - floor(P/2))
                    ref[kh, lh, qs + P // 2] += P * Ai * np.conj(Aj) * ahat(k - ci) * np.conj(ahat(l - cj))
    S = orc.fam(x, orc.hamming_window(Np), Np, L, P)
    assert _rel(S, ref) < 2e-6                          # complex64 rounding of the tones


def test_fam_bpsk_cyclic_features():
    """Rectangular-pulse complex BPSK at 8 samples/symbol: the symbol rate 1/8 is a cycle
    frequency, so |S| at alpha = +-1/8 stands far above the white-noise floor."""
    Np, L, P = 32, 8, 256
    N = (P - 1) * L + Np
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=21, pulse="rect")
    S = orc.fam(x, orc.hamming_window(Np), Np, L, P)
    M = orc.fam_map(S, Np, L, P)
    alpha = (np.arange(2 * P * L) - P * L) / (P * L)
    prof = M.max(axis=0)                                # alpha profile
    floor = np.median(prof[np.abs(alpha) > 0.02])
    for a0 in (1 / 8, -1 / 8):
        i = int(round(a0 * P * L + P * L))
        assert prof[i - 2:i + 3].max() > 5 * floor
    assert prof[P * L] > 20 * floor                       # alpha = 0 (PSD)


def test_fam_real_bpsk_double_carrier_feature():
    """A real passband BPSK also has cycle frequencies at +-2 fc (conjugate feature folded
    into the non-conjugate SCD by the real signal)."""
    Np, L, P = 32, 8, 256
    N = (P - 1) * L + Np
    fc = 0.1
    x = signals.modulated("bpsk", N, 8, fc, 15.0, seed=22, pulse="rect", real=True)
    S = orc.fam(x, orc.hamming_window(Np), Np, L, P)
    M = orc.fam_map(S, Np, L, P)
    alpha = (np.arange(2 * P * L) - P * L) / (P * L)
    prof = M.max(axis=0)
    floor = np.median(prof[np.abs(alpha) > 0.02])
    for a0 in (2 * fc, -2 * fc):
        i = int(round(a0 * P * L + P * L))
        assert prof[i - 2:i + 3].max() > 5 * floor


def test_fam_white_noise_floor():
    """White noise: away from alpha = 0 the estimate is small, about sqrt(pi/4)/sqrt(P) of
    the alpha = 0 level on average; assert below 3/sqrt(P)."""
    Np, L, P = 32, 8, 256
    x = signals.awgn((P - 1) * L + Np, seed=23)
    S = np.abs(orc.fam(x, orc.hamming_window(Np), Np, L, P))
    on = np.mean([S[k, k, P // 2] for k in range(Np)])
    off = []
    for kh in range(Np):
        for lh in range(Np):
            if abs(kh - lh) >= 2:
                off.append(np.mean(S[kh, lh, P // 2 - P // 8:P // 2 + P // 8]))
    assert np.mean(off) / on < 3.0 / math.sqrt(P)
