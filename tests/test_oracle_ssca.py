"""Pins of the SSCA oracle (Sec. II-C, Eq. Xg, Eq. II.B-SSCA_auto) against brute force,
closed forms and exact identities."""
import cmath
import math

import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import signals


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _bruteforce_ssca(x, a, Np):
    """Pure-Python loops over the definitions with floating-point angles:
    X_T(n,f_k) = sum_r a[r] x[n - Np/2 + r] exp(-i 2 pi k (n - Np/2 + r) / Np)   (zero outside)
    X_g(n,k)   = X_T(n,f_k) conj(x[n])
    S(k,q)     = sum_n X_g(n,k) exp(-i 2 pi q n / N)."""
    N = len(x)
    xs = [complex(v) for v in x]
    av = [float(v) for v in a]
    out = np.zeros((Np, N), dtype=np.complex128)
    for kh in range(Np):
        k = kh - Np // 2
        xg = []
        for n in range(N):
            acc = 0j
            for r in range(Np):
                m = n - Np // 2 + r
                if 0 <= m < N:
                    acc += av[r] * xs[m] * cmath.exp(-2j * math.pi * k * m / Np)
            xg.append(acc * xs[n].conjugate())
        for sh in range(N):
            q = sh - N // 2
            out[kh, sh] = sum(xg[n] * cmath.exp(-2j * math.pi * q * n / N) for n in range(N))
    return out


@pytest.mark.parametrize("N,Np", [(16, 4), (32, 8), (64, 16), (15, 4), (24, 8), (33, 16)])
def test_ssca_bruteforce_tiny(N, Np):
    x = signals.awgn(N, seed=100 + N)
    a = orc.hamming_window(Np)
    ref = _bruteforce_ssca(x, a, Np)
    for mode in ("direct", "fft"):
        assert _rel(orc.ssca(x, a, Np, mode=mode), ref) < 1e-12


@pytest.mark.parametrize("N,Np", [(1024, 16), (4096, 32), (2048, 256), (1000, 16), (3001, 64)])
def test_ssca_direct_matches_fft(N, Np):
    x = signals.modulated("qpsk", N, 4, 0.1, 5.0, seed=7)
    a = orc.hamming_window(Np)
    assert _rel(orc.ssca(x, a, Np, "direct"), orc.ssca(x, a, Np, "fft")) < 1e-11


def test_ssca_channel_subset_matches_full():
    N, Np = 4096, 64
    x = signals.modulated("bpsk", N, 4, -0.12, 3.0, seed=8)
    a = orc.hamming_window(Np)
    full = orc.ssca(x, a, Np)
    ch = np.array([0, 7, 32, 63])
    assert _rel(orc.ssca(x, a, Np, channels=ch, chunk=1000), full[ch]) < 1e-14


@pytest.mark.parametrize("N,Np", [(512, 16), (2048, 64), (1008, 16), (3 * 1024, 64)])
def test_ssca_alpha0_is_lag_windowed_correlogram(N, Np):
    """At q = -k N/Np (alpha = 0, f = k/Np):
    S = sum_{tau=-Np/2}^{Np/2-1} a[tau + Np/2] R(tau) W_Np^{k tau},
    R(tau) = sum_n x[n + tau] conj(x[n]) over the valid n (zero padding)."""
    x = signals.modulated("qpsk", N, 4, 0.1, 5.0, seed=12)
    a = orc.hamming_window(Np).astype(np.float64)
    xd = x.astype(np.complex128)
    S = orc.ssca(x, orc.hamming_window(Np), Np)
    taus = np.arange(-Np // 2, Np // 2)
    R = np.array([np.sum(xd[max(0, t) + 0: N + min(0, t)] * np.conj(xd[max(0, -t): N - max(0, t)]))
                  for t in taus])
    for kh in range(Np):
        k = kh - Np // 2
        ref = np.sum(a * R * np.exp(-2j * np.pi * k * taus / Np))
        sh = (N // 2 - k * (N // Np)) % N
        assert abs(S[kh, sh] - ref) < 1e-12 * np.max(np.abs(S))


def test_ssca_channel_shift_invariance():
    """x'[n] = x[n] exp(i 2 pi j n / Np): S'(k, q) = S(k - j, q + j N/Np) (cyclic)."""
    N, Np, j = 2048, 32, 3
    x = signals.modulated("qpsk", N, 4, 0.1, 5.0, seed=13)
    n = np.arange(N)
    xs = (x.astype(np.complex128) * np.exp(2j * np.pi * j * n / Np)).astype(np.complex64)
    a = orc.hamming_window(Np)
    S = orc.ssca(x, a, Np)
    S2 = orc.ssca(xs, a, Np)
    ki = np.mod(np.arange(Np) - j, Np)
    si = np.mod(np.arange(N) + j * N // Np, N)
    assert _rel(S2, S[ki][:, si]) < 1e-6


def test_ssca_scaling():
    N, Np = 1024, 16
    x = signals.awgn(N, seed=14)
    c = np.complex64(-1.5 + 0.5j)
    a = orc.hamming_window(Np)
    assert _rel(orc.ssca((x * c).astype(np.complex64), a, Np), abs(complex(c)) ** 2 * orc.ssca(x, a, Np)) < 1e-6


@pytest.mark.parametrize("N", [4096, 3200])
def test_ssca_two_tones_feature_location(N):
    """Two channel-centred tones A1 exp(i 2 pi f1 n) + A2 exp(i 2 pi f2 n): channel f1
    times conj(x) carries A1 conj(A2) exp(-i 2 pi f2 n), so the cell k = f1 Np,
    q = -f2 N (alpha = f1 - f2, f = (f1 + f2)/2) holds about N A1 conj(A2) sum(a).
    The phase pins which factor is conjugated (the sign convention of alpha), and the
    map puts the peak at that (f, alpha)."""
    Np = 32
    c1, c2 = 5, -3
    f1, f2 = c1 / Np, c2 / Np
    A1, A2 = 1.0, np.exp(1j * 0.7)
    x = signals.tones(N, [f1, f2], [A1, A2])
    a = orc.hamming_window(Np)
    S = orc.ssca(x, a, Np)
    asum = float(np.sum(a.astype(np.float64)))
    for (ca, fa, Aa), (cb, fb, Ab) in (((c1, f1, A1), (c2, f2, A2)), ((c2, f2, A2), (c1, f1, A1))):
        kh = ca + Np // 2
        sh = (int(round(-fb * N)) + N // 2) % N
        expect = N * Aa * np.conj(Ab) * asum
        assert abs(S[kh, sh] - expect) < 0.03 * abs(expect)
    M = orc.ssca_map(S, N, Np)
    alpha, f = f1 - f2, (f1 + f2) / 2
    assert M[int(math.floor((f + 0.5) * Np)), int(round(alpha * N + N))] > 0.9 * M.max()


def test_ssca_bpsk_symbol_rate_feature():
    """Complex BPSK, rectangular pulses, 8 samples/symbol: cycle frequency 1/8 appears."""
    N, Np = 8192, 32
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=31, pulse="rect")
    S = orc.ssca(x, orc.hamming_window(Np), Np)
    M = orc.ssca_map(S, N, Np)
    prof = M.max(axis=0)
    alpha = (np.arange(2 * N) - N) / N
    floor = np.median(prof[np.abs(alpha) > 0.02])
    for a0 in (1 / 8, -1 / 8):
        i = int(round(a0 * N + N))
        assert prof[i - 3:i + 4].max() > 5 * floor


def test_ssca_white_noise_floor():
    """White noise: |S| off alpha = 0 / |S| on alpha = 0 ~ 1/sqrt(N/Np)."""
    N, Np = 8192, 32
    x = signals.awgn(N, seed=33)
    S = np.abs(orc.ssca(x, orc.hamming_window(Np), Np))
    on = np.mean([S[kh, (N // 2 - (kh - Np // 2) * (N // Np)) % N] for kh in range(Np)])
    off = np.mean(S)
    assert off / on < 3.0 / math.sqrt(N / Np)


def test_ssca_odd_length_zero_bin():
    """A constant input: channel k = 0 sees X_T(n, 0) = sum(a) away from the edges, so
    X_g(n, 0) is constant there and its strip transform peaks in the zero bin q = 0,
    stored at floor(N/2) for an odd N as well (a wrong centre would move the peak)."""
    N, Np = 2049, 16
    x = signals.tones(N, [0.0], [1.0])
    S = np.abs(orc.ssca(x, orc.hamming_window(Np), Np))
    assert int(np.argmax(S[Np // 2])) == N // 2
    assert S[Np // 2, N // 2] > 50 * np.median(S[Np // 2])


def test_ssca_map_needs_np_to_divide_n():
    with pytest.raises(ValueError):
        orc.ssca_map_coords(3000, 64)
