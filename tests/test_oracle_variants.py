"""Pins of the cross and conjugate estimates and of the alpha profiles.

The cross estimate pairs the demodulates of two signals (Sec. II-A, Eq. II.A-SCD
function, X_T(r, f1) Y*_T(r, f2)); the SSCA multiplies the demodulate by the conjugated
second signal (Sec. II-C).  The conjugate estimate drops that conjugation.  The alpha
profile is the largest |S| over f for every cycle frequency of the map (the feature the
paper's RFML motivation extracts, Sec. I).  Each pin below comes from brute force or an
identity that the oracle's code does not use.
"""
import cmath
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import signals


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _bruteforce_fam(x, y, a, Np, L, P, conjugate):
    """Triple sum with floating-point angles:
    cross:     sum_p sum_n sum_n' a[n] a[n'] x[pL+n] conj(y[pL+n'])
               exp(-i2pi (k(pL+n) - l(pL+n'))/Np) exp(-i2pi q p/P)
    conjugate: sum_p sum_n sum_n' a[n] a[n'] x[pL+n] y[pL+n']
               exp(-i2pi (k(pL+n) + l(pL+n'))/Np) exp(-i2pi q p/P)"""
    xs = [complex(v) for v in x]
    ys = [complex(v) for v in y]
    av = [float(v) for v in a]
    sgn = 1 if conjugate else -1
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
                        yv = ys[p * L + n2] if conjugate else ys[p * L + n2].conjugate()
                        acc += (av[n] * av[n2] * xs[p * L + n] * yv
                                * cmath.exp(-2j * math.pi * (k * (p * L + n) + sgn * l * (p * L + n2)) / Np))
                z.append(acc)
            for qh in range(P):
                q = qh - P // 2
                out[kh, lh, qh] = sum(z[p] * cmath.exp(-2j * math.pi * q * p / P) for p in range(P))
    return out


def _bruteforce_ssca(x, y, a, Np, conjugate):
    """Loops over the definitions with floating-point angles:
    X_T(n,k) = sum_r a[r] x[n-Np/2+r] exp(-i2pi k (n-Np/2+r)/Np) (zero outside),
    X_g = X_T(n,k) conj(y[n]) (cross) or X_T(n,k) y[n] (conjugate),
    S(k,q) = sum_n X_g(n,k) exp(-i2pi q n/N)."""
    N = len(x)
    xs = [complex(v) for v in x]
    ys = [complex(v) for v in y]
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
            xg.append(acc * (ys[n] if conjugate else ys[n].conjugate()))
        for sh in range(N):
            q = sh - N // 2
            out[kh, sh] = sum(xg[n] * cmath.exp(-2j * math.pi * q * n / N) for n in range(N))
    return out


# ----------------------------------------------------------------------------- brute force
@pytest.mark.parametrize("conjugate", [False, True])
@pytest.mark.parametrize("Np,L,P", [(4, 1, 8), (8, 2, 8)])
def test_fam_cross_and_conjugate_bruteforce(Np, L, P, conjugate):
    N = (P - 1) * L + Np
    x = signals.awgn(N, seed=31 + Np)
    y = signals.awgn(N, seed=37 + Np)
    a = orc.hamming_window(Np)
    ref = _bruteforce_fam(x, y, a, Np, L, P, conjugate)
    for mode in ("direct", "fft"):
        assert _rel(orc.fam(x, a, Np, L, P, mode=mode, y=y, conjugate=conjugate), ref) < 1e-12
    kh, lh = np.array([0, 3, Np - 1]), np.array([Np - 1, 3, 1])
    assert _rel(orc.fam_pairs(x, a, Np, L, P, kh, lh, y=y, conjugate=conjugate), ref[kh, lh]) < 1e-12


@pytest.mark.parametrize("conjugate", [False, True])
@pytest.mark.parametrize("N,Np", [(16, 4), (32, 8)])
def test_ssca_cross_and_conjugate_bruteforce(N, Np, conjugate):
    x = signals.awgn(N, seed=41 + N)
    y = signals.awgn(N, seed=43 + N)
    a = orc.hamming_window(Np)
    ref = _bruteforce_ssca(x, y, a, Np, conjugate)
    for mode in ("direct", "fft"):
        assert _rel(orc.ssca(x, a, Np, mode=mode, y=y, conjugate=conjugate), ref) < 1e-12


# ----------------------------------------------------------------------------- identities
def test_fam_cross_with_itself_is_auto():
    Np, L, P = 16, 4, 32
    x = signals.modulated("qpsk", (P - 1) * L + Np, 4, 0.1, 10.0, seed=51)
    a = orc.hamming_window(Np)
    assert _rel(orc.fam(x, a, Np, L, P, y=x.copy()), orc.fam(x, a, Np, L, P)) < 1e-15


def test_fam_cross_hermitian_swap():
    """S_xy(k, l, q) = conj(S_yx(l, k, -q)): swapping the signals conjugates the product
    and reverses the P-point transform's frequency axis."""
    Np, L, P = 16, 4, 32
    N = (P - 1) * L + Np
    x = signals.modulated("bpsk", N, 8, 0.05, 5.0, seed=52)
    y = signals.modulated("qpsk", N, 4, -0.1, 5.0, seed=53)
    a = orc.hamming_window(Np)
    Sxy = orc.fam(x, a, Np, L, P, y=y)
    Syx = orc.fam(y, a, Np, L, P, y=x)
    qneg = np.mod(P - np.arange(P), P)                        # stored index of -q
    assert _rel(np.conj(Syx.transpose(1, 0, 2)[:, :, qneg]), Sxy) < 1e-12


def test_fam_conjugate_is_cross_with_conjugated_partner():
    """X(p,k) Y(p,l) = X(p,k) conj(Z(p,-l)) with Z the channeliser output of conj(y)
    (the window is real and the down-conversion is Np-periodic in the channel), so the
    conjugate estimate is the cross estimate against conj(y) with the l axis reversed."""
    Np, L, P = 32, 8, 32
    N = (P - 1) * L + Np
    x = signals.modulated("bpsk", N, 8, 0.05, 10.0, seed=54, pulse="rect")
    y = signals.modulated("qpsk", N, 4, 0.12, 10.0, seed=55)
    a = orc.hamming_window(Np)
    conj = orc.fam(x, a, Np, L, P, y=y, conjugate=True)
    cross = orc.fam(x, a, Np, L, P, y=np.conj(y))
    lrev = np.mod(Np - np.arange(Np), Np)                      # stored index of -l
    assert _rel(cross[:, lrev, :], conj) < 1e-12


def test_ssca_conjugate_is_cross_with_conjugated_partner():
    N, Np = 2048, 32
    x = signals.modulated("bpsk", N, 4, 0.07, 10.0, seed=56)
    y = signals.modulated("qpsk", N, 4, -0.05, 10.0, seed=57)
    a = orc.hamming_window(Np)
    assert _rel(orc.ssca(x, a, Np, y=np.conj(y)), orc.ssca(x, a, Np, y=y, conjugate=True)) < 1e-15


# ----------------------------------------------------------------------------- features
def _alpha_index(alpha, scale):
    return int(round(alpha * scale + scale))


def test_fam_conjugate_feature_at_twice_the_carrier():
    """Complex BPSK s[n] e^{i 2 pi fc n} with real symbols: E[x^2] oscillates at 2 fc, so the
    conjugate estimate has its strongest feature at alpha = 2 fc (f = 0), which the
    non-conjugate estimate of the same complex signal does not have; QPSK of the same
    power (E[s^2] = 0) shows only its estimation noise there."""
    Np, L, P = 32, 8, 256
    N = (P - 1) * L + Np
    fc = 0.1
    a = orc.hamming_window(Np)
    PL = P * L
    i2 = _alpha_index(2 * fc, PL)
    bpsk = signals.modulated("bpsk", N, 8, fc, 15.0, seed=58, pulse="rect")
    prof_c = orc.fam_alpha_profile(orc.fam(bpsk, a, Np, L, P, conjugate=True), Np, L, P, conjugate=True)
    prof_n = orc.fam_alpha_profile(orc.fam(bpsk, a, Np, L, P), Np, L, P)
    assert abs(int(np.argmax(prof_c)) - i2) <= 2
    floor_n = np.median(prof_n[prof_n > 0])
    assert prof_n[i2 - 2:i2 + 3].max() < 5 * floor_n
    qpsk = signals.modulated("qpsk", N, 8, fc, 15.0, seed=59, pulse="rect")
    prof_q = orc.fam_alpha_profile(orc.fam(qpsk, a, Np, L, P, conjugate=True), Np, L, P, conjugate=True)
    assert prof_q[i2 - 2:i2 + 3].max() < 0.4 * prof_c[i2 - 2:i2 + 3].max()


def test_ssca_conjugate_feature_at_twice_the_carrier():
    N, Np = 1 << 13, 32
    fc = -0.12
    a = orc.hamming_window(Np)
    x = signals.modulated("bpsk", N, 8, fc, 15.0, seed=60, pulse="rect")
    prof = orc.ssca_alpha_profile(orc.ssca(x, a, Np, conjugate=True), N, Np)
    assert abs(int(np.argmax(prof)) - _alpha_index(2 * fc, N)) <= 2


# ----------------------------------------------------------------------------- profiles
def _profile_by_loops(S, alpha_of_cell, n_alpha, cells):
    prof = np.zeros(n_alpha)
    for c in cells:
        i = alpha_of_cell(*c)
        if 0 <= i < n_alpha:
            prof[i] = max(prof[i], abs(S[c]))
    return prof


@pytest.mark.parametrize("conjugate", [False, True])
def test_fam_alpha_profile_by_loops(conjugate):
    """Per cell alpha = (f_k -+ f_l) + q/(PL) written out from Sec. II-B-2 (sign + for the
    conjugate estimate), band |q| < PL/Np kept as in Algorithm 1's FFT2 output, alpha in
    [-1, 1): the largest |S| per alpha bin."""
    Np, L, P = 16, 4, 32
    N = (P - 1) * L + Np
    x = signals.modulated("qpsk", N, 4, 0.1, 10.0, seed=61)
    a = orc.hamming_window(Np)
    S = orc.fam(x, a, Np, L, P, conjugate=conjugate)
    PL, Q = P * L, P * L // Np
    sgn = 1 if conjugate else -1

    def alpha_bin(kh, lh, qh):
        k, l, q = kh - Np // 2, lh - Np // 2, qh - P // 2
        if not -Q <= q < Q:
            return -1
        alpha = Fr(k, Np) + sgn * Fr(l, Np) + Fr(q, PL)
        return int(alpha * PL) + PL

    cells = [(kh, lh, qh) for kh in range(Np) for lh in range(Np) for qh in range(P)]
    ref = _profile_by_loops(S, alpha_bin, 2 * PL, cells)
    got = orc.fam_alpha_profile(S, Np, L, P, conjugate=conjugate)
    assert np.allclose(got, ref, rtol=1e-15, atol=0)


def test_ssca_alpha_profile_by_loops():
    """alpha = k/Np + q/N (Sec. II-C) per cell; the largest |S| per alpha bin."""
    N, Np = 256, 16
    x = signals.modulated("bpsk", N, 4, 0.05, 10.0, seed=62)
    S = orc.ssca(x, orc.hamming_window(Np), Np)
    cells = [(kh, sh) for kh in range(Np) for sh in range(N)]
    ref = _profile_by_loops(S, lambda kh, sh: (kh - Np // 2) * (N // Np) + (sh - N // 2) + N, 2 * N, cells)
    assert np.allclose(orc.ssca_alpha_profile(S, N, Np), ref, rtol=1e-15, atol=0)


def test_fam_conjugate_map_injective():
    for Np, L, P in [(16, 4, 16), (32, 8, 32), (16, 2, 64)]:
        kh, lh, qh, fh, ah = orc.fam_map_coords(Np, L, P, conjugate=True)
        Q = P * L // Np
        assert kh.shape[0] == Np * Np * 2 * Q - Q              # the Q cells with alpha < -1 dropped
        assert fh.min() >= 0 and fh.max() < 2 * Np and ah.min() >= 0 and ah.max() < 2 * P * L
        cells = fh * (2 * P * L) + ah
        assert np.unique(cells).shape[0] == cells.shape[0]
