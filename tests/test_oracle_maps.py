"""Pins of the (f, alpha) maps: injectivity, the round trip, agreement with the
SSCA_2DFFT mapping formula of Sec. III-B-1 and the alpha = 0 row of the FAM map, plus
the paper's printed parameter relations (tests/golden/paper_parameters.json)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import signals

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


@pytest.mark.parametrize("Np,L,P", [(16, 4, 16), (32, 8, 32), (16, 2, 64), (64, 16, 128), (16, 4, 12), (64, 16, 100)])
def test_fam_map_is_injective_and_inside_grid(Np, L, P):
    kh, lh, qh, fh, ah = orc.fam_map_coords(Np, L, P)
    Q = P * L // Np
    assert kh.shape[0] == Np * Np * 2 * Q
    assert fh.min() >= 0 and fh.max() < 2 * Np and ah.min() >= 0 and ah.max() < 2 * P * L
    cells = fh * (2 * P * L) + ah
    assert np.unique(cells).shape[0] == cells.shape[0]          # no cell written twice
    # round trip (fh, ah) -> (k, l, q): s = k + l, d = k - l has the parity of s and
    # q = (ah - PL) - d Q lies in [-Q, Q)
    s = fh - Np
    t = np.floor_divide(ah - P * L - (s & 1) * Q + Q, 2 * Q)
    d = 2 * t + (s & 1)
    q = ah - P * L - d * Q
    assert np.array_equal((s + d) // 2 + Np // 2, kh)
    assert np.array_equal((s - d) // 2 + Np // 2, lh)
    assert np.array_equal(q + P // 2, qh)
    # at q = 0, |f| + |alpha|/2 = max(|k|, |l|)/Np <= 1/2 (the principal diamond); the
    # kept band |q| <= Q widens that by at most Q/(2 P L) = 1/(2 Np)
    f = (fh - Np) / (2 * Np)
    alpha = (ah - P * L) / (P * L)
    assert np.all(np.abs(f) + np.abs(alpha) / 2 <= 0.5 + 0.5 / Np + 1e-12)


@pytest.mark.parametrize("N,Np", [(64, 16), (4096, 32), (1 << 12, 256), (3 * 1024, 32), (48, 16)])
def test_ssca_map_is_injective_and_inside_grid(N, Np):
    kh, sh, fh, ah = orc.ssca_map_coords(N, Np)
    assert fh.min() >= 0 and fh.max() < Np and ah.min() >= 0 and ah.max() < 2 * N
    cells = fh * (2 * N) + ah
    assert np.unique(cells).shape[0] == cells.shape[0]
    # inverse: c = ah - N = k N/Np + q and fh = k + floor((N - c) Np / (2N))
    c = ah - N
    k = fh - np.floor_divide((N - c) * Np, 2 * N)
    assert np.array_equal(k + Np // 2, kh)
    assert np.array_equal(c - k * (N // Np) + N // 2, sh)


def test_ssca_map_matches_2dfft_mapping_formula():
    """Sec. III-B-1: f = k/(2Np) - (M1 m2' + m1' - N/2)/(2N), alpha = k/Np +
    (M1 m2' + m1' - N/2)/N, where M1 m2' + m1' is the stored bin index.  Exact
    rational arithmetic against our integer grid indices."""
    N, Np, M1 = 1 << 12, 64, 64
    kh, sh, fh, ah = orc.ssca_map_coords(N, Np)
    g = np.random.default_rng(1)
    for i in g.integers(0, kh.shape[0], size=2000):
        k = int(kh[i]) - Np // 2
        m2p, m1p = divmod(int(sh[i]), M1)
        idx = M1 * m2p + m1p
        f = Fraction(k, 2 * Np) - Fraction(idx - N // 2, 2 * N)
        alpha = Fraction(k, Np) + Fraction(idx - N // 2, N)
        assert alpha * N + N == int(ah[i])
        assert math.floor((f + Fraction(1, 2)) * Np) == int(fh[i])


def test_fam_map_alpha0_row_is_periodogram():
    """Even cells of the alpha = 0 column (fh = 2k + Np) hold |S(k,k,0)|, the averaged
    periodogram."""
    Np, L, P = 32, 8, 32
    x = signals.fam_small_bpsk()["x"]
    a = orc.hamming_window(Np)
    M = orc.fam_map(orc.fam(x, a, Np, L, P), Np, L, P)
    blocks = np.stack([x[p * L:p * L + Np].astype(np.complex128) * a for p in range(P)])
    pgram = np.sum(np.abs(np.fft.fft(blocks, axis=1)) ** 2, axis=0)
    for kh in range(Np):
        k = kh - Np // 2
        assert abs(M[2 * k + Np, P * L] - pgram[k % Np]) < 1e-12 * pgram.max()


def test_map_power_two_is_square():
    Np, L, P = 16, 4, 16
    x = signals.awgn((P - 1) * L + Np, seed=4)
    S = orc.fam(x, orc.hamming_window(Np), Np, L, P)
    assert np.allclose(orc.fam_map(S, Np, L, P, power=2), orc.fam_map(S, Np, L, P) ** 2, rtol=1e-13)


def test_paper_parameter_relations():
    """The printed tile counts follow from the parameter reading used here
    (L = Np/4, P = N/L; M1 = M2 = 1024 at N = 2^20)."""
    g = json.load(open(GOLDEN))
    w = g["fam_workload"]
    N, Np, F = w["N"], w["Np"], w["F"]
    L = Np // 4
    assert N // L == w["P"] == 4 * N // Np
    tiles = 1 + math.ceil(4 * N / (2 * F)) + (math.ceil(4 * N / (2 * F)) + math.ceil(4 * N / F)) + min(Np, 128)
    assert tiles == g["fam_tile_count"]["value"]
    s = g["ssca_workload"]
    assert s["M1"] * s["M2"] == s["N"]
    a_cdp = 1 + math.ceil(math.log2(s["Np"]) / 2)
    a_2d = math.ceil(math.log2(s["M1"]) / 2) + 1 + math.ceil(math.log2(s["M2"]) / 2)
    assert a_cdp + a_2d == g["ssca_tile_count"]["value"]
    t = g["fam_throughput"]
    assert abs(N / (t["interval_ms"] * 1e-3) / 1e6 - t["msamples_per_s"]) < 0.01
