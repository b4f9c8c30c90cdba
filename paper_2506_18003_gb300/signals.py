"""Seeded synthetic input signals (modulated waveforms in noise).

This module only draws inputs: symbols, pulse shaping, carrier offset and additive
white Gaussian noise.  It holds none of the SCD estimators' arithmetic and is the one
module that both the CUDA path's tests/benchmark and the FP64 oracle's tests consume.

Conventions: numpy Generator(PCG64(seed)); complex AWGN with variance sigma^2/2 per
component; SNR = mean signal power / noise power per sample; constellations at unit
average power; root-raised-cosine pulses from the textbook closed form, span 8 symbols,
unit energy; the carrier offset is applied as exp(i 2 pi fc n).  Everything is returned
as complex64.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20250618


def seed_for(config_index: int, signal_index: int = 0) -> int:
    """Seed of signal `signal_index` of workload `config_index`."""
    return BASE_SEED + 1000 * config_index + signal_index


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def rrc_taps(beta: float, sps: int, span: int = 8) -> np.ndarray:
    """Root-raised-cosine impulse response (closed form), span symbols long, unit energy."""
    t = np.arange(-span * sps // 2, span * sps // 2 + 1, dtype=np.float64) / sps
    h = np.empty_like(t)
    for i, ti in enumerate(t):
        if abs(ti) < 1e-12:
            h[i] = 1.0 - beta + 4.0 * beta / math.pi
        elif beta > 0 and abs(abs(ti) - 1.0 / (4.0 * beta)) < 1e-9:
            h[i] = (beta / math.sqrt(2.0)) * (
                (1 + 2 / math.pi) * math.sin(math.pi / (4 * beta))
                + (1 - 2 / math.pi) * math.cos(math.pi / (4 * beta)))
        else:
            num = math.sin(math.pi * ti * (1 - beta)) + 4 * beta * ti * math.cos(math.pi * ti * (1 + beta))
            den = math.pi * ti * (1 - (4 * beta * ti) ** 2)
            h[i] = num / den
    return h / np.sqrt(np.sum(h * h))


_CONSTELLATIONS = {
    "bpsk": np.array([1, -1], dtype=np.complex128),
    "qpsk": np.exp(1j * (np.pi / 4 + np.pi / 2 * np.arange(4))),
    "8psk": np.exp(1j * (np.pi / 4 * np.arange(8))),
    "16qam": np.array([(a + 1j * b) for a in (-3, -1, 1, 3) for b in (-3, -1, 1, 3)]) / np.sqrt(10.0),
}


def _symbols(g, kind, count):
    c = _CONSTELLATIONS[kind]
    return c[g.integers(0, c.shape[0], size=count)]


def _shape(symbols, sps, pulse, beta):
    up = np.zeros(symbols.shape[0] * sps, dtype=np.complex128)
    up[::sps] = symbols
    if pulse == "rect":
        return np.convolve(up, np.ones(sps), mode="full")[: up.shape[0]]
    h = rrc_taps(beta, sps)
    y = np.convolve(up, h, mode="full")
    d = (h.shape[0] - 1) // 2
    return y[d:d + up.shape[0]]


def _awgn(g, n, power):
    s = math.sqrt(power / 2.0)
    return s * (g.standard_normal(n) + 1j * g.standard_normal(n))


def _finish(g, s, snr_db, real=False):
    p = float(np.mean(np.abs(s) ** 2)) if s.size else 1.0
    if snr_db is not None:
        noise = _awgn(g, s.shape[0], p / (10.0 ** (snr_db / 10.0)))
        if real:
            noise = noise.real * math.sqrt(2.0)
        s = s + noise
    return s.astype(np.complex64)


def modulated(kind: str, n: int, sps: int, fc: float, snr_db, seed: int,
              pulse: str = "rrc", beta: float = 0.35, real: bool = False) -> np.ndarray:
    """Linear digital modulation (bpsk/qpsk/8psk/16qam) of n samples.

    real=True returns the real passband waveform Re{s(n) exp(i 2 pi fc n)} (imaginary
    part zero), otherwise the complex signal shifted to fc.
    """
    g = rng(seed)
    nsym = n // sps + 16
    s = _shape(_symbols(g, kind, nsym), sps, pulse, beta)
    start = int(g.integers(0, sps))                     # random symbol timing
    s = s[start:start + n]
    s = s / math.sqrt(float(np.mean(np.abs(s) ** 2)))
    s = s * np.exp(2j * np.pi * fc * np.arange(n))
    if real:
        s = s.real.astype(np.complex128)
    return _finish(g, s, snr_db, real)


def am_dsb(n: int, fc: float, snr_db, seed: int, bandwidth: float = 0.02) -> np.ndarray:
    """Real low-pass Gaussian message (one-sided bandwidth `bandwidth`) on a carrier."""
    g = rng(seed)
    w = g.standard_normal(n + 256)
    taps = np.sinc(2 * bandwidth * (np.arange(257) - 128)) * np.hamming(257)
    m = np.convolve(w, taps, mode="same")[128:128 + n]
    m = m / math.sqrt(float(np.mean(m * m)))
    s = m * np.exp(2j * np.pi * fc * np.arange(n))
    return _finish(g, s, snr_db)


def awgn(n: int, seed: int, power: float = 1.0) -> np.ndarray:
    g = rng(seed)
    return _awgn(g, n, power).astype(np.complex64)


def tones(n: int, freqs, amps=None) -> np.ndarray:
    """Sum of complex exponentials sum_i amps[i] exp(i 2 pi freqs[i] n) (no noise)."""
    t = np.arange(n, dtype=np.float64)
    amps = np.ones(len(freqs)) if amps is None else amps
    s = sum(A * np.exp(2j * np.pi * f * t) for f, A in zip(freqs, amps))
    return np.asarray(s, dtype=np.complex64)


def m_sequence_31() -> np.ndarray:
    """Length-31 maximal-length sequence from the primitive polynomial x^5 + x^2 + 1,
    as +/-1 chips."""
    reg = [1, 0, 0, 0, 0]
    out = []
    for _ in range(31):
        out.append(reg[-1])
        fb = reg[4] ^ reg[1]
        reg = [fb] + reg[:-1]
    return 1.0 - 2.0 * np.array(out, dtype=np.float64)


def dsss_bpsk(n: int, snr_db, seed: int, samples_per_chip: int = 4) -> np.ndarray:
    """DSSS BPSK: one data bit per 31-chip m-sequence period, chip rate 1/samples_per_chip,
    rectangular chips (the accuracy signal recipe of Sec. IV-A, code choice ours)."""
    g = rng(seed)
    code = m_sequence_31()
    nbits = n // (31 * samples_per_chip) + 2
    bits = 1.0 - 2.0 * g.integers(0, 2, size=nbits)
    chips = (bits[:, None] * code[None, :]).ravel()
    s = np.repeat(chips, samples_per_chip)[:n].astype(np.complex128)
    return _finish(g, s, snr_db)


# ----------------------------------------------------------------------------- workloads
# Named workloads with the shapes of the evaluated configurations.

def fam_small_bpsk(seed: int | None = None) -> dict:
    """FAM, N=280 (Np=32, L=8, P=32): BPSK, rectangular pulses, 8 samples/symbol,
    carrier 0.05, 10 dB."""
    x = modulated("bpsk", 280, 8, 0.05, 10.0, seed_for(0) if seed is None else seed, pulse="rect")
    return dict(x=x, Np=32, L=8, P=32)


def ssca_qpsk_64k(seed: int | None = None) -> dict:
    """SSCA, N=2^16, Np=256: QPSK, RRC 0.35, 4 samples/symbol, carrier 0.1, 5 dB."""
    x = modulated("qpsk", 1 << 16, 4, 0.1, 5.0, seed_for(1) if seed is None else seed, beta=0.35)
    return dict(x=x, Np=256)


def fam_qam16_paper_scale(seed: int | None = None) -> dict:
    """FAM, N=65,728 (Np=256, L=64, P=1024): 16-QAM, RRC 0.25, 8 samples/symbol,
    SNR drawn uniformly in [0, 15] dB."""
    s = seed_for(2) if seed is None else seed
    snr = float(rng(s + 7).uniform(0.0, 15.0))
    x = modulated("16qam", 65728, 8, 0.0, snr, s, beta=0.25)
    return dict(x=x, Np=256, L=64, P=1024)


def ssca_mixture_1m(seed: int | None = None, n: int = 1 << 20) -> dict:
    """SSCA, N=2^20, Np=256: BPSK (4 sps, carrier -0.12) + QPSK (10 sps, carrier +0.2),
    equal power, 0 dB SNR."""
    s = seed_for(3) if seed is None else seed
    a = modulated("bpsk", n, 4, -0.12, None, s, beta=0.35).astype(np.complex128)
    b = modulated("qpsk", n, 10, 0.2, None, s + 1, beta=0.35).astype(np.complex128)
    y = (a + b) / math.sqrt(2.0)
    g = rng(s + 2)
    y = y + _awgn(g, n, float(np.mean(np.abs(y) ** 2)))
    return dict(x=y.astype(np.complex64), Np=256)


BATCH_KINDS = ("bpsk", "qpsk", "8psk", "16qam", "am_dsb", "awgn")


def batch_lengths(count: int = 512, seed: int | None = None, lo: int = 12, hi: int = 18) -> np.ndarray:
    """Signal lengths drawn log-uniformly in [2^lo, 2^hi]."""
    g = rng(seed_for(4) if seed is None else seed)
    return np.floor(2.0 ** g.uniform(lo, hi, size=count)).astype(np.int64)


def batch_signal(i: int, length: int, seed: int | None = None) -> np.ndarray:
    """Signal i of the mixed batch: modulation uniform over BATCH_KINDS, samples/symbol
    in {2,4,8,16}, carrier uniform in +/-0.25, SNR uniform in [-5, 15] dB, RRC 0.35."""
    s = seed_for(4, i + 1) if seed is None else seed
    g = rng(s)
    kind = BATCH_KINDS[int(g.integers(0, len(BATCH_KINDS)))]
    sps = int((2, 4, 8, 16)[int(g.integers(0, 4))])
    fc = float(g.uniform(-0.25, 0.25))
    snr = float(g.uniform(-5.0, 15.0))
    if kind == "awgn":
        return awgn(int(length), s + 500)
    if kind == "am_dsb":
        return am_dsb(int(length), fc, snr, s + 500)
    return modulated(kind, int(length), sps, fc, snr, s + 500, beta=0.35)
