"""Pins of the input normalisation (Algorithm 1 `Framing`: the norm kernel normalises the
input before decimation, Sec. III-A; mean power 1 or peak magnitude 1 over the samples the
estimate consumes)."""
import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import signals


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_scale_definitions():
    x = signals.modulated("qpsk", 5000, 4, 0.1, 5.0, seed=71)
    v = x[:4000].astype(np.complex128)
    s1 = orc.input_scale(x, 4000, 1)
    assert abs(np.mean(np.abs(v * s1) ** 2) - 1.0) < 1e-12
    s2 = orc.input_scale(x, 4000, 2)
    assert abs(np.max(np.abs(v * s2)) - 1.0) < 1e-12
    assert orc.input_scale(x, 4000, 0) == 1.0
    assert orc.input_scale(np.zeros(64, np.complex64), 64, 1) == 1.0


@pytest.mark.parametrize("mode", [1, 2])
def test_estimates_scale_quadratically(mode):
    """Both estimates are bilinear in the input (X conj(X), X_T conj(x)): multiplying the input
    by the normalisation factor s multiplies them by s^2."""
    Np, L, P = 16, 4, 32
    x = signals.modulated("bpsk", (P - 1) * L + Np + 9, 8, 0.05, 10.0, seed=72, pulse="rect")
    a = orc.hamming_window(Np)
    s = orc.input_scale(x, (P - 1) * L + Np, mode)
    assert _rel(orc.fam(x, a, Np, L, P, normalise=mode), orc.fam(x, a, Np, L, P) * s ** 2) < 1e-12
    N = 1024
    xs = signals.modulated("qpsk", N, 4, -0.1, 5.0, seed=73)
    s = orc.input_scale(xs, N, mode)
    assert _rel(orc.ssca(xs, a, Np, normalise=mode), orc.ssca(xs, a, Np) * s ** 2) < 1e-12


@pytest.mark.parametrize("mode", [1, 2])
def test_normalised_estimate_is_scale_invariant(mode):
    """Normalising removes the input's scale and phase: c x gives the same estimate as x."""
    Np, L, P = 16, 4, 32
    x = signals.modulated("qpsk", (P - 1) * L + Np, 4, 0.1, 8.0, seed=74)
    c = np.complex64(3.7 * np.exp(0.6j))
    a = orc.hamming_window(Np)
    y = (x * c).astype(np.complex64)
    # the products are rounded to complex64 like any input: agreement to float32 level
    assert _rel(orc.fam(y, a, Np, L, P, normalise=mode), orc.fam(x, a, Np, L, P, normalise=mode)) < 1e-6
    xs = signals.modulated("bpsk", 1024, 8, 0.05, 10.0, seed=75)
    ys = (xs * c).astype(np.complex64)
    assert _rel(orc.ssca(ys, a, Np, normalise=mode), orc.ssca(xs, a, Np, normalise=mode)) < 1e-6
