"""Pins of the Dolph-Chebyshev window (the `chebwin[Np]` of Algorithms 1 and 2) against
scipy's chebwin, a library routine, and against the window's defining properties."""
import numpy as np
import pytest

from oracle import scd_oracle as orc


@pytest.mark.parametrize("Np", [16, 31, 32, 64, 100, 128, 256])
@pytest.mark.parametrize("atten", [50.0, 80.0, 100.0])
def test_chebyshev_matches_scipy(Np, atten):
    windows = pytest.importorskip("scipy.signal.windows")
    ref = windows.chebwin(Np, at=atten, sym=True)
    got = orc.chebyshev_window64(Np, atten)
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("Np,atten", [(64, 60.0), (256, 100.0)])
def test_chebyshev_equiripple_sidelobes(Np, atten):
    """Every sidelobe of the window's spectrum lies atten dB below the main lobe (equiripple:
    the largest sidelobe equals the bound to a part in 10^6) and the window is symmetric."""
    w = orc.chebyshev_window64(Np, atten)
    assert np.allclose(w, w[::-1], rtol=0, atol=1e-14)
    spec = np.abs(np.fft.fft(w, 64 * Np))
    spec /= spec[0]
    x0 = np.cosh(np.arccosh(10 ** (atten / 20)) / (Np - 1))
    edge = np.arccos(1 / x0) / np.pi          # main-lobe half width in cycles/sample (cos(pi f) x0 = 1)
    f = np.arange(spec.shape[0]) / spec.shape[0]
    side = spec[(f > edge * 1.0001) & (f < 1 - edge * 1.0001)]
    assert abs(20 * np.log10(side.max()) + atten) < 1e-4


def test_chebyshev_float32_bits():
    w = orc.chebyshev_window(64, 100.0)
    assert w.dtype == np.float32 and w.max() == np.float32(1.0)


# ----------------------------------------------------------------------------- Hamming
# The default window (window = NULL on the C ABI) is the symmetric Hamming window
# a[n] = 0.54 - 0.46 cos(2 pi n / (Np - 1)).  These pins fail for the periodic variant
# (denominator Np), for a swapped pair of coefficients and for a sign slip.

@pytest.mark.parametrize("Np", [16, 32, 64, 128, 256])
def test_hamming_matches_scipy(Np):
    windows = pytest.importorskip("scipy.signal.windows")
    ref = windows.hamming(Np, sym=True)
    got = orc.hamming_window(Np)
    assert got.dtype == np.float32
    # one float32 rounding of the same FP64 values: within half an ulp of numbers <= 1
    assert np.max(np.abs(got.astype(np.float64) - ref)) <= 2.0 ** -24


@pytest.mark.parametrize("Np", [16, 64, 256])
def test_hamming_closed_forms(Np):
    """Endpoints 0.54 - 0.46 = 0.08 at both ends (a periodic window would not return to 0.08 at
    n = Np - 1), exact symmetry a[n] = a[Np - 1 - n], the largest value at the two middle samples
    0.54 + 0.46 cos(pi / (Np - 1)), and the sum 0.54 Np - 0.46 (the cosines over n = 0 .. Np - 2
    are one full period and sum to zero; n = Np - 1 adds cos(2 pi) = 1)."""
    a = orc.hamming_window(Np).astype(np.float64)
    assert a[0] == np.float32(0.08) and a[-1] == np.float32(0.08)
    assert np.array_equal(a, a[::-1])
    mid = 0.54 + 0.46 * np.cos(np.pi / (Np - 1))
    assert abs(a[Np // 2] - mid) <= 2.0 ** -24 and abs(a[Np // 2 - 1] - mid) <= 2.0 ** -24
    assert np.argmax(a) in (Np // 2 - 1, Np // 2)
    assert abs(a.sum() - (0.54 * Np - 0.46)) <= Np * 2.0 ** -24
