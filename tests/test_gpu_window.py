"""GPU parity of the Dolph-Chebyshev window (scd_chebyshev_window) against the FP64 oracle,
and of both estimators run with it (the chebwin windowing of Algorithms 1 and 2)."""
import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import binding, signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    binding.load()
    return t


@pytest.mark.parametrize("Np", [2, 16, 31, 64, 100, 256])
@pytest.mark.parametrize("atten", [30.0, 100.0, 200.0])
def test_chebyshev_window_matches_oracle(torch, Np, atten):
    got = binding.scd_chebyshev_window(Np, atten).cpu().numpy().astype(np.float64)
    ref = orc.chebyshev_window64(Np, atten)
    assert np.max(np.abs(got - ref)) <= 2.0 ** -23          # float32 rounding of an FP64 value in (0, 1]


def test_estimators_with_chebyshev_window(torch):
    Np, L, P = 64, 16, 128
    N = (P - 1) * L + Np
    x = signals.modulated("qpsk", N, 4, 0.1, 8.0, seed=8000)
    w_dev = binding.scd_chebyshev_window(Np, 100.0)
    a = w_dev.cpu().numpy()
    ref = orc.fam(x, a, Np, L, P)
    got = binding.scd_fam(torch.from_numpy(x).cuda(), Np, L, P, window=w_dev).cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5
    Ns = 1 << 13
    xs = signals.modulated("bpsk", Ns, 8, -0.1, 8.0, seed=8001)
    ref = orc.ssca(xs, a, Np)
    got = binding.scd_ssca(torch.from_numpy(xs).cuda(), Np, window=w_dev).cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5
