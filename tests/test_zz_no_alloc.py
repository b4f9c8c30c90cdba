"""scd_fam_noalloc: the FAM entry point for callers that cannot allocate device memory
(real-time loops that forbid allocation after start-up, plug-ins that are only handed device
pointers).  It must give the same estimate as scd_fam, within the FP32 tolerance, on
consecutive calls that share its fixed scratch array, and refuse sizes beyond that array.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from paper_2506_18003_gb300 import binding, signals

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch, binding.load()


def _noalloc(torch, lib, x, Np, L, P, out, window=None):
    o = binding.make_opts(torch.cuda.current_stream(), "fp32", None)
    w = None if window is None else ctypes.c_void_p(window.data_ptr())
    return lib.scd_fam_noalloc(ctypes.c_void_p(x.data_ptr()), x.numel(), Np, L, P, w,
                               ctypes.c_void_p(out.data_ptr()), ctypes.byref(o))


def _rel(a, b):
    return float((a - b).abs().max().item() / b.abs().max().item())


def test_noalloc_matches_scd_fam_on_consecutive_calls(env):
    torch, lib = env
    cases = [(256, 64, 1024, None), (32, 8, 32, "given"), (64, 16, 4096, None)]
    for Np, L, P, win in cases:
        N = (P - 1) * L + Np + 3
        x = torch.from_numpy(signals.modulated("qpsk", N, 8, 0.07, 8.0, seed=7000 + Np)).cuda()
        window = torch.from_numpy(np.hanning(Np).astype(np.float32)).cuda() if win else None
        ref = binding.scd_fam(x, Np, L, P, window=window)
        out = torch.empty_like(ref)
        for _ in range(2):                                      # two calls in a row
            out.fill_(float("nan"))
            assert _noalloc(torch, lib, x, Np, L, P, out, window) == binding.SCD_OK
            torch.cuda.synchronize()
            assert _rel(out, ref) <= FP32_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, lib = env
    Np, L, P = 256, 64, 2048                                    # Np * P = 2^19 > 2^18
    x = torch.zeros((P - 1) * L + Np, dtype=torch.complex64, device="cuda")
    out = torch.empty(8, dtype=torch.complex64, device="cuda")
    assert _noalloc(torch, lib, x, Np, L, P, out) == binding.SCD_ERR_UNSUPPORTED
    assert b"scratch limit" in lib.scd_last_error()
