"""scd_fam_noalloc: the FAM entry point for callers that cannot allocate device memory
(real-time loops that forbid allocation after start-up, plug-ins that are only handed device
pointers).  It must give the same estimate as scd_fam, within the FP32 tolerance, on
consecutive calls that share its fixed scratch array, leave the device's free memory as it
was, and refuse sizes beyond that array.

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


# (Np, L, P, window): Np = 16 with P = 16384 fills the scratch exactly (Np * P = 2^18) and takes
# the single-pass channeliser with the default window
CASES = [(256, 64, 1024, None), (32, 8, 32, "given"), (64, 16, 4096, None), (16, 4, 16384, None)]


@pytest.mark.parametrize("Np,L,P,win", CASES)
def test_noalloc_matches_scd_fam_on_consecutive_calls(env, Np, L, P, win):
    torch, lib = env
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


def test_noalloc_leaves_free_device_memory_unchanged(env):
    """After one warm-up call (which resolves the scratch address), further calls change
    neither the device's free memory nor torch's allocation count."""
    torch, lib = env
    Np, L, P = 64, 16, 2048
    N = (P - 1) * L + Np
    x = torch.from_numpy(signals.modulated("bpsk", N, 4, -0.1, 5.0, seed=7100)).cuda()
    out = torch.empty(Np * Np * P, dtype=torch.complex64, device="cuda")
    assert _noalloc(torch, lib, x, Np, L, P, out) == binding.SCD_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(5):
        assert _noalloc(torch, lib, x, Np, L, P, out) == binding.SCD_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, lib = env
    Np, L, P = 256, 64, 2048                                    # Np * P = 2^19 > 2^18
    x = torch.zeros((P - 1) * L + Np, dtype=torch.complex64, device="cuda")
    out = torch.empty(8, dtype=torch.complex64, device="cuda")
    assert _noalloc(torch, lib, x, Np, L, P, out) == binding.SCD_ERR_UNSUPPORTED
    assert b"scratch limit" in lib.scd_last_error()
