"""Batched runs on host buffers (scd_batch_run_host): the input arena copied in from
page-locked host memory, the estimate copied back on the plan's copy stream.  The host copy
must equal the device run bit for bit, also when calls alternate between two device output
buffers (the second call computes while the first call's copy is in flight) and in the
alpha-profile output mode; one sampled signal per run is also checked against the FP64 oracle."""
import ctypes

import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import binding, signals

pytestmark = pytest.mark.gpu

LENGTHS = [4096, 5000, 9000, 17000, 33000, 6100]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    binding.load()
    return t


def _setup(torch, est, Np, L):
    sigs = [signals.batch_signal(40 + i, n) for i, n in enumerate(LENGTHS)]
    plan = binding.BatchPlan(est, LENGTHS, Np, L, "fp32")
    x = torch.from_numpy(np.concatenate(sigs)).cuda()
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    return sigs, plan, x, ws


def _oracle(est, xs, Np, L, n):
    a = orc.hamming_window(Np)
    return orc.fam(xs, a, Np, L, n) if est == "fam" else orc.ssca(xs[:n].copy(), a, Np)


@pytest.mark.parametrize("est,Np,L", [("fam", 64, 16), ("ssca", 128, 1)])
def test_run_host_equals_device_run(torch, est, Np, L):
    sigs, plan, x, ws = _setup(torch, est, Np, L)
    n_out = plan.out_offsets[-1]
    ref = torch.empty(n_out, dtype=torch.complex64, device="cuda")
    plan.run(x, ref, ws)
    binding.scd_check_device()
    ref_h = ref.cpu()

    hx = binding.HostBuffer(x.numel(), torch.complex64)
    hx.tensor.copy_(x.cpu())
    h0 = binding.HostBuffer(n_out, torch.complex64)
    h1 = binding.HostBuffer(n_out, torch.complex64)
    d0 = torch.zeros(n_out, dtype=torch.complex64, device="cuda")
    d1 = torch.zeros(n_out, dtype=torch.complex64, device="cuda")
    xd = torch.zeros_like(x)
    stream = torch.cuda.Stream()
    # two calls into two device buffers and two host buffers, then a third that reuses the first
    plan.run_host(hx.tensor, xd, d0, h0.tensor, ws, stream=stream)
    plan.run_host(None, xd, d1, h1.tensor, ws, stream=stream)
    plan.host_wait()
    binding.scd_check_device(stream)
    assert torch.equal(h0.tensor, ref_h) and torch.equal(h1.tensor, ref_h)
    h0.tensor.zero_()
    plan.run_host(hx.tensor, xd, d0, h0.tensor, ws, stream=stream)
    plan.host_wait()
    assert torch.equal(h0.tensor, ref_h)

    i = 3
    n = plan.sizes[i]
    a, b = plan.out_offsets[i], plan.out_offsets[i + 1]
    got = h0.tensor[a:b].numpy().reshape((Np, Np, n) if est == "fam" else (Np, n))
    want = _oracle(est, sigs[i], Np, L, n)
    assert float(np.max(np.abs(got - want)) / np.max(np.abs(want))) <= 1e-5
    for h in (hx, h0, h1):
        h.close()
    plan.close()


def test_run_host_profile_mode(torch):
    sigs, plan, x, ws = _setup(torch, "ssca", 128, 1)
    plan.set_output("profile", 1)
    n_out = plan.out_offsets[-1]
    ref = torch.empty(n_out, dtype=torch.float32, device="cuda")
    plan.run(x, ref, ws)
    hp = binding.HostBuffer(n_out, torch.float32)
    d = torch.empty(n_out, dtype=torch.float32, device="cuda")
    plan.run_host(None, x, d, hp.tensor, ws)
    plan.host_wait()
    binding.scd_check_device()
    assert torch.equal(hp.tensor, ref.cpu())
    hp.close()
    plan.close()


def test_run_host_arguments(torch):
    _, plan, x, ws = _setup(torch, "fam", 64, 16)
    lib = binding.load()
    out = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device="cuda")
    p = ctypes.c_void_p
    host = binding.HostBuffer(16, torch.complex64)
    # NULL device input, device output or host output: rejected before anything is enqueued
    for xd, od, oh in ((None, out, host.ptr), (x, None, host.ptr), (x, out, None)):
        st = lib.scd_batch_run_host(plan.handle, None, p(xd.data_ptr()) if xd is not None else None, None,
                                    p(od.data_ptr()) if od is not None else None, p(oh) if oh else None,
                                    p(ws.data_ptr()), None)
        assert st == binding.SCD_ERR_ARG
    host.close()
    assert lib.scd_batch_host_wait(None) == binding.SCD_ERR_ARG
    assert lib.scd_batch_host_wait(plan.handle) == binding.SCD_OK          # nothing queued yet
    with pytest.raises(TypeError):
        plan.run_host(None, x, out, out, ws)                                # a device tensor as out_host
    ptr = ctypes.c_void_p()
    assert lib.scd_host_alloc(0, ctypes.byref(ptr)) == binding.SCD_ERR_ARG
    assert lib.scd_host_free(None) == binding.SCD_OK
    plan.close()
