"""The headline workload at full size: the 512-signal mixed batch (lengths log-uniform in
[2^12, 2^18]) through FAM (Np = 64, L = 16) and SSCA (Np = 128) in the launch configuration
the benchmark times (default schedules).  Every transform-size class is sampled: for each,
the shortest and the longest signal of the class are recomputed by the FP64 oracle over
channel pairs (FAM: full P-bin rows) or channels (SSCA: full N-bin rows) that cover the band
edges, the centre and the boundaries of the fused kernel's channel blocks.  Also the fused SSCA
schedule against the oracle and the three-stage schedule on a smaller batch with every
cluster shape."""
import numpy as np
import pytest

from oracle import scd_oracle as orc
from paper_2506_18003_gb300 import binding, signals

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    binding.load()
    return t


@pytest.fixture(scope="module")
def batch():
    lengths = signals.batch_lengths()
    sigs = [signals.batch_signal(i, n) for i, n in enumerate(lengths)]
    return lengths, sigs


def _run(torch, plan, sigs):
    x = torch.from_numpy(np.concatenate(sigs)).cuda()
    out = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    plan.run(x, out, ws)
    binding.scd_check_device()
    del x, ws
    return out


def _per_class(sizes):
    """Shortest and longest signal of every size class."""
    picks = []
    for s in sorted(set(sizes)):
        idx = [i for i, v in enumerate(sizes) if v == s]
        picks += sorted({idx[0], idx[-1]})
    return picks


def test_fam_batch_512_every_size_class(torch, batch):
    lengths, sigs = batch
    Np, L = 64, 16
    plan = binding.BatchPlan("fam", lengths, Np, L, "fp32")
    out = _run(torch, plan, sigs)
    a = orc.hamming_window(Np)
    kh = np.array([0, 0, 63, 31, 32, 17, 40, 63])
    lh = np.array([0, 63, 0, 32, 31, 17, 5, 63])
    picks = _per_class(plan.sizes)
    assert set(plan.sizes[i] for i in picks) == set(plan.sizes)
    for i in picks:
        P = plan.sizes[i]
        est = plan.output(out, i)
        ref = orc.fam_pairs(sigs[i], a, Np, L, P, kh, lh)
        got = est[torch.from_numpy(kh).cuda(), torch.from_numpy(lh).cuda()].cpu().numpy()
        smax = est.abs().max().item()
        assert float(np.max(np.abs(got - ref))) / smax <= FP32_TOL, (i, P)
        # the largest value sits on the alpha = 0 diagonal: k = l, q = 0
        diag = orc.fam_pairs(sigs[i], a, Np, L, P, np.arange(Np), np.arange(Np))[:, P // 2]
        assert abs(np.max(np.abs(diag)) - smax) / smax <= FP32_TOL, (i, P)
    plan.close()
    del out
    torch.cuda.empty_cache()


def test_ssca_batch_512_every_size_class(torch, batch):
    lengths, sigs = batch
    Np = 128
    plan = binding.BatchPlan("ssca", lengths, Np, 1, "fp32")
    out = _run(torch, plan, sigs)
    a = orc.hamming_window(Np)
    ch = np.array([0, 1, 31, 32, 63, 64, 65, 95, 96, 127])
    picks = _per_class(plan.sizes)
    for i in picks:
        N = plan.sizes[i]
        est = plan.output(out, i)
        ref = orc.ssca(sigs[i][:N].copy(), a, Np, channels=ch, chunk=1 << 15)
        got = est[torch.from_numpy(ch).cuda()].cpu().numpy()
        smax = est.abs().max().item()
        assert float(np.max(np.abs(got - ref))) / smax <= FP32_TOL, (i, N)
    plan.close()
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("Np", [64, 128, 256])
def test_ssca_batch_fused_schedule(torch, Np):
    """Sizes 2^12 .. 2^18 (2^12 at Np = 128 and 256 runs the three-stage kernels inside the
    fused schedule): every signal against the oracle (sampled channels above 2^15) and against
    the three-stage schedule."""
    lengths = [4096, 300000, 9000, 70000, 150000, 33000, 17000]
    sigs = [signals.batch_signal(800 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("ssca", lengths, Np, 1, "fp32")
    plan.set_schedule("fused")
    out_f = _run(torch, plan, sigs)
    plan.set_schedule("stages")
    out_s = _run(torch, plan, sigs)
    a = orc.hamming_window(Np)
    ch = np.array(sorted({0, 1, Np // 4 - 1, Np // 4, Np // 2 - 1, Np // 2, 3 * Np // 4, Np - 1}))
    for i, x in enumerate(sigs):
        N = plan.sizes[i]
        est = plan.output(out_f, i)
        smax = est.abs().max().item()
        assert (est - plan.output(out_s, i)).abs().max().item() / smax <= FP32_TOL, (i, N)
        if N <= 1 << 15:
            ref = orc.ssca(x[:N].copy(), a, Np)
            got = est.cpu().numpy()
        else:
            ref = orc.ssca(x[:N].copy(), a, Np, channels=ch, chunk=1 << 15)
            got = est[torch.from_numpy(ch).cuda()].cpu().numpy()
        assert float(np.max(np.abs(got - ref))) / smax <= FP32_TOL, (i, N)
    plan.close()
    del out_f, out_s
    torch.cuda.empty_cache()


def test_ssca_batch_fused_profiles(torch):
    """Alpha-profile output of the fused schedule equals the profile of its own full estimates
    bit for bit (maxima do not depend on the order of the reductions)."""
    Np = 128
    lengths = [4096, 70000, 9000, 150000]
    sigs = [signals.batch_signal(900 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("ssca", lengths, Np, 1, "fp32")
    plan.set_schedule("fused")
    est_out = _run(torch, plan, sigs)
    est = [plan.output(est_out, i) for i in range(len(lengths))]
    plan.set_output("profile")
    x = torch.from_numpy(np.concatenate(sigs)).cuda()
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    prof = torch.empty(plan.out_offsets[-1], dtype=torch.float32, device="cuda")
    plan.run(x, prof, ws)
    binding.scd_check_device()
    for i in range(len(lengths)):
        N = plan.sizes[i]
        same = binding.scd_ssca_alpha_profile(est[i], N, Np)
        assert torch.equal(plan.output(prof, i), same), i
    plan.close()


def _exact_lengths():
    """40 lengths: powers of two, primes, one above and one below a power of two, and the
    log-uniform mix of the headline workload."""
    fixed = [4096, 8192, 65536, 4099, 8191, 10007, 65537, 131071, 131073, 200003]
    return fixed + [int(v) for v in signals.batch_lengths(30, seed=4242)]


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_ssca_exact_batch_40_signals(torch, precision):
    """Exact-length SSCA plan over 40 signals of mixed lengths (Bluestein for those that are
    not powers of two), one graph: every signal equals the single-estimate call bit for bit;
    the shortest and longest signal of each cyclic length against the FP64 oracle."""
    Np = 128
    lengths = _exact_lengths()
    sigs = [signals.batch_signal(1000 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("ssca", lengths, Np, 1, precision, exact=True)
    assert plan.sizes == lengths
    out = _run(torch, plan, sigs)
    a = orc.hamming_window(Np)
    tol = FP32_TOL if precision == "fp32" else 1e-3
    ad = torch.from_numpy(a).cuda()
    cyc = [n if n & (n - 1) == 0 else 1 << (2 * n - 2).bit_length() for n in lengths]
    ch = np.array([0, 31, 64, 127])
    for c in sorted(set(cyc)):
        idx = [i for i, v in enumerate(cyc) if v == c]
        for i in sorted({idx[0], idx[-1]}):
            est = plan.output(out, i)
            single = binding.scd_ssca(torch.from_numpy(sigs[i]).cuda(), Np, window=ad, precision=precision,
                                      schedule="stages")
            assert torch.equal(est, single), i
            ref = orc.ssca(sigs[i], a, Np, channels=ch, chunk=1 << 15)
            got = est[torch.from_numpy(ch).cuda()].cpu().numpy()
            smax = est.abs().max().item()
            assert float(np.max(np.abs(got - ref))) / smax <= tol, (i, lengths[i])
    plan.close()
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_fam_exact_batch_40_signals(torch, precision):
    """Exact-length FAM plan (P_i = (len_i - Np)//L + 1, Bluestein where P_i is not a power of
    two) over 40 signals, one graph: sampled pairs of the shortest and longest signal of each
    transform size against the FP64 oracle."""
    Np, L = 64, 16
    # P that is not a power of two runs both cyclic transforms inside one CTA: P <= 8192
    lengths = [min(n, 8191 * L + Np) for n in _exact_lengths()]
    sigs = [signals.batch_signal(1100 + i, n) for i, n in enumerate(lengths)]
    plan = binding.BatchPlan("fam", lengths, Np, L, precision, exact=True)
    assert plan.sizes == [(n - Np) // L + 1 for n in lengths]
    out = _run(torch, plan, sigs)
    a = orc.hamming_window(Np)
    tol = FP32_TOL if precision == "fp32" else 1e-3
    kh = np.array([0, 63, 31, 32, 5])
    lh = np.array([0, 0, 32, 31, 60])
    cls = [P if P & (P - 1) == 0 else -(1 << (2 * P - 2).bit_length()) for P in plan.sizes]
    for c in sorted(set(cls)):
        idx = [i for i, v in enumerate(cls) if v == c]
        for i in sorted({idx[0], idx[-1]}):
            P = plan.sizes[i]
            est = plan.output(out, i)
            ref = orc.fam_pairs(sigs[i], a, Np, L, P, kh, lh)
            got = est[torch.from_numpy(kh).cuda(), torch.from_numpy(lh).cuda()].cpu().numpy()
            smax = est.abs().max().item()
            assert float(np.max(np.abs(got - ref))) / smax <= tol, (i, P)
    plan.close()
    del out
    torch.cuda.empty_cache()
