"""Runs one estimator at one size a few times, for profilers (ncu) and quick timing.

    python -m paper_2506_18003_gb300.profile_case ssca --N 262144 --Np 256 --reps 3
    python -m paper_2506_18003_gb300.profile_case fam --N 65728 --Np 256 --L 64 --P 1024 --reps 3
    python -m paper_2506_18003_gb300.profile_case batch_fam --N 0 --Np 64 --L 16 --nsig 64 --reps 2
    python -m paper_2506_18003_gb300.profile_case batch_ssca --N 0 --Np 128 --nsig 32 --schedule fused

Inputs are seeded white noise (the kernels' cost does not depend on the values).  Prints
the CUDA-event time of each call.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main() -> int:
    import torch

    from paper_2506_18003_gb300 import binding, signals

    ap = argparse.ArgumentParser()
    ap.add_argument("estimator", choices=["fam", "ssca", "fam_map", "ssca_map", "batch_fam", "batch_ssca"])
    ap.add_argument("--nsig", type=int, default=64, help="batch_*: signals (lengths log-uniform in [2^12, 2^18])")
    ap.add_argument("--N", type=int, required=True)
    ap.add_argument("--Np", type=int, default=256)
    ap.add_argument("--L", type=int, default=64)
    ap.add_argument("--P", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--schedule", default="auto", help="ssca, batch_*: auto, stages, persistent or fused (SSCA)")
    a = ap.parse_args()

    if a.estimator.startswith("batch_"):
        est = a.estimator[6:]
        lengths = [int(v) for v in signals.batch_lengths(a.nsig)]
        plan = binding.BatchPlan(est, lengths, a.Np, a.L, a.precision)
        plan.set_schedule(a.schedule)
        xa = torch.from_numpy(signals.awgn(int(sum(lengths)), seed=99)).cuda()
        out = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device="cuda")
        ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
        s = torch.cuda.Stream()
        for i in range(a.reps):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(s):
                t0.record(s)
                plan.run(xa, out, ws, stream=s)
                t1.record(s)
            s.synchronize()
            print(f"{a.estimator} rep {i}: {t0.elapsed_time(t1):.4f} ms")
        binding.scd_check_device(s)
        return 0
    x = torch.from_numpy(signals.awgn(a.N, seed=99)).cuda()
    if a.estimator.startswith("fam"):
        out = torch.empty((a.Np, a.Np, a.P), dtype=torch.complex64, device="cuda")
        mp = torch.empty((2 * a.Np, 2 * a.P * a.L), dtype=torch.float32, device="cuda") if a.estimator == "fam_map" else None
    else:
        out = torch.empty((a.Np, a.N), dtype=torch.complex64, device="cuda")
        mp = torch.empty((a.Np, 2 * a.N), dtype=torch.float32, device="cuda") if a.estimator == "ssca_map" else None
    for i in range(a.reps):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        if a.estimator == "fam":
            binding.scd_fam(x, a.Np, a.L, a.P, out=out, precision=a.precision)
        elif a.estimator == "ssca":
            binding.scd_ssca(x, a.Np, out=out, precision=a.precision, schedule=a.schedule)
        elif a.estimator == "fam_map":
            binding.scd_fam_map(out, a.Np, a.L, a.P, map=mp)
        else:
            binding.scd_ssca_map(out, a.N, a.Np, map=mp)
        t1.record()
        torch.cuda.synchronize()
        print(f"{a.estimator} rep {i}: {t0.elapsed_time(t1):.4f} ms")
    return 0


if __name__ == "__main__":
    sys.exit(main())
