#!/usr/bin/env python
"""Benchmark of the SCD hot path (FAM + SSCA estimators and their (f, alpha) maps) on GB300.

One step = one pass of the whole path over one batch of synthetic input:
  paper_scale (default): FAM at N=65,728 (Np=256, L=64, P=1024; 16-QAM) + its map, and
                         SSCA at N=2^20 (Np=256; BPSK+QPSK mixture) + its map.
The metric is input Msamples/s (samples consumed per second, whole job), with SCD points/s
alongside.  Inputs are resident in HBM when the timed region starts; every step's working
set (>2.5 GB of outputs) is larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line on rank 0.  --impl reference times the FP64 CPU oracle instead (the
method's plain reference, on the host cores, on a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import ctypes
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SCD input Msamples/s & points/s at stated error vs FP64; split-prec vs FP32 form"

FAM = dict(N=65728, Np=256, L=64, P=1024)
SSCA = dict(N=1 << 20, Np=256)


def workload_desc():
    return {"workload": "paper_scale: FAM N=65728 Np=256 L=64 P=1024 (16-QAM, RRC 0.25) + FAM map, "
                        "SSCA N=2^20 Np=256 (BPSK+QPSK mixture, 0 dB) + SSCA map",
            "fam": dict(FAM), "ssca": dict(SSCA), "window": "hamming",
            "l2": "working set per step > L2 (no flush needed)"}


def samples_per_step():
    return FAM["N"] + SSCA["N"]


def points_per_step():
    return FAM["Np"] ** 2 * FAM["P"] + SSCA["Np"] * SSCA["N"]


# Algorithmic (compulsory) bytes per launch of each kernel, complex64 = 8 B, float32 = 4 B.
def kernel_bytes():
    Np, L, P, Nf = FAM["Np"], FAM["L"], FAM["P"], FAM["N"]
    N, Ns = SSCA["N"], SSCA["Np"]
    Q = P * L // Np
    return {
        "fam_channelise": 8 * ((P - 1) * L + Np) + 8 * Np * P,
        "fam_pair_fft": 8 * Np * Np * P,
        "fam_map": 8 * Np * Np * 2 * Q + 4 * (2 * Np) * (2 * P * L),
        "ssca_cdp": 8 * N + 8 * Ns * N,
        "ssca_cols": 2 * 8 * Ns * N,
        "ssca_rows": 2 * 8 * Ns * N,
        "ssca_map": 8 * Ns * N + 4 * Ns * 2 * N,
    }


STAGES = ["fam_channelise", "fam_pair_fft", "fam_map", "ssca_cdp", "ssca_cols", "ssca_rows", "ssca_map"]


def captured_traffic(stage):
    """DRAM bytes per launch of `stage` from the committed ncu capture (profiles/traffic.json),
    or None when there is none or the kernel's sources changed since it was taken."""
    import hashlib
    try:
        entry = json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get(stage)
    except (OSError, ValueError):
        return None
    if not entry:
        return None
    h = hashlib.sha256()
    try:
        for f in entry["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
    except OSError:
        return None
    return entry["bytes_per_launch"] if h.hexdigest() == entry["sha256"] else None


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons every 100 ms; only the samples
    taken while the `with` block (the timed region) runs are kept."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.kept = []

    def _reader(self):
        for line in self.proc.stdout:
            self.lines.append(line)

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return self
        threading.Thread(target=self._reader, daemon=True).start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 3.0:      # sampler is up before timing starts
            time.sleep(0.01)
        self.start = len(self.lines)
        return self

    def __exit__(self, *exc):
        if self.proc is None:
            return
        self.kept = self.lines[self.start:]
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO("".join(self.kept))) if len(r) >= 9]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(torch, value, world):
    if world == 1:
        return value
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- CPU oracle
_SIGNALS = {}


def _bench_signals():
    if not _SIGNALS:
        from paper_2506_18003_gb300 import signals
        _SIGNALS["fam"] = signals.fam_qam16_paper_scale()
        _SIGNALS["ssca"] = signals.ssca_mixture_1m()
    return _SIGNALS["fam"], _SIGNALS["ssca"]


def oracle_sample(fam_pairs: int, ssca_slice: int, ssca_rows: int, seed_offset: int = 0):
    """Times the FP64 oracle on a bounded sample of the workload and extrapolates the
    time of one full step (both estimators; the maps are not included).
    Returns (seconds_per_full_step, description)."""
    import numpy as np

    from oracle import scd_oracle as orc

    wf, ws = _bench_signals()
    Np, L, P = FAM["Np"], FAM["L"], FAM["P"]
    a = orc.hamming_window(Np)
    g = np.random.default_rng(17 + seed_offset)
    kh = g.integers(0, Np, fam_pairs)
    lh = g.integers(0, Np, fam_pairs)
    t0 = time.perf_counter()
    orc.fam_pairs(wf["x"], a, Np, L, P, kh, lh)
    t_fam = (time.perf_counter() - t0) * (Np * Np / fam_pairs)

    N, Ns = SSCA["N"], SSCA["Np"]
    a2 = orc.hamming_window(Ns)
    n0 = int(g.integers(0, N - ssca_slice))
    t0 = time.perf_counter()
    orc.ssca_cdp(ws["x"], a2, Ns, np.arange(n0, n0 + ssca_slice))
    t_cdp = (time.perf_counter() - t0) * (N / ssca_slice)
    row = (g.standard_normal((ssca_rows, N)) + 1j * g.standard_normal((ssca_rows, N)))
    t0 = time.perf_counter()
    for i in range(ssca_rows):
        orc.ssca_strip(row[i])
    t_strip = (time.perf_counter() - t0) * (Ns / ssca_rows)
    desc = (f"FAM: {fam_pairs} of {Np * Np} channel pairs (oracle.fam_pairs, scaled x{Np * Np // fam_pairs}); "
            f"SSCA: channeliser+CDP for {ssca_slice} of {N} samples (scaled x{N // ssca_slice}) + "
            f"{ssca_rows} of {Ns} strip FFT rows (scaled x{Ns // ssca_rows}); maps not included")
    return t_fam + t_cdp + t_strip, desc


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    steps = []
    desc = ""
    for i in range(args.warmup + args.steps):
        t, desc = oracle_sample(fam_pairs=256, ssca_slice=1 << 12, ssca_rows=1, seed_offset=i)
        if i >= args.warmup:
            steps.append(t)
    t = statistics.mean(steps)
    v = samples_per_step() / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Msamples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(),
            "cpu_baseline": {"value": v, "unit": "Msamples/s", "cores": 1, "kind": "oracle",
                             "sample": "per step, " + desc + "; numpy FFT and elementwise kernels on one thread"},
            "e2e": {"value": v, "unit": "Msamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_2506_18003_gb300 import binding, signals

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = binding.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    prec = args.precision

    # ---- inputs (seeded per rank: every rank processes its own independent signals)
    wf = signals.fam_qam16_paper_scale(seed=signals.seed_for(2) + 100 * rank)
    wsig = signals.ssca_mixture_1m(seed=signals.seed_for(3) + 100 * rank)
    Np, L, P = FAM["Np"], FAM["L"], FAM["P"]
    N, Ns = SSCA["N"], SSCA["Np"]
    xf = torch.from_numpy(wf["x"]).to(dev)
    xs = torch.from_numpy(wsig["x"]).to(dev)
    Sf = torch.empty((Np, Np, P), dtype=torch.complex64, device=dev)
    Ss = torch.empty((Ns, N), dtype=torch.complex64, device=dev)
    Mf = torch.empty((2 * Np, 2 * P * L), dtype=torch.float32, device=dev)
    Ms = torch.empty((Ns, 2 * N), dtype=torch.float32, device=dev)
    wsp = max(lib.scd_fam_workspace_bytes(FAM["N"], Np, L, P, binding.PRECISIONS[prec]),
              lib.scd_ssca_workspace_bytes(N, Ns, binding.PRECISIONS[prec]))
    work = torch.empty(wsp, dtype=torch.uint8, device=dev)
    binding.scd_prepare("fam", FAM["N"], Np, P)
    binding.scd_prepare("ssca", N, Ns)

    EV_PER_STEP = 11          # FAM 3, FAM map 2, SSCA 4, SSCA map 2

    def opts(prec, events=None, off=0, n=0):
        o = binding.make_opts(stream, prec, work)
        if events is not None:
            o.stage_events = ctypes.cast(ctypes.addressof(events) + off * ctypes.sizeof(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_void_p))
            o.n_stage_events = n
        return o

    def step(prec, events=None, base=0):
        o = opts(prec, events, base + 0, 3)
        binding.check(lib.scd_fam(xf.data_ptr(), FAM["N"], Np, L, P, None, Sf.data_ptr(), ctypes.byref(o)), "fam")
        o = opts(prec, events, base + 3, 2)
        o.map_power = 1
        binding.check(lib.scd_fam_map(Sf.data_ptr(), Np, L, P, Mf.data_ptr(), ctypes.byref(o)), "fam_map")
        o = opts(prec, events, base + 5, 4)
        binding.check(lib.scd_ssca(xs.data_ptr(), N, Ns, None, Ss.data_ptr(), ctypes.byref(o)), "ssca")
        o = opts(prec, events, base + 9, 2)
        o.map_power = 1
        binding.check(lib.scd_ssca_map(Ss.data_ptr(), N, Ns, Ms.data_ptr(), ctypes.byref(o)), "ssca_map")

    def timed(prec):
        """W warm-up steps, then K steps bracketed by barrier + synchronize, per-stage events."""
        for _ in range(args.warmup):
            step(prec)
        torch.cuda.synchronize()
        binding.check(lib.scd_check_device(ctypes.c_void_p(stream.cuda_stream)), "device check")
        nev = EV_PER_STEP * args.steps
        events = (ctypes.c_void_p * nev)()
        binding.check(lib.scd_events_create(nev, events), "events")
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        launches0 = lib.scd_launch_count()
        with ClockSampler(local) as clk:
            t_start.record(stream)
            for s in range(args.steps):
                step(prec, events, EV_PER_STEP * s)
            t_end.record(stream)
            torch.cuda.synchronize()
        launches = lib.scd_launch_count() - launches0
        barrier(world)
        binding.check(lib.scd_check_device(ctypes.c_void_p(stream.cuda_stream)), "device check")
        ms = max_over_ranks(torch, t_start.elapsed_time(t_end), world)

        def el(a, b):
            f = ctypes.c_float()
            binding.check(lib.scd_event_elapsed_ms(events[a], events[b], ctypes.byref(f)), "elapsed")
            return f.value

        stage_ms = {k: 0.0 for k in STAGES}
        for s in range(args.steps):
            b = EV_PER_STEP * s
            stage_ms["fam_channelise"] += el(b + 0, b + 1)
            stage_ms["fam_pair_fft"] += el(b + 1, b + 2)
            stage_ms["fam_map"] += el(b + 3, b + 4)
            stage_ms["ssca_cdp"] += el(b + 5, b + 6)
            stage_ms["ssca_cols"] += el(b + 6, b + 7)
            stage_ms["ssca_rows"] += el(b + 7, b + 8)
            stage_ms["ssca_map"] += el(b + 9, b + 10)
        lib.scd_events_destroy(nev, events)
        for k in stage_ms:
            stage_ms[k] /= args.steps
        return ms / args.steps, stage_ms, int(launches), clk.summary()

    other = "split" if prec == "fp32" else "fp32"
    ms_step, stage_ms, launches, clocks = timed(prec)
    ms_other, stage_other, _, _ = timed(other)

    kb = kernel_bytes()
    top = max(stage_ms, key=stage_ms.get)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = kb[top] / (stage_ms[top] * 1e-3) / 1e9
    traffic = captured_traffic(top) if prec == "fp32" else None

    value = world * samples_per_step() / (ms_step * 1e-3) / 1e6
    dtype = {"fp32": "f32", "split": "bf16x3-split/f32-accumulate"}
    line = {
        "metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype[prec],
        "data": "synthetic (seeded modulated signals of the paper's shapes)", "config": workload_desc(),
        "scd_points_per_s": world * points_per_step() / (ms_step * 1e-3),
        "gpu_launches": launches,
        "stage_ms": {k: round(v, 5) for k, v in stage_ms.items()},
        "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes": kb[top]},
        "clocks": clocks,
        "parity_gate": {"fp32": "max|dS|/max|S| <= 1e-5 (tests)", "split": "<= 1e-3 (tests)"},
        other: {"value": world * samples_per_step() / (ms_other * 1e-3) / 1e6, "unit": "Msamples/s",
                "ms_per_step": ms_other, "dtype": dtype[other],
                "stage_ms": {k: round(v, 5) for k, v in stage_other.items()},
                "speedup_vs_" + prec: ms_step / ms_other},
    }
    # per-kernel roofline fractions (context for the dominant one)
    line["stage_hbm_frac"] = {k: round(kb[k] / (stage_ms[k] * 1e-3) / 1e9 / hbm, 4) for k in STAGES if stage_ms[k] > 0}

    if not args.no_e2e:
        line["e2e"] = e2e(args, lib, binding, torch, stream, wf["x"], wsig["x"], world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t, desc = oracle_sample(fam_pairs=2048, ssca_slice=1 << 15, ssca_rows=8)
        line["cpu_baseline"] = {"value": samples_per_step() / t / 1e6, "unit": "Msamples/s", "cores": 1,
                                "kind": "oracle", "sample": desc + "; numpy FFT and elementwise kernels on one thread"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def e2e(args, lib, binding, torch, stream, xf_np, xs_np, world):
    """Same metric through the host-buffer entry points: every step copies the inputs from
    pinned host memory, runs both estimators and copies both estimates back."""
    Np, L, P = FAM["Np"], FAM["L"], FAM["P"]
    N, Ns = SSCA["N"], SSCA["Np"]
    xf = torch.from_numpy(xf_np).pin_memory()
    xs = torch.from_numpy(xs_np).pin_memory()
    of = torch.empty((Np, Np, P), dtype=torch.complex64).pin_memory()
    os_ = torch.empty((Ns, N), dtype=torch.complex64).pin_memory()
    prec = binding.PRECISIONS[args.precision]
    need = max(lib.scd_fam_host_workspace_bytes(FAM["N"], Np, L, P, prec),
               lib.scd_ssca_host_workspace_bytes(N, Ns, prec))
    work = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    o = binding.make_opts(stream, args.precision, work)

    def step():
        binding.check(lib.scd_fam_host(xf.data_ptr(), FAM["N"], Np, L, P, None, of.data_ptr(), ctypes.byref(o)), "fam_host")
        binding.check(lib.scd_ssca_host(xs.data_ptr(), N, Ns, None, os_.data_ptr(), ctypes.byref(o)), "ssca_host")

    for _ in range(max(1, args.warmup)):
        step()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    import torch as _t
    dt = max_over_ranks(_t, dt, world)
    del work
    return {"value": world * samples_per_step() * args.steps / dt / 1e6, "unit": "Msamples/s",
            "h2d_bytes_per_step": 8 * (FAM["N"] + N), "d2h_bytes_per_step": 8 * (Np * Np * P + Ns * N),
            "api": "scd_fam_host + scd_ssca_host (pinned host buffers, synchronous)"}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "split"], default="fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
