#!/usr/bin/env python
"""Benchmark of the SCD hot path (FAM + SSCA estimators) on GB300.

One step = one pass of the whole path over one batch of synthetic input.  Workloads:

  batch (default)  512 signals, lengths log-uniform in [2^12, 2^18] (mixed BPSK / QPSK / 8-PSK /
                   16-QAM / AM-DSB / noise), through FAM (Np=64, L=16) and SSCA (Np=128): one
                   persistent, graph-captured launch per estimator.
  paper_scale      one FAM estimate at N=65,728 (Np=256, L=64, P=1024) + its (f, alpha) map and
                   one SSCA estimate at N=2^20 (Np=256) + its map.

The metric is input Msamples/s: samples consumed per second by both estimators, whole job
(SCD points/s alongside).  Both forms are timed: the FP32 form is the headline `value`, the
split-precision form (bf16 hi/lo tensor-core GEMMs, FP32 accumulation) is reported beside it.
Inputs are resident in HBM when the timed region starts; every step's working set is far
larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line on rank 0.  --impl reference times the FP64 CPU oracle instead (the
method's plain reference, on the host cores, on a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import csv
import ctypes
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SCD input Msamples/s & points/s at stated error vs FP64; split-prec vs FP32 form"
DTYPE = {"fp32": "f32", "split": "bf16x3-split/f32-accumulate"}


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
        self.start = 0

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
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(torch, value, world):
    """Largest `value` over all ranks (the step time the whole job waited for)."""
    if world == 1:
        return value
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job throughput: every rank processed `units_per_rank` in at most `seconds`."""
    return world * units_per_rank / seconds


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- workloads
def fft_flops(M):
    """Conventional FLOP count of a complex M-point FFT (radix-2 count, 5 M log2 M)."""
    return 5 * M * (M.bit_length() - 1)


def fam_flops(Np, P):
    """Algorithmic FLOPs of one FAM estimate: per frame the window (2 Np), the Np-point FFT and
    the down-conversion (6 Np); per channel pair the conjugate product (6 P) and the P-point
    FFT."""
    return P * (2 * Np + fft_flops(Np) + 6 * Np) + Np * Np * (6 * P + fft_flops(P))


def ssca_flops(Np, N):
    """Algorithmic FLOPs of one SSCA estimate: per time point the window, the Np-point FFT, the
    down-conversion and the channel-data product (2 + 6 + 6 per channel); per channel the
    N-point strip FFT."""
    return N * (2 * Np + fft_flops(Np) + 12 * Np) + Np * fft_flops(N)


def fp32_peak_tflops(sm_count, clock_mhz):
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOP (FMA) x SM clock."""
    return sm_count * 128 * 2 * clock_mhz * 1e6 / 1e12


def _oracle_worker_init():
    # one thread per worker process: the pool supplies the parallelism
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_job(job):
    """One signal of the batch through the FP64 oracle's full FAM and SSCA estimates, in a
    worker process (the signal is regenerated from its seed); returns (samples consumed, s)."""
    i, n, seed, fam_np, fam_l, P, ssca_np, N = job
    from oracle import scd_oracle as orc
    from paper_2506_18003_gb300 import signals
    x = signals.batch_signal(i, n, seed=seed)
    t0 = time.perf_counter()
    orc.fam(x, orc.hamming_window(fam_np), fam_np, fam_l, P)
    orc.ssca(x[:N].copy(), orc.hamming_window(ssca_np), ssca_np)
    return (P - 1) * fam_l + fam_np + N, time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The FP64 oracle as it stands, one signal per task on every host core: a pool of spawned
    worker processes (spawned, not forked, so that no worker inherits a CUDA context)."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or host_cores()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init)
        self.pool.map(_oracle_worker_init_probe, range(self.cores))      # workers up, imports done

    def run(self, jobs):
        """Wall time of the jobs spread over the pool; returns (samples consumed, seconds)."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_job, jobs, chunksize=1)
        return sum(r[0] for r in res), time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def _oracle_worker_init_probe(_):
    from oracle import scd_oracle  # noqa: F401
    from paper_2506_18003_gb300 import signals  # noqa: F401
    return 0


class BatchWorkload:
    """512 mixed signals through the batched FAM and SSCA (one persistent launch each)."""
    name = "batch"
    FAM_NP, FAM_L, SSCA_NP = 64, 16, 128
    stages = ["fam_batch", "ssca_batch"]
    n_marks = 3

    def __init__(self, rank=0, count=512, tune=True):
        from paper_2506_18003_gb300 import signals
        self.tune = tune
        self.lengths = [int(v) for v in signals.batch_lengths(count)]
        # every rank processes its own independent signals (weak scaling)
        self.seeds = [signals.seed_for(4, i + 1) + 7919 * rank for i in range(len(self.lengths))]
        self.sigs = [signals.batch_signal(i, n, seed=self.seeds[i]) for i, n in enumerate(self.lengths)]
        self.fam_P = [self._fam_P(n) for n in self.lengths]
        self.ssca_N = [self._ssca_N(n) for n in self.lengths]

    def _fam_P(self, n):
        P = 8192
        while (P - 1) * self.FAM_L + self.FAM_NP > n:
            P //= 2
        return P

    @staticmethod
    def _ssca_N(n):
        N = 1 << 20
        while N > n:
            N //= 2
        return N

    def desc(self):
        return {"workload": "batch: 512 signals, lengths log-uniform in [2^12, 2^18] (BPSK/QPSK/8PSK/16QAM/"
                            "AM-DSB/AWGN, sps {2,4,8,16}, fc U(+-0.25), SNR U[-5,15] dB); FAM Np=64 L=16 "
                            "(P_i = largest power of two that fits), SSCA Np=128 (N_i = largest power of two "
                            "<= len_i); one CUDA graph per estimator (persistent launch or staged launches, "
                            "autotuned)",
                "signals": len(self.lengths), "input_samples": int(sum(self.lengths)),
                "fam": {"Np": self.FAM_NP, "L": self.FAM_L}, "ssca": {"Np": self.SSCA_NP},
                "window": "hamming", "l2": "working set per step ~95 GB > L2 (no flush needed)"}

    def fam_used(self):
        return sum((P - 1) * self.FAM_L + self.FAM_NP for P in self.fam_P)

    def samples_per_step(self):
        return self.fam_used() + sum(self.ssca_N)

    def rates(self, stage_ms, ms_step):
        """Per-estimator rates beside the headline (which sums both estimators' consumed
        samples), and the rate at which the step consumes the input arena itself."""
        fam_s, ssca_s = self.fam_used(), sum(self.ssca_N)
        inp = int(sum(self.lengths))
        return {"fam_msamples_per_s": round(fam_s / (stage_ms["fam_batch"] * 1e-3) / 1e6, 2),
                "ssca_msamples_per_s": round(ssca_s / (stage_ms["ssca_batch"] * 1e-3) / 1e6, 2),
                "input_msamples_per_s": round(inp / (ms_step * 1e-3) / 1e6, 2),
                "fam_samples": fam_s, "ssca_samples": ssca_s, "input_samples": inp,
                "value_is": "(FAM samples consumed + SSCA samples consumed) per step / step time: both "
                            "estimators read the same input arena, each counted once"}

    def oracle_jobs(self, idx):
        return [(i, self.lengths[i], self.seeds[i], self.FAM_NP, self.FAM_L, self.fam_P[i], self.SSCA_NP,
                 self.ssca_N[i]) for i in idx]

    def cpu_baseline(self, pool):
        """The FP64 oracle on every host core: one signal per worker, `cores` signals of the
        batch at evenly spaced length quantiles, full FAM and SSCA estimates; the rate is the
        sample's consumed samples over the wall time of the pool."""
        import numpy as np
        order = np.argsort(self.lengths)
        k = pool.cores
        pick = [int(order[len(order) * (j + 1) // (k + 1)]) for j in range(k)]
        used, t = pool.run(self.oracle_jobs(pick))
        desc = (f"{k} signals of the batch at evenly spaced length quantiles ({min(self.lengths[i] for i in pick)}"
                f"..{max(self.lengths[i] for i in pick)} samples), full FAM and SSCA estimates, one signal per "
                f"worker process ({k} processes, one thread each); rate = {used} samples consumed / {t:.2f} s wall")
        return used / t / 1e6, t, desc

    def reference_step(self, pool, k):
        """Step k of the reference arm: `cores` signals shorter than 2^15 samples (a rotating
        window over the batch), full FAM and SSCA estimates, one per worker."""
        short = [i for i, n in enumerate(self.lengths) if n < (1 << 15)]
        c = pool.cores
        pick = [short[(k * c + j) % len(short)] for j in range(c)]
        used, t = pool.run(self.oracle_jobs(pick))
        desc = (f"per step {c} signals of the batch shorter than 2^15 samples (a rotating window), full FAM and "
                f"SSCA estimates, one signal per worker process ({c} processes, one thread each)")
        return used, t, desc

    def parity_refs(self, nsig=3):
        """Full FP64 oracle estimates of `nsig` signals (in this process, untimed) for the
        parity check of both forms."""
        import numpy as np
        from oracle import scd_oracle as orc
        order = np.argsort(self.lengths)
        pick = [int(order[len(order) * (k + 1) // (nsig + 1)]) for k in range(nsig)]
        af, as_ = orc.hamming_window(self.FAM_NP), orc.hamming_window(self.SSCA_NP)
        self.oracle_refs = {i: (orc.fam(self.sigs[i], af, self.FAM_NP, self.FAM_L, self.fam_P[i]),
                                orc.ssca(self.sigs[i][:self.ssca_N[i]], as_, self.SSCA_NP)) for i in pick}

    def points_per_step(self):
        return sum(self.FAM_NP ** 2 * P for P in self.fam_P) + sum(self.SSCA_NP * N for N in self.ssca_N)

    def kernel_bytes(self):
        return {"fam_batch": 8 * self.fam_used() + 8 * sum(self.FAM_NP ** 2 * P for P in self.fam_P),
                "ssca_batch": 8 * sum(self.ssca_N) + 8 * sum(self.SSCA_NP * N for N in self.ssca_N)}

    def kernel_flops(self):
        return {"fam_batch": sum(fam_flops(self.FAM_NP, P) for P in self.fam_P),
                "ssca_batch": sum(ssca_flops(self.SSCA_NP, N) for N in self.ssca_N)}

    def setup(self, torch, binding, dev, prec):
        import numpy as np
        self.torch, self.binding = torch, binding
        self.x = torch.from_numpy(np.concatenate(self.sigs)).to(dev)
        self.plans = {}
        for p in ("fp32", "split"):
            fam = binding.BatchPlan("fam", self.lengths, self.FAM_NP, self.FAM_L, p)
            ssca = binding.BatchPlan("ssca", self.lengths, self.SSCA_NP, 1, p)
            self.plans[p] = (fam, ssca)
        fam, ssca = self.plans["fp32"]
        self.out_f = torch.empty(fam.out_offsets[-1], dtype=torch.complex64, device=dev)
        self.out_s = torch.empty(ssca.out_offsets[-1], dtype=torch.complex64, device=dev)
        ws = max(fam.workspace_bytes, ssca.workspace_bytes)
        self.ws = torch.empty(ws, dtype=torch.uint8, device=dev)
        if self.tune:                       # autotune the persistent schedule (outside any timing)
            stream = torch.cuda.current_stream()
            for p in ("fp32", "split"):
                f, s_ = self.plans[p]
                f.tune(self.x, self.out_f, self.ws, stream=stream, reps=2)
                s_.tune(self.x, self.out_s, self.ws, stream=stream, reps=2)
            torch.cuda.synchronize()

    def step(self, prec, stream, marks=None):
        fam, ssca = self.plans[prec]
        if marks is not None:
            marks[0].record(stream)
        fam.run(self.x, self.out_f, self.ws, stream=stream)
        if marks is not None:
            marks[1].record(stream)
        ssca.run(self.x, self.out_s, self.ws, stream=stream)
        if marks is not None:
            marks[2].record(stream)

    def stage_times(self, marks):
        return {"fam_batch": marks[0].elapsed_time(marks[1]), "ssca_batch": marks[1].elapsed_time(marks[2])}

    def parity_sample(self, stream):
        """Error of both forms on the signals whose oracle estimates the CPU-baseline leg just
        computed: max and mean |S_gpu - S_oracle| / max|S_oracle| per estimator (one fresh run
        of each plan, outside any timing)."""
        import numpy as np
        res = {}
        for prec in ("fp32", "split"):
            fam, ssca = self.plans[prec]
            fam.run(self.x, self.out_f, self.ws, stream=stream)
            ssca.run(self.x, self.out_s, self.ws, stream=stream)
            stream.synchronize()
            self.binding.scd_check_device(stream)
            for name, plan, out, k in (("fam", fam, self.out_f, 0), ("ssca", ssca, self.out_s, 1)):
                mx = mean = 0.0
                for i, refs in self.oracle_refs.items():
                    ref = refs[k]
                    d = np.abs(plan.output(out, i).cpu().numpy() - ref)
                    scale = float(np.max(np.abs(ref)))
                    mx = max(mx, float(d.max()) / scale)
                    mean = max(mean, float(d.mean()) / scale)
                res[f"{name}_{prec}"] = {"max_rel": mx, "mean_rel": mean}
        res["signals"] = sorted(int(i) for i in self.oracle_refs)
        res["metric"] = "max (and mean) |S_gpu - S_oracle| / max|S_oracle| over each sampled signal's full estimate"
        return res

    def profile_mode(self, torch, binding, stream, reps=10, warmup=3):
        """The same step with the plans' alpha-profile output (the estimates are reduced to one
        float per alpha column inside the kernels and never written): FP32 form, CUDA events
        around `reps` steps after `warmup`."""
        dev = self.x.device
        plans = []
        for est, Np, L in (("fam", self.FAM_NP, self.FAM_L), ("ssca", self.SSCA_NP, 1)):
            pl = binding.BatchPlan(est, self.lengths, Np, L, "fp32")
            pl.set_output("profile", 1)
            plans.append((pl, torch.empty(pl.out_offsets[-1], dtype=torch.float32, device=dev)))
        with torch.cuda.stream(stream):
            for pl, out in plans:
                pl.tune(self.x, out, self.ws, stream=stream, reps=2)
            for _ in range(warmup):
                for pl, out in plans:
                    pl.run(self.x, out, self.ws, stream=stream)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            tf = ts = 0.0
            for _ in range(reps):
                ev[0].record(stream)
                plans[0][0].run(self.x, plans[0][1], self.ws, stream=stream)
                ev[1].record(stream)
                plans[1][0].run(self.x, plans[1][1], self.ws, stream=stream)
                ev[2].record(stream)
                ev[2].synchronize()
                tf += ev[0].elapsed_time(ev[1]) / reps
                ts += ev[1].elapsed_time(ev[2]) / reps
        binding.scd_check_device(stream)
        out_bytes = 4 * (plans[0][0].out_offsets[-1] + plans[1][0].out_offsets[-1])
        # end to end in this output mode, through scd_batch_run_host: the input arena in from
        # page-locked host memory, both profile plans, both profile arenas out to page-locked host
        # memory, every step; steps pipelined on two device output sets as in e2e()
        hx = binding.HostBuffer(self.x.numel(), self.x.dtype)
        hx.tensor.copy_(self.x.cpu())
        hosts = [binding.HostBuffer(out.numel(), out.dtype) for _, out in plans]
        second = [torch.empty_like(out) for _, out in plans]

        def one(k):
            for j, ((pl, out), h) in enumerate(zip(plans, hosts)):
                pl.run_host(hx.tensor if j == 0 else None, self.x, out if k % 2 == 0 else second[j], h.tensor,
                            self.ws, stream=stream)

        def drain():
            for pl, _ in plans:
                pl.host_wait()
            stream.synchronize()

        with torch.cuda.stream(stream):
            one(0)
            one(1)
            drain()
            t0 = time.perf_counter()
            for k in range(reps):
                one(k)
            drain()
            dt = (time.perf_counter() - t0) / reps
        for pl, _ in plans:
            pl.close()
        for h in [hx] + hosts:
            h.close()
        return {"ms_per_step": round(tf + ts, 4), "stage_ms": {"fam_batch": round(tf, 4), "ssca_batch": round(ts, 4)},
                "msamples_per_s": round(self.samples_per_step() / ((tf + ts) * 1e-3) / 1e6, 2),
                "output_bytes_per_step": out_bytes,
                "e2e": {"value": round(self.samples_per_step() / dt / 1e6, 2), "unit": "Msamples/s",
                        "ms_per_step": round(dt * 1e3, 3), "h2d_bytes_per_step": self.x.numel() * 8,
                        "d2h_bytes_per_step": out_bytes,
                        "api": "scd_batch_run_host (BatchPlan.run_host) in alpha-profile mode on page-locked host "
                               "buffers; steps pipelined on two device output sets"},
                "note": "alpha profiles (|S| max over f per alpha) fused into the last stage; FP32 form; tuned"}

    def exact_ssca(self, torch, binding, stream, reps=3):
        """The batch's SSCA without truncation (exact-length plan: N_i = len_i, Bluestein for
        the lengths that are not powers of two; one CUDA graph: the input preparation and the
        channeliser over every signal, then three passes per cyclic length), FP32, outside the
        step: CUDA events around `reps` runs after one warm-up."""
        plan = binding.BatchPlan("ssca", self.lengths, self.SSCA_NP, 1, "fp32", exact=True)
        out = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device=self.x.device)
        ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device=self.x.device)
        with torch.cuda.stream(stream):
            plan.run(self.x, out, ws, stream=stream)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                plan.run(self.x, out, ws, stream=stream)
            t1.record(stream)
            t1.synchronize()
        binding.scd_check_device(stream)
        ms = t0.elapsed_time(t1) / reps
        used = int(sum(self.lengths))
        res = {"ms": round(ms, 3), "samples": used, "msamples_per_s": round(used / (ms * 1e-3) / 1e6, 2),
               "workspace_bytes": int(plan.workspace_bytes),
               "note": "every sample of the 512 signals (the step's SSCA uses the largest power of two of each "
                       "length); Bluestein's identity with cyclic lengths up to 2^19; FP32; one graph per run"}
        plan.close()
        del out, ws
        torch.cuda.empty_cache()
        return res

    def e2e(self, prec, stream, steps, world, torch):
        """Every step through the C ABI's host-buffer batch call (scd_batch_run_host, via
        BatchPlan.run_host): H2D of the input arena from page-locked host memory, both batched
        estimates, D2H of both output arenas into page-locked host memory (scd_host_alloc).
        Measured twice: one step after the other (`serial`, each step waits for its copies), and
        pipelined the way a stream of batches runs: the steps alternate between two device output
        sets, so that step k's results travel to the host (on each plan's copy stream) while step
        k + 1 computes; the timed region ends when the last step's results are in host memory."""
        fam, ssca = self.plans[prec]
        hx = self.binding.HostBuffer(self.x.numel(), self.x.dtype)
        hf = self.binding.HostBuffer(self.out_f.numel(), self.out_f.dtype)
        hs = self.binding.HostBuffer(self.out_s.numel(), self.out_s.dtype)
        hx.tensor.copy_(self.x.cpu())                 # the input batch, resident in host memory
        outs = [(self.out_f, self.out_s), (torch.empty_like(self.out_f), torch.empty_like(self.out_s))]
        samples = world * self.samples_per_step() * steps

        def one(k):
            of, os_ = outs[k % 2]
            fam.run_host(hx.tensor, self.x, of, hf.tensor, self.ws, stream=stream)
            ssca.run_host(None, self.x, os_, hs.tensor, self.ws, stream=stream)

        def drain():
            fam.host_wait()
            ssca.host_wait()
            stream.synchronize()

        def timed(pipelined):
            one(0)
            one(1)
            drain()
            barrier(world)
            t0 = time.perf_counter()
            for k in range(steps):
                one(k if pipelined else 0)
                if not pipelined:
                    drain()
            drain()
            return max_over_ranks(torch, time.perf_counter() - t0, world)

        dt_serial = timed(False)
        dt = timed(True)
        # one more serial step with events between its parts (not part of either timing)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        fam.run_host(hx.tensor, self.x, self.out_f, hf.tensor, self.ws, stream=stream)
        ev[1].record(stream)
        ssca.run_host(None, self.x, self.out_s, hs.tensor, self.ws, stream=stream)
        ev[2].record(stream)
        t0 = time.perf_counter()
        drain()
        parts = {"h2d_and_fam_ms": round(ev[0].elapsed_time(ev[1]), 2), "ssca_ms": round(ev[1].elapsed_time(ev[2]), 2),
                 "copies_after_compute_ms": round((time.perf_counter() - t0) * 1e3, 2)}
        d2h = (self.out_f.numel() + self.out_s.numel()) * 8
        del outs
        for h in (hx, hf, hs):
            h.close()
        torch.cuda.empty_cache()
        return {"value": samples / dt / 1e6, "unit": "Msamples/s",
                "h2d_bytes_per_step": self.x.numel() * 8, "d2h_bytes_per_step": d2h,
                "steps": steps, "ms_per_step": round(dt / steps * 1e3, 3),
                "d2h_gbs": round(d2h * steps / dt / 1e9, 1),
                "serial": {"value": round(samples / dt_serial / 1e6, 2), "ms_per_step": round(dt_serial / steps * 1e3, 3),
                           "parts": parts},
                "api": "scd_batch_run_host (BatchPlan.run_host) on page-locked host buffers from scd_host_alloc; "
                       "steps pipelined on two device output sets (step k's copies to the host while step k+1 "
                       "computes); `serial`: each step waits for its own copies"}


class PaperScaleWorkload:
    """FAM N=65,728 Np=256 L=64 P=1024 + map, SSCA N=2^20 Np=256 + map."""
    name = "paper_scale"
    FAM = dict(N=65728, Np=256, L=64, P=1024)
    SSCA = dict(N=1 << 20, Np=256)
    stages = ["fam_channelise", "fam_pair_fft", "fam_map", "ssca", "ssca_map"]
    n_marks = 9

    def __init__(self, rank=0, tune=True):
        from paper_2506_18003_gb300 import signals
        self.tune = tune
        self.wf = signals.fam_qam16_paper_scale(seed=signals.seed_for(2) + 100 * rank)
        self.ws_ = signals.ssca_mixture_1m(seed=signals.seed_for(3) + 100 * rank)

    def desc(self):
        return {"workload": "paper_scale: FAM N=65728 Np=256 L=64 P=1024 (16-QAM, RRC 0.25) + FAM map, "
                            "SSCA N=2^20 Np=256 (BPSK+QPSK mixture, 0 dB) + SSCA map",
                "fam": dict(self.FAM), "ssca": dict(self.SSCA), "window": "hamming",
                "l2": "working set per step > L2 (no flush needed)"}

    def samples_per_step(self):
        return self.FAM["N"] + self.SSCA["N"]

    def points_per_step(self):
        return self.FAM["Np"] ** 2 * self.FAM["P"] + self.SSCA["Np"] * self.SSCA["N"]

    def kernel_bytes(self):
        Np, L, P = self.FAM["Np"], self.FAM["L"], self.FAM["P"]
        N, Ns = self.SSCA["N"], self.SSCA["Np"]
        Q = P * L // Np
        return {"fam_channelise": 8 * ((P - 1) * L + Np) + 8 * Np * P, "fam_pair_fft": 8 * Np * Np * P,
                "fam_map": 8 * Np * Np * 2 * Q + 4 * (2 * Np) * (2 * P * L), "ssca": 8 * N + 8 * Ns * N,
                "ssca_map": 8 * Ns * N + 4 * Ns * 2 * N}

    def kernel_flops(self):
        F, S = self.FAM, self.SSCA
        ff = fam_flops(F["Np"], F["P"])
        return {"fam_channelise": F["P"] * (8 * F["Np"] + fft_flops(F["Np"])),
                "fam_pair_fft": ff - F["P"] * (8 * F["Np"] + fft_flops(F["Np"])),
                "fam_map": 0, "ssca": ssca_flops(S["Np"], S["N"]), "ssca_map": 0}

    def setup(self, torch, binding, dev, prec):
        self.torch, self.binding = torch, binding
        self.lib = binding.load()
        F, S = self.FAM, self.SSCA
        self.xf = torch.from_numpy(self.wf["x"]).to(dev)
        self.xs = torch.from_numpy(self.ws_["x"]).to(dev)
        self.Sf = torch.empty((F["Np"], F["Np"], F["P"]), dtype=torch.complex64, device=dev)
        self.Ss = torch.empty((S["Np"], S["N"]), dtype=torch.complex64, device=dev)
        self.Mf = torch.empty((2 * F["Np"], 2 * F["P"] * F["L"]), dtype=torch.float32, device=dev)
        self.Ms = torch.empty((S["Np"], 2 * S["N"]), dtype=torch.float32, device=dev)
        wsp = max(self.lib.scd_fam_workspace_bytes(F["N"], F["Np"], F["L"], F["P"], 0),
                  self.lib.scd_ssca_workspace_bytes(S["N"], S["Np"], 0), self.lib.scd_ssca_workspace_bytes(S["N"], S["Np"], 1))
        self.work = torch.empty(wsp, dtype=torch.uint8, device=dev)
        binding.scd_prepare("fam", F["N"], F["Np"], F["P"])
        binding.scd_prepare("ssca", S["N"], S["Np"])
        self.events = None
        if self.tune:                       # pick scd_ssca's schedule for both forms (outside timing)
            for p in ("fp32", "split"):
                binding.scd_ssca_tune(self.xs, S["Np"], out=self.Ss, precision=p, workspace=self.work, reps=2)
            torch.cuda.synchronize()

    def _opts(self, prec, stream, base, n):
        o = self.binding.make_opts(stream, prec, self.work)
        if self.events is not None:
            o.stage_events = ctypes.cast(ctypes.addressof(self.events) + base * ctypes.sizeof(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_void_p))
            o.n_stage_events = n
        return o

    def step(self, prec, stream, marks=None):
        lib, chk, F, S = self.lib, self.binding.check, self.FAM, self.SSCA
        self.events = marks
        o = self._opts(prec, stream, 0, 3)
        chk(lib.scd_fam(self.xf.data_ptr(), F["N"], F["Np"], F["L"], F["P"], None, self.Sf.data_ptr(),
                        ctypes.byref(o)), "fam")
        o = self._opts(prec, stream, 3, 2)
        chk(lib.scd_fam_map(self.Sf.data_ptr(), F["Np"], F["L"], F["P"], self.Mf.data_ptr(), ctypes.byref(o)), "fam_map")
        # the SSCA estimate may run as 1 or 3 kernels (autotuned schedule): time the whole call
        o = self._opts(prec, stream, 5, 0)
        o.stage_events, o.n_stage_events = None, 0
        st = ctypes.c_void_p(stream.cuda_stream)
        if marks is not None:
            chk(lib.scd_event_record(marks[5], st), "event")
        chk(lib.scd_ssca(self.xs.data_ptr(), S["N"], S["Np"], None, self.Ss.data_ptr(), ctypes.byref(o)), "ssca")
        if marks is not None:
            chk(lib.scd_event_record(marks[6], st), "event")
        o = self._opts(prec, stream, 7, 2)
        chk(lib.scd_ssca_map(self.Ss.data_ptr(), S["N"], S["Np"], self.Ms.data_ptr(), ctypes.byref(o)), "ssca_map")
        self.events = None

    def make_marks(self, n):
        arr = (ctypes.c_void_p * n)()
        self.binding.check(self.lib.scd_events_create(n, arr), "events")
        return arr

    def stage_times(self, ev):
        def el(a, b):
            f = ctypes.c_float()
            self.binding.check(self.lib.scd_event_elapsed_ms(ev[a], ev[b], ctypes.byref(f)), "elapsed")
            return f.value
        return {"fam_channelise": el(0, 1), "fam_pair_fft": el(1, 2), "fam_map": el(3, 4), "ssca": el(5, 6),
                "ssca_map": el(7, 8)}

    def e2e(self, prec, stream, steps, world, torch):
        lib, chk, F, S = self.lib, self.binding.check, self.FAM, self.SSCA
        xf = torch.from_numpy(self.wf["x"]).pin_memory()
        xs = torch.from_numpy(self.ws_["x"]).pin_memory()
        of = torch.empty((F["Np"], F["Np"], F["P"]), dtype=torch.complex64).pin_memory()
        os_ = torch.empty((S["Np"], S["N"]), dtype=torch.complex64).pin_memory()
        need = max(lib.scd_fam_host_workspace_bytes(F["N"], F["Np"], F["L"], F["P"], 0),
                   lib.scd_ssca_host_workspace_bytes(S["N"], S["Np"], 0))
        work = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        o = self.binding.make_opts(stream, prec, work)

        def one():
            chk(lib.scd_fam_host(xf.data_ptr(), F["N"], F["Np"], F["L"], F["P"], None, of.data_ptr(),
                                 ctypes.byref(o)), "fam_host")
            chk(lib.scd_ssca_host(xs.data_ptr(), S["N"], S["Np"], None, os_.data_ptr(), ctypes.byref(o)), "ssca_host")

        one()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(steps):
            one()
        dt = max_over_ranks(torch, time.perf_counter() - t0, world)
        return {"value": world * self.samples_per_step() * steps / dt / 1e6, "unit": "Msamples/s",
                "h2d_bytes_per_step": 8 * (F["N"] + S["N"]),
                "d2h_bytes_per_step": 8 * (F["Np"] ** 2 * F["P"] + S["Np"] * S["N"]), "steps": steps,
                "api": "scd_fam_host + scd_ssca_host (pinned host buffers, synchronous; maps not included)"}

    def oracle_sample(self, reduced=False):
        import numpy as np
        from oracle import scd_oracle as orc
        F, S = self.FAM, self.SSCA
        pairs, nslice, rows = (256, 1 << 12, 1) if reduced else (2048, 1 << 15, 8)
        g = np.random.default_rng(17)
        a = orc.hamming_window(F["Np"])
        t0 = time.perf_counter()
        orc.fam_pairs(self.wf["x"], a, F["Np"], F["L"], F["P"], g.integers(0, F["Np"], pairs),
                      g.integers(0, F["Np"], pairs))
        t_fam = (time.perf_counter() - t0) * F["Np"] ** 2 / pairs
        a2 = orc.hamming_window(S["Np"])
        n0 = int(g.integers(0, S["N"] - nslice))
        t0 = time.perf_counter()
        orc.ssca_cdp(self.ws_["x"], a2, S["Np"], np.arange(n0, n0 + nslice))
        t_cdp = (time.perf_counter() - t0) * S["N"] / nslice
        row = g.standard_normal((rows, S["N"])) + 1j * g.standard_normal((rows, S["N"]))
        t0 = time.perf_counter()
        for i in range(rows):
            orc.ssca_strip(row[i])
        t_strip = (time.perf_counter() - t0) * S["Np"] / rows
        desc = (f"FAM: {pairs} of {F['Np'] ** 2} pairs; SSCA: channeliser+CDP on {nslice} of {S['N']} samples + "
                f"{rows} of {S['Np']} strip rows; each scaled linearly to the full workload; maps not included")
        return t_fam + t_cdp + t_strip, desc


WORKLOADS = {"batch": BatchWorkload, "paper_scale": PaperScaleWorkload}


# ----------------------------------------------------------------------------- arms
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]()
    if hasattr(wl, "reference_step"):
        # the FP64 oracle on every host core, each step a real (not extrapolated) sample of the
        # workload: value = the samples those steps consumed / the time they took
        pool = OraclePool()
        used = secs = 0.0
        desc = ""
        for k in range(args.warmup + args.steps):
            u, t, desc = wl.reference_step(pool, k)
            if k >= args.warmup:
                used += u
                secs += t
        pool.close()
        cores = pool.cores
        v = used / secs / 1e6
        ms = secs / args.steps * 1e3
    else:
        steps = []
        desc = ""
        for i in range(args.warmup + args.steps):
            t, desc = wl.oracle_sample(reduced=True)
            if i >= args.warmup:
                steps.append(t)
        t = statistics.mean(steps)
        cores = 1
        v = wl.samples_per_step() / t / 1e6
        ms = t * 1e3
        desc += "; numpy FFT and elementwise kernels on one thread"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Msamples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": wl.desc(),
            "cpu_baseline": {"value": v, "unit": "Msamples/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "Msamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def strip_fft_rates(binding, lib, stream, xs, Ss, work, hbm, reps):
    """The SSCA's N-point strip FFT at N=2^20, Np=256 on its own: the staged schedule's three
    kernels timed with the library's stage events (channeliser + CDP, column pass, row pass;
    median of `reps` calls after 2 warm-ups, both forms).  Each four-step pass reads and writes
    the Np x N intermediate once (design traffic 2 x 8 Np N bytes per pass, which the ncu
    capture of these kernels at N=2^18 matches within 1%); the fraction is of the measured
    copy bandwidth."""
    import numpy as np
    N, Np = xs.numel(), Ss.shape[0]
    ev = (ctypes.c_void_p * 4)()
    binding.check(lib.scd_events_create(4, ev), "events")
    res = {"N": N, "Np": Np, "schedule": "stages", "bytes_per_pass": 2 * 8 * Np * N}
    for prec in ("fp32", "split"):
        o = binding.make_opts(stream, prec, work, schedule="stages")
        o.stage_events = ctypes.cast(ev, ctypes.POINTER(ctypes.c_void_p))
        o.n_stage_events = 4
        xp, op = ctypes.c_void_p(xs.data_ptr()), ctypes.c_void_p(Ss.data_ptr())
        rows = []
        for r in range(reps + 2):
            binding.check(lib.scd_ssca(xp, N, Np, None, op, ctypes.byref(o)), "scd_ssca")
            if r < 2:
                continue
            t = []
            for i in range(3):
                f = ctypes.c_float()
                binding.check(lib.scd_event_elapsed_ms(ev[i], ev[i + 1], ctypes.byref(f)), "elapsed")
                t.append(f.value)
            rows.append(t)
        cdp, cols, rows_ms = (float(v) for v in np.median(np.array(rows), axis=0))
        per_pass = 2 * 8 * Np * N
        res[prec] = {"channeliser_cdp_ms": round(cdp, 5), "column_pass_ms": round(cols, 5),
                     "row_pass_ms": round(rows_ms, 5),
                     "column_pass_hbm_frac": round(per_pass / (cols * 1e-3) / 1e9 / hbm, 4),
                     "row_pass_hbm_frac": round(per_pass / (rows_ms * 1e-3) / 1e9 / hbm, 4),
                     "strip_fft_hbm_frac": round(2 * per_pass / ((cols + rows_ms) * 1e-3) / 1e9 / hbm, 4)}
    lib.scd_events_destroy(4, ev)
    return res


def paper_match(torch, binding, dev, stream, reps):
    """The paper's own configurations (Sec. IV) on DSSS BPSK at 10 dB: FAM N=2048 (zero-padded to
    (P-1)L+Np = 2240), Np=256, L=64, P=32; SSCA N=2^20, Np=64.  Per call, CUDA events around
    `reps` calls after 2 warm-ups, FP32; the paper's VCK5000 times beside them as context only."""
    from paper_2506_18003_gb300 import signals
    res = {}
    Np, L, P = 256, 64, 32
    xf = torch.zeros((P - 1) * L + Np, dtype=torch.complex64, device=dev)
    xf[:2048] = torch.from_numpy(signals.dsss_bpsk(2048, 10.0, seed=9400)).to(dev)
    Sf = torch.empty((Np, Np, P), dtype=torch.complex64, device=dev)
    xs = torch.from_numpy(signals.dsss_bpsk(1 << 20, 10.0, seed=9401)).to(dev)
    Ss = torch.empty((64, 1 << 20), dtype=torch.complex64, device=dev)
    lib = binding.load()
    work = torch.empty(max(lib.scd_fam_workspace_bytes(xf.numel(), Np, L, P, 0),
                           lib.scd_ssca_workspace_bytes(1 << 20, 64, 0)), dtype=torch.uint8, device=dev)
    cases = {"fam": (lambda: binding.scd_fam(xf, Np, L, P, out=Sf, stream=stream, workspace=work), 2048, Np * Np * P,
                     0.630),
             "ssca": (lambda: binding.scd_ssca(xs, 64, out=Ss, stream=stream, workspace=work), 1 << 20, 64 << 20,
                      114.0)}
    with torch.cuda.stream(stream):
        for name, (fn, samples, points, paper_ms) in cases.items():
            for _ in range(2):
                fn()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                fn()
            t1.record(stream)
            t1.synchronize()
            ms = t0.elapsed_time(t1) / reps
            res[name] = {"ms": round(ms, 5), "msamples_per_s": round(samples / (ms * 1e-3) / 1e6, 2),
                         "scd_points_per_s": round(points / (ms * 1e-3), 0),
                         "context_paper_vck5000_ms": paper_ms}
    binding.scd_check_device(stream)
    del Sf, Ss, work
    torch.cuda.empty_cache()
    res["config"] = "FAM N=2048 (zero-padded to 2240) Np=256 L=64 P=32; SSCA N=2^20 Np=64; DSSS BPSK 10 dB; FP32"
    return res


def measure_variants(torch, binding, dev, stream, reps=10, warmup=2):
    """Times the cross / conjugate estimates and the alpha profiles at the paper-scale sizes
    (FAM N=65,728 Np=256 L=64 P=1024; SSCA N=2^20 Np=256), outside the step's timed region:
    CUDA events on the launching stream around `reps` calls after `warmup` calls; HBM
    fraction on algorithmic bytes (inputs read + outputs written)."""
    from paper_2506_18003_gb300 import signals
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, ValueError, KeyError):
        hbm = 6800.0
    wf = signals.fam_qam16_paper_scale()
    ws_ = signals.ssca_mixture_1m()
    Np, L, P, Nf = 256, 64, 1024, wf["x"].shape[0]
    Ns, Nps = ws_["x"].shape[0], 256
    Q = P * L // Np
    xf = torch.from_numpy(wf["x"]).to(dev)
    yf = torch.from_numpy(signals.modulated("qpsk", Nf, 4, 0.1, 10.0, seed=5100)).to(dev)
    xs = torch.from_numpy(ws_["x"]).to(dev)
    ys = torch.from_numpy(signals.modulated("qpsk", Ns, 4, 0.05, 5.0, seed=6200)).to(dev)
    Sf = torch.empty((Np, Np, P), dtype=torch.complex64, device=dev)
    Ss = torch.empty((Nps, Ns), dtype=torch.complex64, device=dev)
    pf = torch.empty(2 * P * L, dtype=torch.float32, device=dev)
    ps = torch.empty(2 * Ns, dtype=torch.float32, device=dev)
    lib = binding.load()
    # lengths that are not powers of two (Bluestein's identity): FAM P = 1000, SSCA N = 500,000
    Pa, Na = 1000, 500000
    work = torch.empty(max(lib.scd_fam_workspace_bytes(Nf, Np, L, P, 0), lib.scd_ssca_workspace_bytes(Ns, Nps, 0),
                           lib.scd_fam_workspace_bytes(Nf, Np, L, Pa, 0), lib.scd_ssca_workspace_bytes(Na, Nps, 0)),
                       dtype=torch.uint8, device=dev)
    used = (P - 1) * L + Np
    used_a = (Pa - 1) * L + Np
    cases = {
        "fam_cross": (lambda: binding.scd_fam(xf, Np, L, P, out=Sf, stream=stream, workspace=work, y=yf),
                      16 * used + 8 * Np * Np * P),
        "fam_conjugate": (lambda: binding.scd_fam(xf, Np, L, P, out=Sf, stream=stream, workspace=work, conjugate=True),
                          8 * used + 8 * Np * Np * P),
        "fam_alpha_profile": (lambda: binding.scd_fam_alpha_profile(Sf, Np, L, P, pf, stream=stream),
                              8 * Np * Np * 2 * Q + 4 * 2 * P * L),
        "ssca_cross": (lambda: binding.scd_ssca(xs, Nps, out=Ss, stream=stream, workspace=work, y=ys),
                       16 * Ns + 8 * Nps * Ns),
        "ssca_conjugate": (lambda: binding.scd_ssca(xs, Nps, out=Ss, stream=stream, workspace=work, conjugate=True),
                           8 * Ns + 8 * Nps * Ns),
        "ssca_alpha_profile": (lambda: binding.scd_ssca_alpha_profile(Ss, Ns, Nps, ps, stream=stream),
                               8 * Nps * Ns + 4 * 2 * Ns),
        "fam_any_p1000": (lambda: binding.scd_fam(xf[:used_a], Np, L, Pa, out=Sf.view(-1)[:Np * Np * Pa],
                                                  stream=stream, workspace=work),
                          8 * used_a + 8 * Np * Np * Pa),
        "ssca_any_n500000": (lambda: binding.scd_ssca(xs[:Na], Nps, out=Ss.view(-1)[:Nps * Na], stream=stream,
                                                      workspace=work),
                             8 * Na + 8 * Nps * Na),
    }
    out = {"ssca_strip_fft": strip_fft_rates(binding, lib, stream, xs, Ss, work, hbm, reps)}
    with torch.cuda.stream(stream):
        for name, (fn, nbytes) in cases.items():
            for _ in range(warmup):
                fn()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                fn()
            t1.record(stream)
            t1.synchronize()
            ms = t0.elapsed_time(t1) / reps
            out[name] = {"ms": round(ms, 5), "algorithmic_bytes": nbytes,
                         "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / hbm, 4)}
    binding.scd_check_device(stream)
    del Sf, Ss, work
    torch.cuda.empty_cache()
    out["paper_match"] = paper_match(torch, binding, dev, stream, reps)
    out["sizes"] = ("FAM N=65728 Np=256 L=64 P=1024; SSCA N=2^20 Np=256; any-length: FAM P=1000 (N=64,192), "
                    "SSCA N=500,000 (Bluestein, cyclic length 2^20); FP32 form; %d calls each" % reps)
    # streaming: one group of windows per step, new samples copied in from pinned host memory
    # every step (scd_stream_advance) and the plan's graph replayed (scd_batch_run)
    for name, est, W, hop, nwin, Npw, Lw in (("ssca_stream", "ssca", 1 << 16, 1 << 15, 16, 256, 1),
                                              ("fam_stream", "fam", 65728, 16384, 8, 256, 64)):
        plan = binding.StreamPlan(est, W, hop, nwin, Npw, Lw)
        total = plan.span + (reps + warmup) * nwin * hop
        sx = signals.modulated("qpsk", total, 4, 0.1, 10.0, seed=6300)
        arena = torch.from_numpy(sx[:plan.span].copy()).to(dev)
        # group k >= 1 takes the samples from k*nwin*hop + keep = span + (k-1)*nwin*hop on
        chunks = [torch.from_numpy(sx[plan.span + g * nwin * hop:][:nwin * hop].copy()).pin_memory()
                  for g in range(reps + warmup)]
        sout = torch.empty(plan.out_offsets[-1], dtype=torch.complex64, device=dev)
        sws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device=dev)
        with torch.cuda.stream(stream):
            plan.run(arena, sout, sws, stream=stream)
            for g in range(warmup):
                plan.advance(arena, chunks[g], stream=stream)
                plan.run(arena, sout, sws, stream=stream)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for g in range(warmup, warmup + reps):
                plan.advance(arena, chunks[g], stream=stream)
                plan.run(arena, sout, sws, stream=stream)
            t1.record(stream)
            t1.synchronize()
        binding.scd_check_device(stream)
        ms = t0.elapsed_time(t1) / reps
        nbytes = 8 * nwin * hop + (plan.out_offsets[-1]) * 8
        out[name] = {"ms_per_group": round(ms, 5), "windows_per_group": nwin, "window": W, "hop": hop, "Np": Npw,
                     "stream_msamples_per_s": round(nwin * hop / (ms * 1e-3) / 1e6, 2),
                     "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / hbm, 4),
                     "timed": "host-to-device copy of the group's new samples + the persistent launch"}
        plan.close()
        del arena, sout, sws
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    from paper_2506_18003_gb300 import binding

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    oracle_pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "batch":
        oracle_pool = OraclePool()          # worker processes spawned before this process touches the GPU
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = binding.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    wl = WORKLOADS[args.workload](rank, tune=not args.no_tune)
    with torch.cuda.stream(stream):
        wl.setup(torch, binding, dev, args.precision)
    torch.cuda.synchronize()

    def marks_for(n):
        if hasattr(wl, "make_marks"):
            return wl.make_marks(n)
        return [torch.cuda.Event(enable_timing=True) for _ in range(n)]

    def timed(prec):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                wl.step(prec, stream)
        torch.cuda.synchronize()
        binding.scd_check_device(stream)
        marks = [marks_for(wl.n_marks) for _ in range(args.steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        launches0 = lib.scd_launch_count()
        with ClockSampler(local) as clk, torch.cuda.stream(stream):
            t0.record(stream)
            for s in range(args.steps):
                wl.step(prec, stream, marks[s])
            t1.record(stream)
            torch.cuda.synchronize()
        launches = lib.scd_launch_count() - launches0
        barrier(world)
        binding.scd_check_device(stream)
        ms = max_over_ranks(torch, t0.elapsed_time(t1), world)
        stage = {k: 0.0 for k in wl.stages}
        for m in marks:
            for k, v in wl.stage_times(m).items():
                stage[k] += v / args.steps
        if hasattr(wl, "make_marks"):
            for m in marks:
                lib.scd_events_destroy(len(m), m)
        return ms / args.steps, stage, int(launches), clk.summary()

    prec = args.precision
    other = "split" if prec == "fp32" else "fp32"
    ms_step, stage_ms, launches, clocks = timed(prec)
    ms_other, stage_other, _, _ = timed(other)

    kb = wl.kernel_bytes()
    top = max(stage_ms, key=stage_ms.get)
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {}
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback 6800 GB/s"
    hbm = hbm or 6800.0
    # roofline of the dominant kernel: whichever floor is higher, its algorithmic bytes at the
    # measured HBM bandwidth or its algorithmic FLOPs at the FP32 CUDA-core peak
    kf = wl.kernel_flops()
    # FP32 CUDA-core peak from this device's SM count and the SM clock sampled under load
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    alu_peak = fp32_peak_tflops(sm_count, clock_mhz)
    alu_bound = kf[top] / (alu_peak * 1e12) > kb[top] / (hbm * 1e9)
    ach_gbs = kb[top] / (stage_ms[top] * 1e-3) / 1e9
    ach_tf = kf[top] / (stage_ms[top] * 1e-3) / 1e12
    if alu_bound:
        roof = {"bound": "alu", "kernel": top, "achieved": ach_tf, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": ach_tf / alu_peak, "peak_source": f"derived FP32 CUDA-core peak: sm_count x 128 lanes x "
                f"2 FLOP x clock_mhz (median SM clock sampled in the timed region)", "sm_count": sm_count,
                "clock_mhz": clock_mhz, "algorithmic_flops": kf[top], "hbm_frac": ach_gbs / hbm,
                "hbm_peak": hbm, "algorithmic_bytes": kb[top]}
    else:
        roof = {"bound": "hbm", "kernel": top, "achieved": ach_gbs, "peak": hbm, "unit": "GB/s",
                "frac": ach_gbs / hbm, "peak_source": peak_src, "algorithmic_bytes": kb[top],
                "alu_frac": ach_tf / alu_peak, "alu_peak": alu_peak, "sm_count": sm_count, "clock_mhz": clock_mhz,
                "algorithmic_flops": kf[top]}
    roof["traffic"] = captured_traffic(top) if prec == "fp32" else None
    if roof["traffic"]:
        # the captured DRAM bytes at the live stage time, against the copy bandwidth: how close
        # the stage runs to HBM on the traffic it really moves
        roof["traffic_hbm_frac"] = roof["traffic"] / (stage_ms[top] * 1e-3) / 1e9 / hbm
    value = job_throughput(world, wl.samples_per_step(), ms_step * 1e-3) / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[prec],
        "data": "synthetic (seeded modulated signals of the paper's shapes)", "config": wl.desc(),
        "scd_points_per_s": world * wl.points_per_step() / (ms_step * 1e-3),
        "gpu_launches": launches,
        "stage_ms": {k: round(v, 5) for k, v in stage_ms.items()},
        "roofline": roof,
        "rates": wl.rates(stage_ms, ms_step) if hasattr(wl, "rates") else None,
        "stage_hbm_frac": {k: round(kb[k] / (v * 1e-3) / 1e9 / hbm, 4) for k, v in stage_ms.items() if v > 0},
        "stage_alu_frac": {k: round(kf[k] / (v * 1e-3) / 1e12 / alu_peak, 4) for k, v in stage_ms.items()
                           if v > 0 and kf[k]},
        "clocks": clocks,
        "parity_gate": {"fp32": "max|dS|/max|S| <= 1e-5 vs FP64 oracle (tests)",
                        "split": "<= 1e-3 (tests; measured ~2e-6)"},
        other: {"value": world * wl.samples_per_step() / (ms_other * 1e-3) / 1e6, "unit": "Msamples/s",
                "ms_per_step": ms_other, "dtype": DTYPE[other],
                "stage_ms": {k: round(v, 5) for k, v in stage_other.items()},
                f"speedup_vs_{prec}": ms_step / ms_other},
    }
    if not args.no_e2e:
        with torch.cuda.stream(stream):
            line["e2e"] = wl.e2e(prec, stream, min(args.steps, args.e2e_steps), world, torch)
    if not args.no_variants:
        if hasattr(wl, "profile_mode"):
            line["profile_output"] = wl.profile_mode(torch, binding, stream)
        if hasattr(wl, "exact_ssca"):
            line["ssca_exact_lengths"] = wl.exact_ssca(torch, binding, stream)
        line["variants"] = measure_variants(torch, binding, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if hasattr(wl, "cpu_baseline"):
            v, t, desc = wl.cpu_baseline(oracle_pool)
            line["cpu_baseline"] = {"value": v, "unit": "Msamples/s", "cores": oracle_pool.cores, "kind": "oracle",
                                    "sample": desc, "wall_s": round(t, 3)}
            oracle_pool.close()
            wl.parity_refs()
        else:
            t, desc = wl.oracle_sample()
            line["cpu_baseline"] = {"value": wl.samples_per_step() / t / 1e6, "unit": "Msamples/s", "cores": 1,
                                    "kind": "oracle", "sample": desc + "; numpy FFT and elementwise kernels on one thread"}
        if getattr(wl, "oracle_refs", None):
            with torch.cuda.stream(stream):
                line["cpu_baseline"]["parity"] = wl.parity_sample(stream)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="batch")
    ap.add_argument("--precision", choices=["fp32", "split"], default="fp32")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default sizing)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the cross / conjugate / alpha-profile timings at paper-scale sizes")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
