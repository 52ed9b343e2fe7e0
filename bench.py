"""Benchmark: TF-bin EM iterations per second of FastFCA (and conventional FCA) on GB300.

Headline (the workload the metric is quoted on): one mixture M=4, F=513, N=1000, L=50,
complex64, seeded synthetic (mask-based initialisation). One step = one whole EM job: load the
mixture and initial parameters into the library state (device-resident inputs) with the initial
generalised eigendecomposition, L FastFCA iterations with the per-iteration log-likelihood, and
the posterior means (Algorithm 1). bin-iters per step = F * N * L.

The same line carries, as sub-records measured in the same run:
  precision  M=8, F=1025, N=4000, L=100, y stored as FP16 with a per-frequency scale;
  batch      512 mixtures (M in {2,4,6}, N in [200,6000], F=513, L=50) as one CUDA-graph job,
             against per-mixture launches;
  serve      requests (M in {2,4,8}, N in [60,1000], F=513, L=30) arriving at 200/s;
each with FastFCA and conventional rates, errors against the FP64 oracle and the oracle's own
rate on the host cores; and the three eigensolver precisions (FCA_GEVD_*) at the headline and
precision workloads, with their errors from both initialisations.

Under torchrun each rank runs its own mixture (weak scaling: frequencies and mixtures are
independent, there is no exchange on the data path); value = all ranks' bin-iters / the
slowest rank's time; the sub-records are measured at N=1 only.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload all|mid|precision|batch|serve] [--no-cpu-baseline]

--impl reference times the FP64 CPU oracle (the reference of this project) on the host
cores on a bounded sample of the headline workload.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TF-bin EM iters/s, FastFCA vs frame-wise FCA on 1 GB300, rel err ≤1e-4 vs FP64"
UNIT = "bin-iters/s"
TOLERANCE = "median <= 1e-4, max <= 1e-3 (v, mu, S); ll <= 1e-6 relative"
MODES = {"fp32": 0, "fp64": 1, "refined": 2}  # FCA_GEVD_*; "refined" is the library default


# ------------------------------------------------------------------------------ accounting
def bytes_per_bin_iter(M: int, storage: str = "c64") -> int:
    """Streaming byte model: a TF-bin-iteration reads y (8M bytes as complex64, 4M as FP16
    pairs) and reads and writes v (2 x 8 bytes: two sources, FP32) if nothing stays on chip."""
    return (8 if storage == "c64" else 4) * M + 16


def fast_flops_per_bin_iter(M: int) -> int:
    """Algorithmic FP32 flops of one FastFCA time-frequency point per iteration (counted from
    the equations: P^H y 8M^2; d, 1/d, |yt|^2, the mut coefficients 9M; the two v updates
    9M+2; two rank-1-plus-diagonal Gram updates 2(5M^2+3M+1); log-likelihood terms 3M)."""
    return 18 * M * M + 27 * M + 4


def conv_flops_per_bin_iter(M: int) -> int:
    """Algorithmic FP32 flops of one conventional time-frequency point per iteration: Rx
    4M^2; Cholesky 4M^3/3; two triangular solves for u 8M^2; mu_1, mu_2 16M^2; L^-1 S_1 and
    L^-1 S_2 8M^3; C = v1 v2 (L^-1 S1)^H (L^-1 S2), upper triangle 4M^3; the v updates as sums of
    squares (K_j^H u 8M^2, L^-1 K_j 8M^3/3); two Gram updates 2(5M^2+3M+1); log-likelihood
    terms 3M."""
    return round(4 * M**3 / 3 + 8 * M**3 + 4 * M**3 + 8 * M**3 / 3) + 4 * M * M + 8 * M * M \
        + 16 * M * M + 8 * M * M + 2 * (5 * M * M + 3 * M + 1) + 3 * M


def hbm_peak():
    """HBM bandwidth the rooflines are stated against: the driver's measured copy bandwidth
    (MEASURED_PEAKS.json) when present, else the profiling recipe's fallback figure."""
    try:
        v = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement)"


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from profiles/dram_traffic.json (written by
    paper_1805_06572_gb300.ncu_traffic from an Nsight Compute capture), if it was captured at
    the current kernel source; else None."""
    from paper_1805_06572_gb300.ncu_traffic import source_sha
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))[kernel]
    except (OSError, ValueError, KeyError):
        return None
    if rec.get("source_sha") != source_sha():
        return None
    return rec.get("bytes_per_launch")


def roofline(M, units, kernel_ms, peaks, flops_fn, kernel, storage="c64", mode=None):
    """Roofline of a fused EM kernel: the streaming HBM model (bytes_per_bin_iter: 48 B per
    TF-bin-iteration at M=4) and, next to it, the FP32 ALU fraction against the FP32 FMA peak
    measured in this run."""
    hbm, hbm_src = peaks["hbm_gbs"], peaks["hbm_src"]
    gbs = bytes_per_bin_iter(M, storage) * units / (kernel_ms / 1e3) / 1e9
    tf = flops_fn(M) * units / (kernel_ms / 1e3) / 1e12
    out = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
           "traffic": profiled_traffic(kernel), "kernel": kernel, "kernel_ms": kernel_ms,
           "bytes_per_bin_iter": bytes_per_bin_iter(M, storage), "peak_source": hbm_src,
           "alu": {"achieved": tf, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                   "frac": tf / peaks["fp32_tflops"], "flops_per_bin_iter": flops_fn(M),
                   "peak_source": "FP32 FMA throughput measured in this run (fca_measure_peaks)"}}
    if mode is not None:
        out["eigensolver"] = mode
    return out


# -------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons over the whole benchmark;
    the summary keeps the samples that fall inside the timed regions (mark())."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.regions, self.lines = index, None, [], []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def stop(self):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
            self.proc = None

    def mark(self, label, t0, t1):
        self.regions.append((label, t0, t1))

    def summary(self, labels=None):
        sm, mx, reasons, n = [], None, set(), 0
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                clk, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            if not any(t0 - 0.1 <= ts <= t1 + 0.1 for lab, t0, t1 in self.regions
                       if labels is None or lab in labels):
                continue
            n += 1
            sm.append(clk)
            for name, p in zip(self.NAMES, parts[4:8]):
                if p.lower() in ("active", "1"):
                    reasons.add(name)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
               "reasons": sorted(reasons), "samples": n,
               "window": "nvidia-smi samples inside the timed regions" +
                         ("" if labels is None else f" of {sorted(labels)}")}
        return out


# ------------------------------------------------------------------------------- helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_rate(y, v0, S0, iters, n_bins, form="fast", min_seconds=0.0, nthreads=0):
    """Time the FP64 oracle (as it stands) on a bounded sample: n_bins frequencies spread over
    the band, all frames, all iterations, repeated until at least min_seconds of work, on
    nthreads host threads (0: all cores). Returns (bin-iters/s, seconds, threads, sample, bins,
    the last result)."""
    import numpy as np

    import oracle
    F = y.shape[0]
    fs = np.unique(np.linspace(0, F - 1, n_bins).round().astype(int))
    ys = np.asarray(y)[fs].astype(np.complex128)
    reps, dt = 0, 0.0
    while reps == 0 or dt < min_seconds:
        t0 = time.perf_counter()
        res = oracle.em(form, ys, v0[:, fs], S0[:, fs], iters, want_mu=True, nthreads=nthreads)
        dt += time.perf_counter() - t0
        reps += 1
    units = reps * len(fs) * ys.shape[1] * iters
    return (units / dt, dt, nthreads or oracle.threads(),
            f"{reps} x ({len(fs)} of {F} bins x N={ys.shape[1]} x L={iters})", fs, res)


def parity_errors(gpu, ref, y, fs=None):
    """Errors of GPU outputs against the oracle (the parity tests' metrics), over the bins the
    oracle ran on: per entry |v - v*| / v*, ||mu - mu*|| / ||y|| per time-frequency point,
    ||S - S*||_F / ||S*||_F per bin, and the largest relative log-likelihood error over the
    iterations (summed over those bins). Returns {name: [median, max]}."""
    import numpy as np
    sel = slice(None) if fs is None else fs
    ys = np.asarray(y)[sel]
    ev = np.abs(gpu["v"][:, sel] - ref["v"]) / ref["v"]
    yn = np.linalg.norm(ys, axis=2)
    yn = np.where(yn > 0, yn, 1.0)
    emu = np.stack([np.linalg.norm(gpu["mu1"][sel] - ref["mu1"], axis=2) / yn,
                    np.linalg.norm(gpu["mu2"][sel] - ref["mu2"], axis=2) / yn])
    out = {"v": [float(np.median(ev)), float(ev.max())],
           "mu": [float(np.median(emu)), float(emu.max())]}
    if gpu.get("S") is not None:
        eS = np.linalg.norm(gpu["S"][:, sel] - ref["S"], axis=(2, 3)) / np.linalg.norm(ref["S"], axis=(2, 3))
        out["S"] = [float(np.median(eS)), float(eS.max())]
    if gpu.get("llf") is not None and len(ref["ll"]):
        llr = ref["ll"].sum(axis=1)
        ell = np.abs(gpu["llf"][:, sel].sum(axis=1) - llr) / np.abs(llr)
        out["ll"] = [float(np.median(ell)), float(ell.max())]
    return out


def timed_events(fn, steps, before=None):
    """CUDA-event time (ms) of each of `steps` calls of fn on the current stream."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    out = []
    for k in range(steps):
        if before is not None:
            before()
        evs[k][0].record()
        r = fn()
        evs[k][1].record()
        out.append(r)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs], out


# --------------------------------------------------------------------- one-mixture jobs
class OneMixture:
    """A mixture resident on the device, a library state, and the outputs of a whole job."""

    def __init__(self, fca, torch, y, v0, S0, iters, y_scale=None, dev=None):
        self.fca, self.torch = fca, torch
        self.dev = dev or torch.device("cuda")
        self.y, self.v0, self.S0, self.g, self.L = y, v0, S0, y_scale, iters
        self.st = fca.fca_init(y, v0, S0, y_scale=y_scale)
        F, N, M = self.st.F, self.st.N, self.st.M
        self.F, self.N, self.M = F, N, M
        self.x1 = torch.empty((F, N, M), dtype=torch.complex64, device=self.dev)
        self.x2 = torch.empty_like(self.x1)
        self.ll = torch.empty(max(iters, 1), dtype=torch.float64, device=self.dev)

    def step(self, form="fast", mode=None):
        fca = self.fca
        fca.fca_load(self.st, self.y, self.v0, self.S0, y_scale=self.g)
        if mode is not None:
            fca.fca_set_eigensolver(self.st, mode, 30)
        (fca.fca_em_fast if form == "fast" else fca.fca_em_conventional)(self.st, self.L, self.ll)
        fca.fca_separate(self.st, self.x1, self.x2, fca.FCA_SEP_ALG1)

    def kernel_ms(self):
        return self.fca.fca_last_em_kernel_ms(self.st)

    def outputs(self, fs=None):
        import numpy as np
        torch, fca = self.torch, self.fca
        v = torch.empty((2, self.F, self.N), dtype=torch.float32, device=self.dev)
        S = torch.empty((2, self.F, self.M, self.M), dtype=torch.complex128)
        fca.fca_get_params(self.st, v=v, S=S)
        assert fca.fca_sync_status(self.st) == 0
        return {"v": v.cpu().numpy().astype(np.float64), "S": S.numpy(), "mu1": self.x1.cpu().numpy(),
                "mu2": self.x2.cpu().numpy(), "llf": fca.fca_loglik_bins(self.st).numpy()}

    def free(self):
        self.fca.fca_free(self.st)


def kernel_ms_of(job, form, mode, steps):
    """Mean CUDA-event time of the fused EM kernel over `steps` whole jobs."""
    ks = []
    for _ in range(steps):
        job.step(form, mode)
        ks.append(job.kernel_ms())
    return statistics.mean(ks)


def mode_records(job, y_ref, v0, S0, iters, oracles, steps, fs=None, y_scale_note=""):
    """Kernel time and errors against the oracle of each eigensolver precision, from the
    initialisations in `oracles` ({recipe: (v0, S0, oracle result)})."""
    fca = job.fca
    out = {}
    for name, mode in MODES.items():
        rec = {"kernel_ms": kernel_ms_of(job, "fast", mode, steps)}
        for recipe, (v0r, S0r, ref) in oracles.items():
            fca.fca_load(job.st, job.y, v0r, S0r, y_scale=job.g)
            fca.fca_set_eigensolver(job.st, mode, 30)
            fca.fca_em_fast(job.st, iters, job.ll)
            fca.fca_separate(job.st, job.x1, job.x2, fca.FCA_SEP_ALG1)
            rec[f"errors_{recipe}"] = parity_errors(job.outputs(), ref, y_ref, fs)
        out[name] = rec
    fca.fca_set_eigensolver(job.st, fca.FCA_GEVD_DEFAULT, 30)
    return out


# ---------------------------------------------------------------------------- headline
def run_mid(args, fca, torch, dev, peaks, clk, world, rank):
    """The headline: one mixture M=4, F=513, N=1000, L=50 per step (per rank)."""
    import numpy as np

    import synth
    import torch.distributed as dist
    from paper_1805_06572_gb300.shard import allreduce_max, weak_scaling_value

    c, mix, v0, S0 = synth.make_config("mid", mixture_index=rank)
    F, N, M, L = c.F, c.N, c.M, c.iters
    units = F * N * L
    y_h = torch.from_numpy(mix["y"]).pin_memory()
    v0_h = torch.from_numpy(v0).pin_memory()
    S0_h = torch.from_numpy(S0).pin_memory()
    y_d, v0_d, S0_d = y_h.to(dev), v0_h.to(dev), S0_h.to(dev)
    job = OneMixture(fca, torch, y_d, v0_d, S0_d, L, dev=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        return x if world == 1 else allreduce_max(x, dist, device=dev)

    def timed(form, steps, mode=None):
        barrier()
        l0 = fca.fca_kernel_launches()
        t0 = time.time()
        ms, _ = timed_events(lambda: job.step(form, mode), steps, before=flush.zero_)
        barrier()
        t1 = time.time()
        return ms, t0, t1, fca.fca_kernel_launches() - l0

    for _ in range(args.warmup):
        job.step("fast")
    torch.cuda.synchronize()
    if fca.fca_sync_status(job.st) != 0:
        raise RuntimeError("device status error during warm-up")
    ms_fast, t0, t1, launches = timed("fast", args.steps)
    clk.mark("mid", t0, t1)
    if fca.fca_sync_status(job.st) != 0:
        raise RuntimeError("device status error in the timed region")
    kern_fast = kernel_ms_of(job, "fast", None, max(3, args.steps // 2))

    steps_conv = max(3, args.steps // 2)
    for _ in range(3):
        job.step("conventional")
    ms_conv, t0c, t1c, _ = timed("conventional", steps_conv)
    clk.mark("mid", t0c, t1c)
    kern_conv = kernel_ms_of(job, "conventional", None, 3)

    # End to end through the public API as a caller streaming mixtures would run it: two
    # states on two CUDA streams, so one mixture's host<->device copies overlap the other's
    # kernels. Every step copies its inputs from pinned host memory and its outputs (posterior
    # means and log-likelihood) back.
    streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    states = [job.st, fca.fca_init(y_d, v0_d, S0_d)]
    bufs = []
    for _ in range(2):
        bufs.append((torch.empty_like(job.x1), torch.empty_like(job.x2), torch.empty_like(job.ll),
                     torch.empty(job.x1.shape, dtype=torch.complex64).pin_memory(),
                     torch.empty(job.x2.shape, dtype=torch.complex64).pin_memory(),
                     torch.empty(job.ll.shape, dtype=torch.float64).pin_memory()))

    def step_e2e(k):
        s, stk = streams[k % 2], states[k % 2]
        a, b, l, ah, bh, lh = bufs[k % 2]
        with torch.cuda.stream(s):
            fca.fca_load(stk, y_h, v0_h, S0_h, stream=s)
            fca.fca_em_fast(stk, L, l, stream=s)
            fca.fca_separate(stk, a, b, fca.FCA_SEP_ALG1, stream=s)
            ah.copy_(a, non_blocking=True)
            bh.copy_(b, non_blocking=True)
            lh.copy_(l, non_blocking=True)

    for k in range(4):
        step_e2e(k)
    barrier()
    t0e = time.perf_counter()
    for k in range(args.steps):
        step_e2e(k)
    barrier()
    wall_e2e = time.perf_counter() - t0e
    if fca.fca_sync_status(states[0]) != 0 or fca.fca_sync_status(states[1]) != 0:
        raise RuntimeError("device status error")

    t_fast = max_over_ranks(sum(ms_fast) / 1e3)
    t_conv = max_over_ranks(sum(ms_conv) / 1e3)
    t_e2e = max_over_ranks(wall_e2e)
    value = weak_scaling_value(units * args.steps, world, t_fast)
    conv_value = weak_scaling_value(units * steps_conv, world, t_conv)
    e2e_value = weak_scaling_value(units * args.steps, world, t_e2e)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_over_ranks(statistics.mean(ms_fast)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"mid: M={M} F={F} N={N} L={L}, 2 sources, complex64, seeded mixture "
                               f"per rank (delta={c.delta}, sigma={c.sigma}), mask-based initialisation",
                   "form": "FastFCA", "eigensolver": "refined (library default: Gram merge as compensated FP32 pairs, "
                   "FP32 Newton/Jacobi solve, compensated-FP32 refinement step)",
                   "l2": "flushed between steps (256 MiB write, outside the step events)",
                   "parallelism": f"replicas x{world}",
                   "step": "load + initial GEVD + L iterations with log-likelihood + posterior means"},
        "roofline": roofline(M, units, kern_fast, peaks, fast_flops_per_bin_iter,
                             "fast_em_kernel<4,c64,128,refined>"),
        "conventional": {"value": conv_value, "unit": UNIT, "ms_per_step": statistics.mean(ms_conv),
                         "steps": steps_conv, "kernel_ms": kern_conv, "fast_speedup": value / conv_value,
                         "roofline": roofline(M, units, kern_conv, peaks, conv_flops_per_bin_iter,
                                              "conv_em_kernel<4,c64,128>")},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": y_h.numel() * 8 + v0_h.numel() * 8 + S0_h.numel() * 16,
                "d2h_bytes_per_step": job.x1.numel() * 8 * 2 + job.ll.numel() * 8,
                "ms_per_step": 1e3 * wall_e2e / args.steps,
                "timing": "host wall clock around all steps, synchronised on both sides; two states "
                          "on two streams (copies of one step overlap another's kernels)"},
        "gpu_launches": launches,
    }
    fca.fca_free(states[1])
    if rank == 0 and world == 1:
        # The oracle on the same inputs (both initialisations, both forms) and the errors of each
        # form and eigensolver precision against it.
        import oracle
        y64 = mix["y"].astype(np.complex128)
        _, _, v0r, S0r = synth.make_config("mid", recipe="random")
        if not args.no_cpu_baseline:
            rate, dt, threads, sample, _, ref_fast = cpu_oracle_rate(y64, v0, S0, L, F, min_seconds=10.0)
            rate_c, dt_c, _, sample_c, _, ref_conv = cpu_oracle_rate(y64, v0, S0, L, F, form="conventional",
                                                                     min_seconds=10.0)
            rate_1, dt_1, _, sample_1, _, _ = cpu_oracle_rate(y64, v0, S0, L, 32, min_seconds=3.0, nthreads=1)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                    "sample": f"FastFCA form, {sample} ({dt:.1f} s)",
                                    "conventional_value": rate_c,
                                    "conventional_sample": f"{sample_c} ({dt_c:.1f} s)",
                                    "one_thread": {"value": rate_1, "cores": 1,
                                                   "sample": f"FastFCA form, {sample_1} ({dt_1:.1f} s)"}}
        else:
            ref_fast = oracle.em("fast", y64, v0, S0, L)
            ref_conv = oracle.em("conventional", y64, v0, S0, L)
        ref_fast_r = oracle.em("fast", y64, v0r, S0r, L)
        ref_conv_r = oracle.em("conventional", y64, v0r, S0r, L)
        v0r_d, S0r_d = torch.from_numpy(v0r).to(dev), torch.from_numpy(S0r).to(dev)
        parity = {}
        for form, refs in (("fast", {"mask": ref_fast, "random": ref_fast_r}),
                           ("conventional", {"mask": ref_conv, "random": ref_conv_r})):
            for recipe, ref in refs.items():
                vv, ss = (v0_d, S0_d) if recipe == "mask" else (v0r_d, S0r_d)
                fca.fca_load(job.st, y_d, vv, ss)
                (fca.fca_em_fast if form == "fast" else fca.fca_em_conventional)(job.st, L, job.ll)
                fca.fca_separate(job.st, job.x1, job.x2, fca.FCA_SEP_ALG1)
                parity[f"{form}_{recipe}"] = parity_errors(job.outputs(), ref, y64)
        line["parity_vs_oracle"] = dict(parity, tolerance=TOLERANCE,
                                        note="mask: the benchmark's initialisation; random: the "
                                             "seeded random initialisation of the same mixture")
        line["eigensolver_modes"] = mode_records(
            job, y64, v0, S0, L, {"mask": (v0_d, S0_d, ref_fast), "random": (v0r_d, S0r_d, ref_fast_r)},
            max(3, args.steps // 4))
    job.free()
    return line


# ------------------------------------------------------------------------- precision
def run_precision(args, fca, torch, dev, peaks, clk):
    """M=8, F=1025, N=4000, L=100; the mixture stored as FP16 pairs with a per-frequency power
    scale; FP32 bin arithmetic; the eigensolver precisions of FCA_GEVD_*. Same step as the
    headline. The oracle runs on the decoded FP16 mixture."""
    import numpy as np

    import oracle
    import synth
    c, mix, v0, S0 = synth.make_config("precision")
    y16, g, deq = synth.quantize_f16(mix["y"])
    F, N, M, L = c.F, c.N, c.M, c.iters
    units = F * N * L
    yd, gd = torch.from_numpy(y16).to(dev), torch.from_numpy(g).to(dev)
    v0d, S0d = torch.from_numpy(v0).to(dev), torch.from_numpy(S0).to(dev)
    job = OneMixture(fca, torch, yd, v0d, S0d, L, y_scale=gd, dev=dev)
    steps = max(3, args.steps // 2)
    for _ in range(3):
        job.step("fast")
    t0 = time.time()
    ms, _ = timed_events(lambda: job.step("fast"), steps)
    clk.mark("precision", t0, time.time())
    kf = kernel_ms_of(job, "fast", None, 3)
    job.step("conventional")
    t0 = time.time()
    ms_c, _ = timed_events(lambda: job.step("conventional"), max(2, steps // 3))
    clk.mark("precision", t0, time.time())
    kc = kernel_ms_of(job, "conventional", None, 2)
    t, tc = statistics.mean(ms) / 1e3, statistics.mean(ms_c) / 1e3
    rec = {"workload": f"precision: M={M} F={F} N={N} L={L}, y as FP16 pairs with a per-frequency "
                       "scale, seeded (delta=0.05, sigma=1.5), mask-based initialisation",
           "value": units / t, "unit": UNIT, "ms_per_step": 1e3 * t, "steps": steps,
           "dtype": "f32 (y stored f16)",
           "l2": "inputs (131 MB FP16 mixture + source powers) larger than L2",
           "roofline": roofline(M, units, kf, peaks, fast_flops_per_bin_iter,
                                "fast_em_kernel<8,f16,128,refined>", storage="f16"),
           "conventional": {"value": units / tc, "ms_per_step": 1e3 * tc, "kernel_ms": kc,
                            "fast_speedup": tc / t,
                            "roofline": roofline(M, units, kc, peaks, conv_flops_per_bin_iter,
                                                 "conv_em_kernel<8,f16,128>", storage="f16")}}
    # Errors against the oracle: FastFCA on every bin, conventional on a sample of bins (bins
    # are independent, so a sample is exact). The oracle's FastFCA run is also the CPU baseline.
    t0 = time.perf_counter()
    ref = oracle.em("fast", deq, v0, S0, L)
    dt = time.perf_counter() - t0
    rec["cpu_baseline"] = {"value": units / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                           "sample": f"FastFCA form, the whole workload once ({dt:.1f} s)"}
    fs = np.array([0, 1, 200, 511, 512, 777, 1023, 1024])
    ref_c = oracle.em("conventional", deq[fs], v0[:, fs], S0[:, fs], L)
    job.step("fast")
    rec["parity_vs_oracle"] = {"fast_mask": parity_errors(job.outputs(), ref, deq)}
    job.step("conventional")
    rec["parity_vs_oracle"]["conventional_mask"] = parity_errors(job.outputs(), ref_c, deq, fs)
    _, _, v0r, S0r = synth.make_config("precision", recipe="random")
    ref_r = oracle.em("fast", deq, v0r, S0r, L)
    v0r_d, S0r_d = torch.from_numpy(v0r).to(dev), torch.from_numpy(S0r).to(dev)
    fca.fca_load(job.st, yd, v0r_d, S0r_d, y_scale=gd)
    fca.fca_em_fast(job.st, L, job.ll)
    fca.fca_separate(job.st, job.x1, job.x2, fca.FCA_SEP_ALG1)
    rec["parity_vs_oracle"]["fast_random"] = parity_errors(job.outputs(), ref_r, deq)
    rec["parity_vs_oracle"]["tolerance"] = TOLERANCE + "; from the random start the parity tests " \
        "hold bins the exact EM amplifies rounding-level perturbations on to a conditioning-scaled bound"
    rec["eigensolver_modes"] = mode_records(job, deq, v0, S0, L,
                                            {"mask": (v0d, S0d, ref), "random": (v0r_d, S0r_d, ref_r)}, 3)
    job.free()
    return rec


# ----------------------------------------------------------------------------- batch
def run_batch(args, fca, torch, dev, peaks, clk):
    """512 mixtures, M in {2,4,6}, N in [200, 6000], F=513, L=50, all in one batch (tuned launch
    shapes, the whole job replayed as one CUDA graph), against the same mixtures run one by one
    through the one-mixture entry points, and the conventional form of the same batch. Inputs
    (26 GB of mixtures) exceed L2."""
    import numpy as np

    import oracle
    from synth import device as sdev
    p = sdev.make_packed("batch", dev, count=args.batch_count)
    M, F, N, L = p["M"], p["F"], p["N"], p["iters"]
    units = sum(f * n for f, n in zip(F, N)) * L
    b = fca.fca_batch_init(M, F, N, p["y"], p["v0"], p["S0"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fca.fca_batch_tune(b, L)
    tune_s = time.perf_counter() - t0
    shapes = {f"M={m}": dict(zip(("bins", "threads", "smem_bytes"), fca.fca_batch_shape(b, m)))
              for m in sorted(set(M))}
    x1 = torch.empty(b.x_elems, dtype=torch.complex64, device=dev)
    x2 = torch.empty_like(x1)
    ll = torch.empty(b.count * L, dtype=torch.float64, device=dev)
    v = torch.empty(b.v_elems, dtype=torch.float32, device=dev)
    steps = max(3, args.steps // 2)

    def job(form=fca.FCA_FORM_FAST, graph=True):
        fca.fca_batch_run(b, form, L, x1, x2, loglik=ll, v=v, use_graph=graph)

    for _ in range(2):
        job()
    if fca.fca_batch_sync_status(b) != 0:
        raise RuntimeError("device status error in the batch warm-up")
    l0 = fca.fca_kernel_launches()
    t0 = time.time()
    ms, _ = timed_events(job, steps)
    clk.mark("batch", t0, time.time())
    launches = fca.fca_kernel_launches() - l0
    if fca.fca_batch_sync_status(b) != 0:
        raise RuntimeError("device status error in the batch timed region")
    ms_nograph, _ = timed_events(lambda: job(graph=False), max(2, steps // 2))
    # Errors against the oracle on sampled bins of sampled mixtures (v, mu, S, per-bin LL), and
    # the oracle's time on them (the CPU baseline, per bin-iteration, extrapolated).
    job()
    torch.cuda.synchronize()
    sample_mix, sample_f = (0, 97, 211, 305, 406, 511), np.array([0, 131, 256, 512])
    errs, cpu_s, cpu_units = {}, 0.0, 0
    for k in sample_mix:
        if k >= b.count:
            continue
        m, f, n = b.M[k], b.F[k], b.N[k]
        xo, vo, so = int(b.x_off[k]), int(b.v_off[k]), int(b.S_off[k])
        fs = sample_f[sample_f < f]
        y = p["y"][xo:xo + f * n * m].view(f, n, m)[fs].cpu().numpy()
        v0 = p["v0"][vo:vo + 2 * f * n].view(2, f, n)[:, fs].cpu().numpy()
        S0 = p["S0"][so:so + 2 * f * m * m].view(2, f, m, m)[:, fs].cpu().numpy()
        t0 = time.perf_counter()
        r = oracle.em("fast", y, v0, S0, L)
        cpu_s += time.perf_counter() - t0
        cpu_units += len(fs) * n * L
        S, llf = fca.fca_batch_get_params(b, k, want_llf=True, iters=L)
        got = {"mu1": x1[xo:xo + f * n * m].view(f, n, m)[fs].cpu().numpy(),
               "mu2": x2[xo:xo + f * n * m].view(f, n, m)[fs].cpu().numpy(),
               "v": v[vo:vo + 2 * f * n].view(2, f, n)[:, fs].cpu().numpy().astype(np.float64),
               "S": S.numpy()[:, fs], "llf": llf.numpy()[:, fs]}
        errs[f"mixture {k} (M={m}, N={n})"] = parity_errors(got, r, y, np.arange(len(fs)))
    job(fca.FCA_FORM_CONVENTIONAL)
    t0 = time.time()
    ms_conv, _ = timed_events(lambda: job(fca.FCA_FORM_CONVENTIONAL), max(2, steps // 3))
    clk.mark("batch", t0, time.time())
    if fca.fca_batch_sync_status(b) != 0:
        raise RuntimeError("device status error in the conventional batch")
    # Per-mixture launches: one state per mixture, each job loaded and run on its own.
    y, v0, S0 = p["y"], p["v0"], p["S0"]
    (xo, vo, so), _ = fca.batch_offsets(M, F, N)
    views = []
    for k, (m, f, n) in enumerate(zip(M, F, N)):
        views.append((y[xo[k]:xo[k] + f * n * m].view(f, n, m), v0[vo[k]:vo[k] + 2 * f * n].view(2, f, n),
                      S0[so[k]:so[k] + 2 * f * m * m].view(2, f, m, m),
                      x1[xo[k]:xo[k] + f * n * m].view(f, n, m), x2[xo[k]:xo[k] + f * n * m].view(f, n, m),
                      ll[k * L:(k + 1) * L]))
    states = [fca.fca_init(yk, vk, sk) for yk, vk, sk, *_ in views]

    def per_mixture():
        for st, (yk, vk, sk, x1k, x2k, llk) in zip(states, views):
            fca.fca_load(st, yk, vk, sk)
            fca.fca_em_fast(st, L, llk)
            fca.fca_separate(st, x1k, x2k, fca.FCA_SEP_ALG1)

    per_mixture()
    ms_pm, _ = timed_events(per_mixture, max(2, steps // 3))
    for st in states:
        fca.fca_free(st)
    fca.fca_batch_free(b)
    t = statistics.mean(ms) / 1e3
    Mbar = sum(m * f * n for m, f, n in zip(M, F, N)) / sum(f * n for f, n in zip(F, N))
    bpi = sum(bytes_per_bin_iter(m) * f * n for m, f, n in zip(M, F, N)) / sum(f * n for f, n in zip(F, N))
    flops = sum(fast_flops_per_bin_iter(m) * f * n for m, f, n in zip(M, F, N)) * L
    flops_c = sum(conv_flops_per_bin_iter(m) * f * n for m, f, n in zip(M, F, N)) * L
    del p, x1, x2, ll, v, views
    torch.cuda.empty_cache()
    return {
        "workload": f"batch: {len(M)} mixtures, M uniform in {{2,4,6}}, N uniform in [200,6000], F=513, "
                    "L=50, complex64, seeded (delta=0.05, sigma=1.5), mask-based initialisation",
        "value": units / t, "unit": UNIT, "ms_per_step": 1e3 * t, "steps": steps,
        "bin_iters_per_step": units, "mixtures_by_M": {f"M={m}": M.count(m) for m in sorted(set(M))},
        "l2": "inputs (26 GB) larger than L2", "eigensolver": "refined (library default)",
        "step": "whole batch job as one CUDA graph launch: initial GEVD + L iterations with "
                "per-mixture log-likelihood + posterior means",
        "tuned_shapes": shapes, "tune_s": tune_s,
        "roofline": {"bound": "hbm", "achieved": bpi * units / t / 1e9, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": bpi * units / t / 1e9 / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "whole job (all groups' kernels; job time)", "bytes_per_bin_iter": bpi,
                     "mean_M": Mbar, "peak_source": peaks["hbm_src"],
                     "alu": {"achieved": flops / t / 1e12, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                             "frac": flops / t / 1e12 / peaks["fp32_tflops"]}},
        "graph_off": {"value": units / (statistics.mean(ms_nograph) / 1e3),
                      "ms_per_step": statistics.mean(ms_nograph)},
        "per_mixture_launches": {"value": units / (statistics.mean(ms_pm) / 1e3),
                                 "ms_per_step": statistics.mean(ms_pm),
                                 "batch_speedup": statistics.mean(ms_pm) / statistics.mean(ms)},
        "conventional": {"value": units / (statistics.mean(ms_conv) / 1e3),
                         "ms_per_step": statistics.mean(ms_conv),
                         "fast_speedup": statistics.mean(ms_conv) / statistics.mean(ms),
                         "alu": {"achieved": flops_c / (statistics.mean(ms_conv) / 1e3) / 1e12,
                                 "peak": peaks["fp32_tflops"], "unit": "TFLOP/s"}},
        "parity_vs_oracle": dict(errs, tolerance=TOLERANCE,
                                 sample="bins 0, 131, 256, 512 of mixtures 0, 97, 211, 305, 406, 511"),
        "cpu_baseline": {"value": cpu_units / cpu_s if cpu_s else None, "unit": UNIT, "kind": "oracle",
                         "cores": oracle.threads(),
                         "sample": f"FastFCA form on the sampled bins above ({cpu_s:.1f} s); per "
                                   "bin-iteration, extrapolated to the whole batch"},
        "gpu_launches": launches,
    }


# ------------------------------------------------------------------------------ serve
def run_serve(args, fca, torch, dev, peaks, clk):
    """Requests with M in {2,4,8}, N in [60, 1000], F=513, L=30, Poisson arrivals at 200
    requests/s, host (pinned) inputs and outputs. The server (continuous admission by device
    memory, concurrent streams) against a plain loop that serves one request at a time on one
    state per M; both see the same arrival times. Latency = result on the host minus scheduled
    arrival. A saturated run (every request submitted at once) gives the server's capacity."""
    import numpy as np

    import oracle
    import synth
    from synth import device as sdev
    n_req, n_distinct = args.serve_requests, 100
    c = sdev.MANY["serve"]
    M, F, N, gaps = sdev.shapes("serve", n_req)
    arrivals = np.cumsum(gaps)
    L = c.iters
    pool = []
    for k in range(n_distinct):
        yk, vk, sk = sdev.mixture(M[k], F[k], N[k], c.delta, c.sigma, synth.config_seed("serve", k), dev)
        pool.append(tuple(t.cpu().pin_memory() for t in (yk, vk, sk)) +
                    (torch.empty(yk.shape, dtype=torch.complex64).pin_memory(),
                     torch.empty(yk.shape, dtype=torch.complex64).pin_memory(),
                     torch.empty(L, dtype=torch.float64).pin_memory(),
                     torch.empty((2,) + tuple(yk.shape[:2]), dtype=torch.float32).pin_memory()))
    units = [F[k % n_distinct] * N[k % n_distinct] * L for k in range(n_req)]
    Mk = [M[k % n_distinct] for k in range(n_req)]
    budget = 8 << 30
    srv = fca.fca_server_create(budget, max_inflight=16)

    def serve(times, mark=None):
        launches0 = fca.fca_kernel_launches()
        t0 = time.monotonic() + 0.05
        w0 = time.time() + 0.05
        tickets = []
        for k in range(len(times)):
            target = t0 + times[k]
            while True:
                d = target - time.monotonic()
                if d <= 0:
                    break
                time.sleep(d if d > 2e-3 else 0)
            y, v0, S0, x1, x2, ll, vv = pool[k % n_distinct]
            tickets.append(fca.fca_server_submit(srv, y, v0, S0, x1, x2, L, loglik=ll, v=vv))
        infos = [fca.fca_server_wait(srv, t) for t in tickets]
        if any(rc != 0 for rc, _ in infos):
            raise RuntimeError("a request failed")
        lat = [inf["t_done"] - (t0 + times[k]) for k, (_, inf) in enumerate(infos)]
        end = max(inf["t_done"] for _, inf in infos)
        if mark:
            clk.mark(mark, w0, w0 + (end - t0))
        return lat, end - t0, fca.fca_kernel_launches() - launches0

    serve(arrivals[:50] - arrivals[0])  # warm-up
    lat, wall, launches = serve(arrivals, mark="serve")
    st = fca.fca_server_stats(srv)
    lat_sat, wall_sat, _ = serve(np.zeros(n_req), mark="serve")
    fca.fca_server_destroy(srv)
    # Plain per-request serving: one request at a time, in arrival order.
    cap = {}
    for k in range(n_distinct):
        cap[M[k]] = max(cap.get(M[k], 0), N[k])
    states = {}
    for m, n in cap.items():
        k = next(k for k in range(n_distinct) if M[k] == m and N[k] == n)
        states[m] = fca.fca_init(*pool[k][:3])
    stream = torch.cuda.Stream()
    xd = {m: (torch.empty((513, cap[m], m), dtype=torch.complex64, device=dev),
              torch.empty((513, cap[m], m), dtype=torch.complex64, device=dev)) for m in states}
    lld = torch.empty(L, dtype=torch.float64, device=dev)

    def plain(times):
        t0 = time.monotonic() + 0.05
        out = []
        for k in range(len(times)):
            target = t0 + times[k]
            while time.monotonic() < target:
                pass
            y, v0, S0, x1, x2, ll, _ = pool[k % n_distinct]
            m, n = y.shape[2], y.shape[1]
            with torch.cuda.stream(stream):
                st_m = states[m]
                fca.fca_load(st_m, y, v0, S0, stream=stream)
                fca.fca_em_fast(st_m, L, lld, stream=stream)
                a = xd[m][0].view(-1)[:513 * n * m].view(513, n, m)
                b = xd[m][1].view(-1)[:513 * n * m].view(513, n, m)
                fca.fca_separate(st_m, a, b, fca.FCA_SEP_ALG1, stream=stream)
                x1.copy_(a, non_blocking=True)
                x2.copy_(b, non_blocking=True)
                ll.copy_(lld, non_blocking=True)
            stream.synchronize()
            out.append(time.monotonic() - target)
        return out

    plain(arrivals[:50] - arrivals[0])
    lat_plain = plain(arrivals)
    for s in states.values():
        fca.fca_free(s)
    pct = lambda a, q: float(np.percentile(np.asarray(a) * 1e3, q))  # noqa: E731
    total = float(sum(units))
    # Errors of one served request against the oracle, and the oracle serving five requests.
    y, v0, S0, x1, x2, ll, vv = pool[3]
    ref = oracle.em("fast", y.numpy().astype(np.complex128), v0.numpy(), S0.numpy(), L)
    got = {"mu1": x1.numpy(), "mu2": x2.numpy(), "v": vv.numpy().astype(np.float64),
           "llf": None}
    err = parity_errors(got, ref, y.numpy())
    err["ll"] = [float(np.max(np.abs(ll.numpy() - ref["ll"].sum(axis=1)) / np.abs(ref["ll"].sum(axis=1))))] * 2
    lat_o = []
    for k in range(5):
        y, v0, S0 = pool[k][:3]
        t0 = time.perf_counter()
        oracle.em("fast", y.numpy().astype(np.complex128), v0.numpy(), S0.numpy(), L, want_mu=True)
        lat_o.append(time.perf_counter() - t0)
    return {
        "workload": f"serving: {n_req} requests, Poisson arrivals at {c.rate:.0f}/s, M uniform in {{2,4,8}}, "
                    "N uniform in [60,1000], F=513, L=30, host inputs/outputs "
                    f"({n_distinct} distinct mixtures, cycled), mask-based initialisation",
        "value": total / wall, "unit": UNIT, "requests_per_s": n_req / wall,
        "server": {"device_bytes": budget, "max_inflight": 16},
        "requests_by_M": {f"M={m}": Mk.count(m) for m in sorted(set(Mk))},
        "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": pct(lat, 100)},
        "server_stats": {k: st[k] for k in ("max_in_flight", "bytes_peak", "completed")},
        "saturated": {"value": total / wall_sat, "requests_per_s": n_req / wall_sat,
                      "latency_ms": {"p50": pct(lat_sat, 50), "p99": pct(lat_sat, 99)}},
        "plain_per_request": {"latency_ms": {"p50": pct(lat_plain, 50), "p99": pct(lat_plain, 99),
                                             "max": pct(lat_plain, 100)}},
        "parity_vs_oracle": {"request 3": err, "tolerance": TOLERANCE},
        "cpu_baseline": {"kind": "oracle", "cores": oracle.threads(),
                         "latency_ms": {"p50": pct(lat_o, 50), "max": pct(lat_o, 100)},
                         "value": float(sum(units[k] for k in range(5))) / sum(lat_o), "unit": UNIT,
                         "sample": "requests 0-4 served one after another, FastFCA form "
                                   f"(M={[M[k] for k in range(5)]}, N={[N[k] for k in range(5)]})"},
        "gpu_launches": launches,
    }


# -------------------------------------------------------------------------- reference
def run_reference(args):
    """The reference arm: the FP64 oracle timed on the host cores, one bounded sample per step."""
    import numpy as np

    import synth
    world, rank, _ = dist_env()
    if rank != 0:
        return
    c, mix, v0, S0 = synth.make_config("mid")
    import oracle
    oracle.build()
    y = mix["y"].astype(np.complex128)
    for _ in range(args.warmup):
        cpu_oracle_rate(y, v0, S0, c.iters, c.F)
    units, secs = 0.0, []
    for _ in range(args.steps):
        r, dt, threads, sample, _, _ = cpu_oracle_rate(y, v0, S0, c.iters, c.F)
        units += r * dt
        secs.append(dt)
    value = units / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"mid: M={c.M} F={c.F} N={c.N} L={c.iters}, 2 sources, complex64, seeded "
                               f"mixture per rank (delta={c.delta}, sigma={c.sigma}), mask-based "
                               "initialisation",
                   "form": "FastFCA (FP64 oracle, host cores)",
                   "step": "L iterations with log-likelihood + posterior means, every bin"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["all", "mid", "batch", "serve", "precision"], default="all")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-count", type=int, default=None,
                    help="batch workload: the first K of its 512 mixtures (profiling runs)")
    ap.add_argument("--serve-requests", type=int, default=1000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1805_06572_gb300 as pkg
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    from paper_1805_06572_gb300 import fca
    dev = torch.device("cuda", local)
    fp32, fp64 = fca.fca_measure_peaks()
    hbm, hbm_src = hbm_peak()
    peaks = {"hbm_gbs": hbm, "hbm_src": hbm_src, "fp32_tflops": fp32, "fp64_tflops": fp64}
    clk = ClockSampler(local).start()
    subs = {}
    try:
        if args.workload in ("all", "mid"):
            line = run_mid(args, fca, torch, dev, peaks, clk, world, rank)
        else:
            line = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                    "warmup": args.warmup, "higher_is_better": True, "data": "synthetic"}
        torch.cuda.empty_cache()
        if world == 1:
            for name, fn in (("precision", run_precision), ("batch", run_batch), ("serve", run_serve)):
                if args.workload in ("all", name):
                    subs[name] = fn(args, fca, torch, dev, peaks, clk)
                    torch.cuda.empty_cache()
    finally:
        clk.stop()
    line["clocks"] = clk.summary()
    line["clocks_headline"] = clk.summary({"mid"})
    line["measured_peaks"] = {"fp32_tflops": fp32, "fp64_tflops": fp64,
                              "note": "FMA throughput measured in this run (fca_measure_peaks)",
                              "hbm_gbs": hbm, "hbm_source": hbm_src}
    if subs:
        line["sub"] = subs
        if args.workload != "all" and args.workload in subs:
            rec = subs[args.workload]
            line.update({k: rec[k] for k in ("value", "ms_per_step") if k in rec})
            line["config"] = {"workload": rec["workload"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
