"""Benchmark: TF-bin EM iterations per second of FastFCA (and conventional FCA) on GB300.

One step = one whole EM job of the hot path on one mixture: load the mixture and initial
parameters into the library state (device-resident inputs), the initial generalised
eigendecomposition, L FastFCA iterations with the per-iteration log-likelihood, and the
posterior-mean outputs (Algorithm 1). Workload: M=4 channels, F=513 bins, N=1000 frames,
L=50 iterations, complex64, synthetic seeded mixture. bin-iters per step = F * N * L.

Under torchrun each rank runs its own mixture (weak scaling: frequencies and mixtures are
independent, there is no exchange on the data path); value = all ranks' bin-iters / the
slowest rank's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference of this project) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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
WORKLOAD = "mid"
# FP32 peak derived from the unit counts and the maximum SM clock: 152 SMs x 128 FP32 lanes
# x 2 flop per FMA x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def fast_flops_per_bin_iter(M: int) -> int:
    """Algorithmic FP32 flops of one FastFCA time-frequency point per iteration (counted from
    the equations: P^H y 8M^2; d, 1/d, |yt|^2, the mut coefficients 9M; the two v updates
    9M+2; two rank-1-plus-diagonal Gram updates 2(5M^2+3M+1); log-likelihood terms 3M)."""
    return 18 * M * M + 27 * M + 4


def conv_flops_per_bin_iter(M: int) -> int:
    """Algorithmic FP32 flops of one conventional time-frequency point per iteration: Rx
    4M^2; Cholesky 4M^3/3; two triangular solves for u 8M^2; mu_1, mu_2 16M^2; L^-1 S_1 and
    L^-1 S_2 8M^3; C = v1 v2 (L^-1 S1)^H (L^-1 S2), upper triangle 4M^3; two v updates 16M^2;
    two Gram updates 2(5M^2+3M+1); log-likelihood terms 3M."""
    return round(4 * M**3 / 3 + 8 * M**3 + 4 * M**3) + 4 * M * M + 8 * M * M + 16 * M * M \
        + 16 * M * M + 2 * (5 * M * M + 3 * M + 1) + 3 * M


def source_sha() -> str:
    h = hashlib.sha256()
    for f in ("fca_fast.cuh", "fca_dev.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1805_06572_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def profiled_traffic(name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source; else None."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("source_sha") != source_sha():
        return None
    try:
        return float(kv["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, p in zip(names, parts[3:7]):
                if p.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_rate(mix, v0, S0, iters, n_bins, form="fast", min_seconds=0.0, nthreads=0):
    """Time the FP64 oracle (as it stands) on a bounded sample: n_bins frequencies spread over
    the band, all frames, all iterations, repeated until at least min_seconds of work, on
    nthreads host threads (0: all cores). Returns (bin-iters/s, seconds, threads, sample)."""
    import numpy as np

    import oracle
    F = mix["y"].shape[0]
    fs = np.unique(np.linspace(0, F - 1, n_bins).round().astype(int))
    y = mix["y"][fs].astype(np.complex128)
    reps, dt = 0, 0.0
    while reps == 0 or dt < min_seconds:
        t0 = time.perf_counter()
        res = oracle.em(form, y, v0[:, fs], S0[:, fs], iters, want_mu=True, nthreads=nthreads)
        dt += time.perf_counter() - t0
        reps += 1
    units = reps * len(fs) * y.shape[1] * iters
    cpu_oracle_rate.last = (fs, res)
    return units / dt, dt, nthreads or oracle.threads(), \
        f"{reps} x ({len(fs)} of {F} bins x N={y.shape[1]} x L={iters})"


def parity_errors(gpu, ref, y):
    """Errors of GPU outputs against the oracle (the parity tests' metrics): per entry
    |v - v*| / v*, ||mu - mu*|| / ||y|| per time-frequency point, and the largest relative
    log-likelihood error over the iterations. Returns {name: [median, max]}."""
    import numpy as np
    ev = np.abs(gpu["v"] - ref["v"]) / ref["v"]
    yn = np.linalg.norm(y, axis=2)
    yn = np.where(yn > 0, yn, 1.0)
    emu = np.stack([np.linalg.norm(gpu["mu1"] - ref["mu1"], axis=2) / yn,
                    np.linalg.norm(gpu["mu2"] - ref["mu2"], axis=2) / yn])
    llr = ref["ll"].sum(axis=1)
    ell = np.abs(gpu["ll"] - llr) / np.abs(llr)
    return {"v": [float(np.median(ev)), float(ev.max())],
            "mu": [float(np.median(emu)), float(emu.max())],
            "ll": [float(np.median(ell)), float(ell.max())]}


def hbm_model(M, value):
    """Streaming byte model: a TF-bin-iteration reads y (8M bytes) and reads and writes v
    (16 bytes) if nothing stays on chip. GB/s that the measured rate implies under it, and its
    fraction of the measured HBM copy bandwidth."""
    peak, src = 6800.0, "fallback"
    try:
        peak, src = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        pass
    gbs = (8 * M + 16) * value / 1e9
    return {"bytes_per_bin_iter": 8 * M + 16, "model_gbs": gbs, "peak_gbs": peak, "peak": src,
            "frac": gbs / peak}


def mid_workload(c) -> str:
    """The headline workload's description, shared by both arms."""
    return (f"M={c.M} F={c.F} N={c.N} L={c.iters}, 2 sources, complex64, seeded mixture per rank "
            f"(delta={c.delta}, sigma={c.sigma})")


def run_reference(args):
    """The reference arm: the FP64 oracle timed on the host cores, one bounded sample per step."""
    import synth
    world, rank, _ = dist_env()
    if rank != 0:
        return
    c, mix, v0, S0 = synth.make_config(WORKLOAD)
    import oracle
    oracle.build()
    n_bins = c.F  # the whole workload per step: about a second on 16 cores
    for _ in range(args.warmup):
        cpu_oracle_rate(mix, v0, S0, c.iters, n_bins)
    units, secs = 0.0, []
    for _ in range(args.steps):
        r, dt, threads, sample = cpu_oracle_rate(mix, v0, S0, c.iters, n_bins)
        units += r * dt
        secs.append(dt)
    value = units / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": mid_workload(c), "form": "FastFCA (FP64 oracle, host cores)",
                   "step": "L iterations with log-likelihood + posterior means, every bin"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Many-mixture workload: 512 mixtures, M in {2,4,6}, N in [200, 6000], F=513, L=50, all
    in one batch (tuned launch shapes, the whole job replayed as one CUDA graph), against the
    same mixtures run one by one through the one-mixture entry points (per-mixture launches),
    and the conventional form of the same batch. Inputs (26 GB of mixtures) exceed L2."""
    import torch

    import paper_1805_06572_gb300 as pkg
    from synth import device as sdev

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    pkg.build()
    from paper_1805_06572_gb300 import fca

    dev = torch.device("cuda", local)
    p = sdev.make_packed("batch", dev, count=args.batch_count)
    M, F, N, L = p["M"], p["F"], p["N"], p["iters"]
    units = sum(f * n for f, n in zip(F, N)) * L
    flops = sum(fast_flops_per_bin_iter(m) * f * n for m, f, n in zip(M, F, N)) * L
    flops_c = sum(conv_flops_per_bin_iter(m) * f * n for m, f, n in zip(M, F, N)) * L
    b = fca.fca_batch_init(M, F, N, p["y"], p["v0"], p["S0"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if not args.no_tune:
        fca.fca_batch_tune(b, L)
    tune_s = time.perf_counter() - t0
    shapes = {f"M={m}": dict(zip(("bins", "threads", "smem_bytes"), fca.fca_batch_shape(b, m)))
              for m in sorted(set(M))}
    x1 = torch.empty(b.x_elems, dtype=torch.complex64, device=dev)
    x2 = torch.empty_like(x1)
    ll = torch.empty(b.count * L, dtype=torch.float64, device=dev)

    def timed(fn, steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize()
        l0 = fca.fca_kernel_launches()
        for k in range(steps):
            evs[k][0].record()
            fn()
            evs[k][1].record()
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in evs], fca.fca_kernel_launches() - l0

    def job(form=fca.FCA_FORM_FAST, graph=True):
        fca.fca_batch_run(b, form, L, x1, x2, loglik=ll, use_graph=graph)

    for _ in range(args.warmup):
        job()
    if fca.fca_batch_sync_status(b) != 0:
        raise RuntimeError("device status error in the batch warm-up")
    with ClockSampler(local) as clk:
        ms, launches = timed(job, args.steps)
    clocks = clk.summary()
    if fca.fca_batch_sync_status(b) != 0:
        raise RuntimeError("device status error in the batch timed region")
    ms_nograph, _ = timed(lambda: job(graph=False), max(2, args.steps // 2))
    job(fca.FCA_FORM_CONVENTIONAL)
    ms_conv, _ = timed(lambda: job(fca.FCA_FORM_CONVENTIONAL), max(2, args.steps // 3))
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
    ms_pm, _ = timed(per_mixture, max(2, args.steps // 3))
    for st in states:
        fca.fca_free(st)
    t = statistics.mean(ms) / 1e3
    value = units / t
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch: {len(M)} mixtures, M uniform in {{2,4,6}}, N uniform in "
                               "[200,6000], F=513, L=50, complex64, seeded (delta=0.05, sigma=1.5)",
                   "form": "FastFCA", "mixtures_by_M": {f"M={m}": M.count(m) for m in sorted(set(M))},
                   "bin_iters_per_step": units, "l2": "inputs (26 GB) larger than L2",
                   "step": "whole batch job as one CUDA graph launch: initial GEVD + L iterations "
                           "with per-mixture log-likelihood + posterior means",
                   "tuned_shapes": shapes, "tune_s": tune_s},
        "hbm_streaming_model": hbm_model(sum(m * f * n for m, f, n in zip(M, F, N)) /
                                         sum(f * n for f, n in zip(F, N)), units / t),
        "roofline": {"bound": "alu", "achieved": flops / t / 1e12, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": flops / t / 1e12 / FP32_PEAK_TFLOPS,
                     "traffic": None, "kernel": "fast_em_kernel<M,c64,tuned> (all groups, job time)",
                     "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
        "graph_off": {"value": units / (statistics.mean(ms_nograph) / 1e3),
                      "ms_per_step": statistics.mean(ms_nograph)},
        "per_mixture_launches": {"value": units / (statistics.mean(ms_pm) / 1e3),
                                 "ms_per_step": statistics.mean(ms_pm),
                                 "batch_speedup": statistics.mean(ms_pm) / statistics.mean(ms)},
        "conventional": {"value": units / (statistics.mean(ms_conv) / 1e3),
                         "ms_per_step": statistics.mean(ms_conv),
                         "fast_speedup": statistics.mean(ms_conv) / statistics.mean(ms),
                         "roofline": {"bound": "alu", "achieved": flops_c / (statistics.mean(ms_conv) / 1e3) / 1e12,
                                      "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s"}},
        "gpu_launches": launches, "clocks": clocks,
    }
    fca.fca_batch_free(b)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving workload: requests with M in {2,4,8}, N in [60, 1000], F=513, L=30, Poisson
    arrivals at 200 requests/s, host (pinned) inputs and outputs. The server (continuous
    admission by device memory, concurrent streams) against a plain loop that serves one
    request at a time on one state per M; both see the same arrival times. Latency = result
    on the host minus scheduled arrival. A saturated run (every request submitted at once)
    gives the server's capacity."""
    import numpy as np
    import torch

    import paper_1805_06572_gb300 as pkg
    from synth import device as sdev

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    pkg.build()
    from paper_1805_06572_gb300 import fca

    dev = torch.device("cuda", local)
    n_req = max(200, args.steps * 100)
    n_distinct = 100
    c = sdev.MANY["serve"]
    M, F, N, gaps = sdev.shapes("serve", n_req)
    arrivals = np.cumsum(gaps)
    L = c.iters
    # Distinct requests (cycled): pinned host inputs and outputs.
    pool = []
    for k in range(n_distinct):
        yk, vk, sk = sdev.mixture(M[k], F[k], N[k], c.delta, c.sigma, synth_seed("serve", k), dev)
        pool.append(tuple(t.cpu().pin_memory() for t in (yk, vk, sk)) +
                    (torch.empty(yk.shape, dtype=torch.complex64).pin_memory(),
                     torch.empty(yk.shape, dtype=torch.complex64).pin_memory(),
                     torch.empty(L, dtype=torch.float64).pin_memory()))
    units = [F[k % n_distinct] * N[k % n_distinct] * L for k in range(n_req)]
    Mk = [M[k % n_distinct] for k in range(n_req)]
    budget = 8 << 30
    srv = fca.fca_server_create(budget, max_inflight=16)

    def serve(times):
        launches0 = fca.fca_kernel_launches()
        t0 = time.monotonic() + 0.05
        tickets = []
        for k in range(len(times)):
            target = t0 + times[k]
            while True:
                d = target - time.monotonic()
                if d <= 0:
                    break
                time.sleep(d if d > 2e-3 else 0)
            y, v0, S0, x1, x2, ll = pool[k % n_distinct]
            tickets.append(fca.fca_server_submit(srv, y, v0, S0, x1, x2, L, loglik=ll))
        infos = [fca.fca_server_wait(srv, t) for t in tickets]
        if any(rc != 0 for rc, _ in infos):
            raise RuntimeError("a request failed")
        lat = [inf["t_done"] - (t0 + times[k]) for k, (_, inf) in enumerate(infos)]
        end = max(inf["t_done"] for _, inf in infos)
        return lat, end - t0, fca.fca_kernel_launches() - launches0

    serve(arrivals[:50] - arrivals[0])  # warm-up
    with ClockSampler(local) as clk:
        lat, wall, launches = serve(arrivals)
    clocks = clk.summary()
    st = fca.fca_server_stats(srv)
    lat_sat, wall_sat, _ = serve(np.zeros(n_req))
    fca.fca_server_destroy(srv)

    # Plain per-request serving: one request at a time, in arrival order.
    cap = {}
    for k in range(n_distinct):
        cap[M[k]] = max(cap.get(M[k], 0), N[k])
    states = {}  # one state per M, sized for its longest request (fca_load takes shorter ones)
    for m, n in cap.items():
        k = next(k for k in range(n_distinct) if M[k] == m and N[k] == n)
        y, v0, S0 = pool[k][:3]
        states[m] = fca.fca_init(y, v0, S0)
    stream = torch.cuda.Stream()
    xd = {m: (torch.empty((513, cap[m], m), dtype=torch.complex64, device=dev),
              torch.empty((513, cap[m], m), dtype=torch.complex64, device=dev)) for m in states}
    lld = torch.empty(L, dtype=torch.float64, device=dev)

    def plain(times):
        t0 = time.monotonic() + 0.05
        lat = []
        for k in range(len(times)):
            target = t0 + times[k]
            while time.monotonic() < target:
                pass
            y, v0, S0, x1, x2, ll = pool[k % n_distinct]
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
            lat.append(time.monotonic() - target)
        return lat

    plain(arrivals[:50] - arrivals[0])
    lat_plain = plain(arrivals)
    pct = lambda a, q: float(np.percentile(np.asarray(a) * 1e3, q))  # noqa: E731
    total = float(sum(units))
    line = {
        "metric": METRIC, "value": total / wall, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / n_req, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serving: {n_req} requests, Poisson arrivals at {c.rate:.0f}/s, "
                               "M uniform in {2,4,8}, N uniform in [60,1000], F=513, L=30, "
                               f"host inputs/outputs ({n_distinct} distinct mixtures, cycled)",
                   "form": "FastFCA", "server": {"device_bytes": budget, "max_inflight": 16},
                   "requests_by_M": {f"M={m}": Mk.count(m) for m in sorted(set(Mk))}},
        "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": pct(lat, 100)},
        "requests_per_s": n_req / wall,
        "server_stats": {k: st[k] for k in ("max_in_flight", "bytes_peak", "completed")},
        "saturated": {"value": total / wall_sat, "requests_per_s": n_req / wall_sat,
                      "latency_ms": {"p50": pct(lat_sat, 50), "p99": pct(lat_sat, 99)}},
        "plain_per_request": {"latency_ms": {"p50": pct(lat_plain, 50), "p99": pct(lat_plain, 99),
                                             "max": pct(lat_plain, 100)}},
        "gpu_launches": launches, "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        # The FP64 oracle serving the first few distinct requests one after another (host cores).
        import oracle
        lat_o = []
        for k in range(5):
            y, v0, S0 = pool[k][:3]
            t0 = time.perf_counter()
            oracle.em("fast", y.numpy().astype(np.complex128), v0.numpy(), S0.numpy(), L, want_mu=True)
            lat_o.append(time.perf_counter() - t0)
        line["cpu_baseline"] = {
            "kind": "oracle", "cores": oracle.threads(),
            "latency_ms": {"p50": pct(lat_o, 50), "max": pct(lat_o, 100)},
            "value": float(sum(units[k] for k in range(5))) / sum(lat_o), "unit": UNIT,
            "sample": "requests 0-4 served one after another, FastFCA form "
                      f"(M={[M[k] for k in range(5)]}, N={[N[k] for k in range(5)]})"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_precision(args):
    """Precision workload: M=8, F=1025, N=4000, L=100; the mixture stored as FP16 pairs with a
    per-frequency power scale, FP32 bin arithmetic, FP64 Gram/log-likelihood merges and basis.
    Same step as the mid workload (load, initial GEVD, L iterations with LL, outputs)."""
    import torch

    import synth
    import paper_1805_06572_gb300 as pkg

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    pkg.build()
    from paper_1805_06572_gb300 import fca

    dev = torch.device("cuda", local)
    c, mix, v0, S0 = synth.make_config("precision")
    y16, g, _ = synth.quantize_f16(mix["y"])
    F, N, M, L = c.F, c.N, c.M, c.iters
    units = F * N * L
    yd, gd = torch.from_numpy(y16).to(dev), torch.from_numpy(g).to(dev)
    v0d, S0d = torch.from_numpy(v0).to(dev), torch.from_numpy(S0).to(dev)
    st = fca.fca_init(yd, v0d, S0d, y_scale=gd)
    x1 = torch.empty((F, N, M), dtype=torch.complex64, device=dev)
    x2 = torch.empty_like(x1)
    ll = torch.empty(L, dtype=torch.float64, device=dev)

    def step(form):
        fca.fca_load(st, yd, v0d, S0d, y_scale=gd)
        (fca.fca_em_fast if form == "fast" else fca.fca_em_conventional)(st, L, ll)
        fca.fca_separate(st, x1, x2, fca.FCA_SEP_ALG1)

    def timed(form, steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        kms = []
        torch.cuda.synchronize()
        l0 = fca.fca_kernel_launches()
        for k in range(steps):
            evs[k][0].record()
            step(form)
            evs[k][1].record()
            kms.append(fca.fca_last_em_kernel_ms(st))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs], kms, fca.fca_kernel_launches() - l0

    for _ in range(args.warmup):
        step("fast")
    with ClockSampler(local) as clk:
        ms, kms, launches = timed("fast", args.steps)
    clocks = clk.summary()
    step("conventional")
    ms_c, kms_c, _ = timed("conventional", max(2, args.steps // 3))
    if fca.fca_sync_status(st) != 0:
        raise RuntimeError("device status error")
    t, tc = statistics.mean(ms) / 1e3, statistics.mean(ms_c) / 1e3
    kf, kc = statistics.mean(kms) / 1e3, statistics.mean(kms_c) / 1e3
    ach = fast_flops_per_bin_iter(M) * units / kf / 1e12
    line = {
        "metric": METRIC, "value": units / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (y stored f16)", "data": "synthetic",
        "config": {"workload": f"precision: M={M} F={F} N={N} L={L}, y as FP16 pairs with a "
                               "per-frequency scale, seeded (delta=0.05, sigma=1.5)",
                   "form": "FastFCA", "l2": "inputs (131 MB FP16 mixture + source powers) larger than L2",
                   "step": "load + initial GEVD + L iterations with log-likelihood + posterior means"},
        "roofline": {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach / FP32_PEAK_TFLOPS, "traffic": None,
                     "kernel": f"fast_em_kernel<{M},f16,128>", "kernel_ms": 1e3 * kf,
                     "flops_per_bin_iter": fast_flops_per_bin_iter(M)},
        "conventional": {"value": units / tc, "unit": UNIT, "ms_per_step": 1e3 * tc,
                         "kernel_ms": 1e3 * kc, "fast_speedup": tc / t},
        "gpu_launches": launches, "clocks": clocks,
    }
    fca.fca_free(st)
    if rank == 0:
        print(json.dumps(line), flush=True)


def synth_seed(name, k):
    import synth
    return synth.config_seed(name, k)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["mid", "batch", "serve", "precision"], default="mid")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-count", type=int, default=None,
                    help="batch workload: the first K of its 512 mixtures (profiling runs)")
    ap.add_argument("--no-tune", action="store_true",
                    help="batch workload: keep the default launch shapes (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "precision":
        return run_precision(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_1805_06572_gb300 as pkg

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    from paper_1805_06572_gb300 import fca
    from paper_1805_06572_gb300.shard import allreduce_max, weak_scaling_value

    dev = torch.device("cuda", local)
    c, mix, v0, S0 = synth.make_config(WORKLOAD, mixture_index=rank)
    F, N, M, L = c.F, c.N, c.M, c.iters
    units = F * N * L
    y_h = torch.from_numpy(mix["y"]).pin_memory()
    v0_h = torch.from_numpy(v0).pin_memory()
    S0_h = torch.from_numpy(S0).pin_memory()
    y_d, v0_d, S0_d = y_h.to(dev), v0_h.to(dev), S0_h.to(dev)
    st = fca.fca_init(y_d, v0_d, S0_d)
    x1 = torch.empty((F, N, M), dtype=torch.complex64, device=dev)
    x2 = torch.empty_like(x1)
    ll = torch.empty(L, dtype=torch.float64, device=dev)
    x1_h = torch.empty((F, N, M), dtype=torch.complex64).pin_memory()
    x2_h = torch.empty_like(x1_h).pin_memory()
    ll_h = torch.empty(L, dtype=torch.float64).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step(form):
        fca.fca_load(st, y_d, v0_d, S0_d)
        (fca.fca_em_fast if form == "fast" else fca.fca_em_conventional)(st, L, ll)
        fca.fca_separate(st, x1, x2, fca.FCA_SEP_ALG1)

    # End to end through the public API as a caller streaming mixtures would run it: two
    # states on two CUDA streams, so one mixture's host<->device copies overlap the other's
    # kernels. Every step copies its inputs from pinned host memory and its outputs (posterior
    # means and log-likelihood) back.
    e2e_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    e2e_states = [st, fca.fca_init(y_d, v0_d, S0_d)]
    e2e_bufs = [(x1, x2, ll, x1_h, x2_h, ll_h)]
    e2e_bufs.append((torch.empty_like(x1), torch.empty_like(x2), torch.empty_like(ll),
                     torch.empty_like(x1_h).pin_memory(), torch.empty_like(x2_h).pin_memory(),
                     torch.empty_like(ll_h).pin_memory()))

    def step_e2e(k):
        s, stk = e2e_streams[k % 2], e2e_states[k % 2]
        a, b, l, ah, bh, lh = e2e_bufs[k % 2]
        with torch.cuda.stream(s):
            fca.fca_load(stk, y_h, v0_h, S0_h, stream=s)
            fca.fca_em_fast(stk, L, l, stream=s)
            fca.fca_separate(stk, a, b, fca.FCA_SEP_ALG1, stream=s)
            ah.copy_(a, non_blocking=True)
            bh.copy_(b, non_blocking=True)
            lh.copy_(l, non_blocking=True)

    def timed_e2e(steps):
        barrier()
        t0 = time.perf_counter()
        for k in range(steps):
            step_e2e(k)
        barrier()
        return time.perf_counter() - t0

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps, form=None):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        kms = []
        barrier()
        launches0 = fca.fca_kernel_launches()
        t0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            evs[k][0].record()
            fn() if form is None else fn(form)
            evs[k][1].record()
            if form is not None:
                kms.append(fca.fca_last_em_kernel_ms(st))
        barrier()
        wall = time.perf_counter() - t0
        launches = fca.fca_kernel_launches() - launches0
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, kms, wall, launches

    def max_over_ranks(x: float) -> float:
        return x if world == 1 else allreduce_max(x, dist, device=dev)

    for _ in range(args.warmup):
        step("fast")
    torch.cuda.synchronize()
    code = fca.fca_sync_status(st)
    if code != 0:
        raise RuntimeError(f"device status {code} during warm-up")

    with ClockSampler(local) as clk:
        ms_fast, k_fast, wall_fast, launches = timed(step, args.steps, "fast")
    clocks = clk.summary()
    if fca.fca_sync_status(st) != 0:
        raise RuntimeError("device status error in the timed region")

    steps_conv = max(3, args.steps // 2)
    for _ in range(3):
        step("conventional")
    ms_conv, k_conv, _, _ = timed(step, steps_conv, "conventional")
    for k in range(4):
        step_e2e(k)
    wall_e2e = timed_e2e(args.steps)
    ms_e2e = [1e3 * wall_e2e / args.steps] * args.steps
    if fca.fca_sync_status(st) != 0 or fca.fca_sync_status(e2e_states[1]) != 0:
        raise RuntimeError("device status error")

    t_fast = max_over_ranks(sum(ms_fast) / 1e3)
    t_conv = max_over_ranks(sum(ms_conv) / 1e3)
    t_e2e = max_over_ranks(sum(ms_e2e) / 1e3)
    value = weak_scaling_value(units * args.steps, world, t_fast)
    conv_value = weak_scaling_value(units * steps_conv, world, t_conv)
    e2e_value = weak_scaling_value(units * args.steps, world, t_e2e)
    kern_fast = statistics.mean(k_fast) / 1e3
    kern_conv = statistics.mean(k_conv) / 1e3
    ach = fast_flops_per_bin_iter(M) * units / kern_fast / 1e12
    ach_c = conv_flops_per_bin_iter(M) * units / kern_conv / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_over_ranks(statistics.mean(ms_fast)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": mid_workload(c),
                   "form": "FastFCA", "l2": "flushed between steps (256 MiB write, outside the "
                   "step events)", "parallelism": f"replicas x{world}",
                   "step": "load + initial GEVD + L iterations with log-likelihood + "
                           "posterior means"},
        "roofline": {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach / FP32_PEAK_TFLOPS,
                     "traffic": profiled_traffic("fast_em_kernel_mid.md"),
                     "kernel": "fast_em_kernel<4,c64,128>", "kernel_ms": 1e3 * kern_fast,
                     "flops_per_bin_iter": fast_flops_per_bin_iter(M),
                     "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
        "conventional": {"value": conv_value, "unit": UNIT, "ms_per_step": statistics.mean(ms_conv),
                         "steps": steps_conv, "kernel_ms": 1e3 * kern_conv,
                         "fast_speedup": value / conv_value,
                         "roofline": {"bound": "alu", "achieved": ach_c, "peak": FP32_PEAK_TFLOPS,
                                      "unit": "TFLOP/s", "frac": ach_c / FP32_PEAK_TFLOPS,
                                      "flops_per_bin_iter": conv_flops_per_bin_iter(M)}},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": y_h.numel() * 8 + v0_h.numel() * 8 + S0_h.numel() * 16,
                "d2h_bytes_per_step": x1_h.numel() * 8 * 2 + ll_h.numel() * 8,
                "ms_per_step": statistics.mean(ms_e2e),
                "timing": "host wall clock around all steps, synchronised on both sides; "
                          "two states on two streams (copies of one step overlap another's kernels)"},
        "hbm_streaming_model": dict(hbm_model(M, value), note="y and v stay on chip; ncu DRAM "
                                                              "traffic per launch is in roofline.traffic"),
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s_timed_region": wall_fast,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, dt, threads, sample = cpu_oracle_rate(mix, v0, S0, L, F, min_seconds=10.0)
        _, ref_fast = cpu_oracle_rate.last
        rate_c, dt_c, _, sample_c = cpu_oracle_rate(mix, v0, S0, L, F, form="conventional",
                                                    min_seconds=10.0)
        _, ref_conv = cpu_oracle_rate.last
        rate_1, dt_1, _, sample_1 = cpu_oracle_rate(mix, v0, S0, L, 32, min_seconds=3.0, nthreads=1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"FastFCA form, {sample} ({dt:.1f} s)",
                                "conventional_value": rate_c,
                                "conventional_sample": f"{sample_c} ({dt_c:.1f} s)",
                                "one_thread": {"value": rate_1, "cores": 1,
                                               "sample": f"FastFCA form, {sample_1} ({dt_1:.1f} s)"}}
        # The GPU outputs of one step of each form against those oracle runs (same inputs).
        import numpy as np
        parity = {}
        for form, ref in (("fast", ref_fast), ("conventional", ref_conv)):
            step(form)
            v = torch.empty((2, F, N), dtype=torch.float32, device=dev)
            fca.fca_get_params(st, v=v)
            got = {"v": v.cpu().numpy().astype(np.float64), "mu1": x1.cpu().numpy(),
                   "mu2": x2.cpu().numpy(), "ll": ll.cpu().numpy()}
            parity[form] = parity_errors(got, ref, mix["y"].astype(np.complex128))
        line["parity_vs_oracle"] = dict(parity, tolerance="median <= 1e-4, max <= 1e-3 (v, mu); "
                                                          "ll <= 1e-6 relative")
    if rank == 0:
        print(json.dumps(line), flush=True)
    for stk in e2e_states:
        fca.fca_free(stk)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
