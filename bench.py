#!/usr/bin/env python
"""Benchmark of the MSP Barnes-Hut connectivity update on GB300.

Metric: neuron-searches per second per connectivity update on the 2^20-neuron
workload (64 isotropic Gaussian clusters, std 300 um, centres uniform in a 10 mm
cube, Poisson(2) vacancies clipped to 0..8, sigma = 750 um, theta = 0.3).

One step = one pass of the whole path over that network, starting from empty
connectivity: octree build (Morton codes, sort, topology), 10 consecutive
connectivity updates (bottom-up update, Barnes-Hut search, acceptance, apply),
each followed by spike delivery (5 % of neurons spiking), then a deletion pass
in which every element is retracted, which returns the network to empty so
that every step does the same work. value = searches of all 10 updates / step
time (device time, CUDA events); L2 is flushed between steps. The step's calls
are captured once in a CUDA graph and replayed (--no-graph: direct calls); the
search-kernel times for the roofline come from direct steps with the library's
events.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.

--workload batch measures the batched form instead: 256 independent networks
(log-uniform 10^3 .. 10^6 neurons, about 3.7e7 in total, constant density,
per-network sigma in [500, 1000] um, theta = 0.3). One step = the batched octree
build of all networks + one connectivity update of all of them (one search
launch) + full deletion, captured once in a CUDA graph and replayed; the search
kernel's walk width is chosen by the autotuner before capture.

--workload diff measures the differentiable form: 2^18 neurons uniform in a
4 mm cube, Poisson(2) vacancies, sigma = 800 um, theta = 0.3. One step = the
torch autograd op's forward (octree build, bottom-up update, expected synapse
length over every source's root frontier) and its hand-written adjoint
(gradients for sigma and every position); the config also reports the 50 Adam
steps that calibrate sigma to a 600 um mean length.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "neuron-searches/sec per connectivity update at 2^20 neurons; % of GB300 roofline"
UNIT = "neuron-searches/s"
UPDATES_PER_STEP = 10
FLOPS_PER_EVAL = 12            # d^2 (3 sub + 3 fma/mul), criterion, shifted exponent, count, sum
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--theta", type=float, default=0.3)
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--group", type=int, default=0,
                    help="source neurons per octree walk in the search kernel (0 = default)")
    ap.add_argument("--workload", choices=["clusters", "batch", "diff"], default="clusters")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="run the step as direct calls instead of one captured CUDA graph")
    ap.add_argument("--regroup", action="store_true",
                    help="two-phase search: restarts regrouped by subtree (RELEARN_FLAG_REGROUP)")
    ap.add_argument("--networks", type=int, default=256)
    return ap.parse_args()


def workload(n):
    from paper_2509_26193_gb300 import workloads
    return workloads.gaussian_clusters(n=n)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def search_traffic():
    """DRAM bytes per search-kernel launch from the committed ncu summary, or None when
    the kernel sources changed since those counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "bh_search_traffic_gaussian_clusters_2p20.md")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for f in ("search.cu", "device.cuh", "octree.cu"):
        with open(os.path.join(ROOT, "paper_2509_26193_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    fields = dict(line.split(": ", 1) for line in open(path).read().splitlines()
                  if line.startswith(("sources-sha256", "traffic-bytes-per-launch")))
    if fields.get("sources-sha256", "").strip() != h.hexdigest():
        return None
    return int(fields["traffic-bytes-per-launch"])


def workload_config(net, theta, extra=None):
    cfg = {"workload": f"gaussian_clusters n={net.n} (64 clusters, std 300 um, 10 mm cube, "
                       f"Poisson(2) vacancies 0..8, 20% inhibitory)",
           "n": net.n, "sigma_um": net.sigma, "theta": theta,
           "updates_per_step": UPDATES_PER_STEP,
           "step": "build + 10 x (update + spike delivery) + full deletion",
           "l2": "flushed between steps (256 MB write)"}
    if extra:
        cfg.update(extra)
    return cfg


def warm(fn, steps, min_seconds=2.0):
    """At least `steps` untimed calls, and at least `min_seconds` of them: the first
    process on a fresh GPU runs a few percent slow for its first second or so."""
    import torch
    t0 = time.perf_counter()
    k = 0
    while k < steps or time.perf_counter() - t0 < min_seconds:
        fn()
        k += 1
        if k >= steps:
            torch.cuda.synchronize()
    return k


# ---------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(local_units, local_seconds, world, backend_device=None):
    """Whole-job value: units of all ranks / the slowest rank's time (replicas)."""
    import torch
    import torch.distributed as dist
    if world <= 1:
        return local_units, local_seconds
    dev = backend_device or "cpu"
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------- our arm
class Runner:
    def __init__(self, net, theta, device, group=0, extra_flags=0):
        import torch
        from paper_2509_26193_gb300 import build, relearn as R, workloads
        build.build()
        self.torch, self.R, self.net, self.theta = torch, R, net, theta
        self.group = group
        self.extra_flags = extra_flags
        self.dev = device
        n = net.n
        self.spk_host = [workloads.spikes(n, net.seed, u) for u in range(UPDATES_PER_STEP)]
        self.retract_host = np.full(n, 1 << 20, np.int32)
        # a step's inputs live in one device buffer, each array at a 256-byte aligned
        # offset, so that the end-to-end variant brings them over with one copy from
        # one pinned host buffer of the same layout
        arrays = [("x", net.x), ("y", net.y), ("z", net.z), ("vac_ax", net.vac_ax),
                  ("vac_de", net.vac_de), ("type", net.type), ("retract", self.retract_host)]
        arrays += [(f"spiked{u}", sp) for u, sp in enumerate(self.spk_host)]
        layout, off = {}, 0
        for name, a in arrays:
            a = np.ascontiguousarray(a)
            layout[name] = (off, a)
            off += (a.nbytes + 255) // 256 * 256
        host = np.zeros(off, np.uint8)
        for name, (o, a) in layout.items():
            host[o:o + a.nbytes] = a.view(np.uint8).ravel()
        self.h_in = torch.from_numpy(host).pin_memory()
        self.dev_in = self.h_in.to(device)
        tdt = {np.dtype(np.float32): torch.float32, np.dtype(np.int32): torch.int32,
               np.dtype(np.uint8): torch.uint8}
        view = lambda name: self.dev_in[layout[name][0]:layout[name][0] + layout[name][1].nbytes] \
            .view(tdt[layout[name][1].dtype])
        self.x, self.y, self.z = view("x"), view("y"), view("z")
        self.vac_ax0, self.vac_de0 = view("vac_ax"), view("vac_de")
        self.vac_ax, self.vac_de = self.vac_ax0.clone(), self.vac_de0.clone()
        self.type = view("type")
        self.retract = view("retract")
        self.spiked = [view(f"spiked{u}") for u in range(UPDATES_PER_STEP)]
        self.input = torch.zeros(n, dtype=torch.int32, device=device)
        cap = int(min(net.vac_ax.sum(), net.vac_de.sum())) + 1024
        self.ctx = R.relearn_create(n, cap, 0, device=device.index)
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        self.h_out = torch.empty(n, dtype=torch.int32).pin_memory()
        self.h_cnt = torch.empty(2, dtype=torch.int64).pin_memory()
        self.step_index = 0

    def h2d_bytes(self):
        return int(self.h_in.numel())  # the one input copy of a step (payload + alignment)

    def d2h_bytes(self):
        return 4 * self.net.n + 16

    def step(self, e2e=False, timing=True):
        R, torch = self.R, self.torch
        if e2e:  # this step's inputs arrive from pinned host memory, one copy
            self.dev_in.copy_(self.h_in, non_blocking=True)
        # element-model output for this step: the initial vacancies
        self.vac_ax.copy_(self.vac_ax0)
        self.vac_de.copy_(self.vac_de0)
        R.relearn_build_octree(self.ctx, self.x, self.y, self.z)
        base = 1000 * self.step_index
        for u in range(UPDATES_PER_STEP):
            p = R.params(self.net.sigma, self.theta, self.net.seed, base + u,
                         (R.FLAG_TIMING if timing else 0) | self.extra_flags, self.group)
            R.relearn_update_connectivity(self.ctx, p, self.vac_ax, self.vac_de, self.type)
            R.relearn_deliver_spikes(self.ctx, self.spiked[u], self.input)
        p = R.params(self.net.sigma, self.theta, self.net.seed, base + 999)
        R.relearn_delete_synapses(self.ctx, p, self.retract, self.retract, self.vac_ax,
                                  self.vac_de)
        if e2e:
            self.h_out.copy_(self.input, non_blocking=True)
        self.step_index += 1

    def counters(self):
        s = self.R.relearn_get_last_stats(self.ctx)
        return s["searches_total"], s["evals_total"], s["walk_steps_total"]

    def capture(self):
        """The whole step (vacancy reset, build, 10 updates with delivery, deletion) as
        one CUDA graph; every replay recomputes everything (same inputs, same draws)."""
        torch = self.torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step(timing=False)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step(timing=False)
        torch.cuda.synchronize()

    def timed_graph(self, steps, e2e):
        torch = self.torch
        st = torch.cuda.current_stream()
        total_ms = 0.0
        q0, e0, w0 = self.counters()
        for _ in range(steps):
            self.flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            if e2e:  # this step's inputs arrive from pinned host memory, one copy
                self.dev_in.copy_(self.h_in, non_blocking=True)
            self.graph.replay()
            if e2e:
                self.h_out.copy_(self.input, non_blocking=True)
            b.record(st)
            torch.cuda.synchronize()
            total_ms += a.elapsed_time(b)
        q1, e1, w1 = self.counters()
        return {"ms": total_ms, "searches": q1 - q0, "evals": e1 - e0, "walk_steps": w1 - w0}

    def timed(self, steps, e2e):
        torch = self.torch
        st = torch.cuda.current_stream()
        total_ms = 0.0
        q0, e0, w0 = self.counters()
        self.R.relearn_collect_search_times(self.ctx)
        k_ms, k_n = 0.0, 0
        l0 = self.R.relearn_launch_count()
        for _ in range(steps):
            self.flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            self.step(e2e=e2e)
            b.record(st)
            torch.cuda.synchronize()
            total_ms += a.elapsed_time(b)
            ms, kn = self.R.relearn_collect_search_times(self.ctx)
            k_ms += ms
            k_n += kn
        launches = self.R.relearn_launch_count() - l0
        q1, e1, w1 = self.counters()
        return {"ms": total_ms, "searches": q1 - q0, "evals": e1 - e0, "walk_steps": w1 - w0,
                "kernel_ms": k_ms,
                "kernel_launches": k_n, "launches": launches}


def first_update_profile(runner):
    """Phase times of the first (largest) update of a step, for the breakdown."""
    R = runner.R
    torch = runner.torch
    runner.vac_ax.copy_(runner.vac_ax0)
    runner.vac_de.copy_(runner.vac_de0)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record()
    R.relearn_build_octree(runner.ctx, runner.x, runner.y, runner.z)  # a1-a3
    b1.record()
    p = R.params(runner.net.sigma, runner.theta, runner.net.seed, 0, runner.extra_flags,
                 runner.group)
    s = R.relearn_update_connectivity(runner.ctx, p, runner.vac_ax, runner.vac_de, runner.type,
                                      stats=True)
    s["ms_build"] = b0.elapsed_time(b1)
    p = R.params(runner.net.sigma, runner.theta, runner.net.seed, 999)
    R.relearn_delete_synapses(runner.ctx, p, runner.retract, runner.retract, runner.vac_ax,
                              runner.vac_de)
    runner.torch.cuda.synchronize()
    return s


# ------------------------------------------------------------------ CPU side
def cpu_baseline(net, theta, sample=1 << 17):
    """The FP64 oracle on the host cores: tree build + bottom-up update + a random
    sample of the first update's searches, extrapolated to the whole update."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    if not oracle.openmp_available():
        threads = 1
    t0 = time.perf_counter()
    t = oracle.Tree(net.x, net.y, net.z)
    t1 = time.perf_counter()
    t.reduce(net.vac_de)
    t2 = time.perf_counter()
    qi, qe = oracle.queries(net.vac_ax)
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(len(qi), min(sample, len(qi)), replace=False))
    t3 = time.perf_counter()
    _, diag = t.search_batch(net.sigma, theta, net.seed, 0, qi[sel], qe[sel], threads=threads)
    t4 = time.perf_counter()
    q = len(qi)
    est = (t1 - t0) + (t2 - t1) + (t4 - t3) * q / len(sel)
    return {"value": q / est, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"2^20 octree build + bottom-up update + {len(sel)} of the first update's "
                      f"{q} searches (random sample), search time scaled to all {q}; "
                      f"build {t1 - t0:.2f} s, update {t2 - t1:.2f} s, sample {t4 - t3:.2f} s",
            "evals_per_search": float(diag["evals"].mean())}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    net = workload(args.n)
    threads = (os.cpu_count() or 1) if oracle.openmp_available() else 1
    sample = 1 << 15
    qi, qe = oracle.queries(net.vac_ax)
    rng = np.random.default_rng(1)

    def one(step):
        sel = np.sort(rng.choice(len(qi), sample, replace=False))
        t0 = time.perf_counter()
        t = oracle.Tree(net.x, net.y, net.z)
        t.reduce(net.vac_de)
        t.search_batch(net.sigma, args.theta, net.seed, step, qi[sel], qe[sel], threads=threads)
        return time.perf_counter() - t0

    for w in range(args.warmup):
        one(w)
    secs = [one(args.warmup + k) for k in range(args.steps)]
    tot = sum(secs)
    value = sample * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(net, args.theta),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"per step: octree build + bottom-up update of the 2^20 "
                                       f"network + {sample} random searches of it"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local if ws > 1 else torch.cuda.current_device())
    torch.cuda.set_device(device)
    net = workload(args.n)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(net, args.theta)  # before any CUDA context-heavy work
    from paper_2509_26193_gb300 import relearn as R
    run = Runner(net, args.theta, device, args.group, R.FLAG_REGROUP if args.regroup else 0)
    prof = first_update_profile(run)
    warm(run.step, max(args.warmup, 3))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    if args.graph:
        # search-kernel times (library events) come from direct steps; the step time
        # from graph replays of the same step
        res_k = run.timed(args.steps, e2e=False)
        run.capture()
        warm(run.graph.replay, max(args.warmup, 3))
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(device.index)
    clocks.start()
    res = run.timed_graph(args.steps, e2e=False) if args.graph else run.timed(args.steps, False)
    clk = clocks.stop()
    if args.graph:
        res.update({k: res_k[k] for k in ("kernel_ms", "kernel_launches", "launches")})
    if ws > 1:
        dist.barrier()
    units, secs = aggregate(res["searches"], res["ms"] / 1000.0, ws, device)
    e2e = None
    if not args.no_e2e:
        if not args.graph:
            run.step(e2e=True)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ck2 = ClockSampler(device.index)
        ck2.start()
        r2 = run.timed_graph(args.steps, e2e=True) if args.graph else run.timed(args.steps, True)
        clk2 = ck2.stop()
        u2, s2 = aggregate(r2["searches"], r2["ms"] / 1000.0, ws, device)
        e2e = {"value": u2 / s2, "unit": UNIT, "h2d_bytes_per_step": run.h2d_bytes(),
               "d2h_bytes_per_step": run.d2h_bytes(), "clocks": clk2}
    if ws > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return
    pk, src = peaks()
    clock_mhz = SM_MAX_MHZ
    peak_tflops = SM_COUNT * FP32_LANES * 2 * clock_mhz * 1e6 / 1e12
    flops = FLOPS_PER_EVAL * res["evals"]
    achieved = flops / (res["kernel_ms"] / 1000.0) / 1e12 if res["kernel_ms"] > 0 else 0.0
    roof = {"bound": "alu", "kernel": "search (bh_search_kernel + bh_split_kernel, one launch "
                                      "pair per update)", "achieved": achieved,
            "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "traffic": search_traffic(),
            "peak_source": f"derived: {SM_COUNT} SMs x {FP32_LANES} FP32 lanes x 2 flop/FMA x "
                           f"{clock_mhz:.0f} MHz (FP32 pipe; MEASURED_PEAKS.json has only HBM and "
                           f"bf16 peaks, {src})",
            "work": f"{FLOPS_PER_EVAL} flop per node evaluation x {res['evals']} evaluations in "
                    f"{res['kernel_launches']} launches",
            "kernel_ms_per_launch": res["kernel_ms"] / max(res["kernel_launches"], 1),
            "kernel_share_of_step": res["kernel_ms"] / res["ms"]}
    # the second ALU ceiling: one ex2 on the special-function unit per node evaluation
    # at most, 16 per SM per clock
    mufu_peak = SM_COUNT * 16 * clock_mhz * 1e6 / 1e12
    mufu = res["evals"] / (res["kernel_ms"] / 1000.0) / 1e12 if res["kernel_ms"] > 0 else 0.0
    roof["secondary"] = {"mufu": {"achieved": mufu, "peak": mufu_peak, "unit": "T ex2/s",
                                  "frac": mufu / mufu_peak,
                                  "peak_source": f"derived: {SM_COUNT} SMs x 16 ex2 per clock x "
                                                 f"{clock_mhz:.0f} MHz",
                                  "work": "at most one ex2 per node evaluation"}}
    line = {"metric": METRIC, "value": units / secs, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": res["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(net, args.theta, {
                "parallelism": "replicas" if ws > 1 else "single GPU",
                "searches_per_step": res["searches"] / args.steps,
                "first_update": {"searches": prof["searches"], "formed": prof["formed"],
                                 "ms_total": prof["ms_total"], "ms_reduce": prof["ms_reduce"],
                                 "ms_search": prof["ms_search"],
                                 "ms_search_kernel": prof["ms_search_kernel"],
                                 "ms_accept": prof["ms_accept"], "ms_apply": prof["ms_apply"],
                                 "ms_build_a1_a3": prof["ms_build"],
                                 "searches_per_s": prof["searches"] / (prof["ms_total"] / 1e3)},
                "evals_per_search": res["evals"] / max(res["searches"], 1),
                "search_group": args.group or "default",
                "restarts": "regrouped by subtree" if args.regroup else "inline",
                "execution": "one CUDA graph replay per step" if args.graph else
                             "direct calls (one C-ABI call per operation)",
                "walk_steps_per_search": res["walk_steps"] / max(res["searches"], 1)}),
            "clocks": clk, "e2e": e2e, "gpu_launches": res["launches"],
            "roofline": roof, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------- batched form
BATCH_METRIC = ("neuron-searches/sec per connectivity update, batched form: 256 networks of "
                "10^3..10^6 neurons in one launch; % of GB300 roofline")


def batch_workload(networks):
    from paper_2509_26193_gb300 import workloads
    return workloads.network_batch(networks=networks, seed=4)


def batch_config(b, extra=None):
    cfg = {"workload": f"network_batch: {b.num_networks} networks, sizes log-uniform "
                       f"{b.params['n_range']}, n={b.n}, uniform at 4096 neurons/mm^3, "
                       f"Poisson(2) vacancies 0..8, sigma U[500, 1000] um per network, "
                       f"20% inhibitory",
           "n": b.n, "networks": b.num_networks, "theta": b.theta,
           "step": "batched build + 1 update (all networks, one search launch) + full "
                   "deletion, one CUDA graph replay",
           "l2": f"inputs larger than L2 ({12 * b.n / 1e6:.0f} MB of positions) and 256 MB "
                 f"flush between steps"}
    if extra:
        cfg.update(extra)
    return cfg


class BatchRunner:
    def __init__(self, b, device):
        import torch
        from paper_2509_26193_gb300 import build, relearn as R
        build.build()
        self.torch, self.R, self.b = torch, R, b
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.x, self.y, self.z = d(b.x), d(b.y), d(b.z)
        self.vac_ax0, self.vac_de0 = d(b.vac_ax), d(b.vac_de)
        self.vac_ax, self.vac_de = self.vac_ax0.clone(), self.vac_de0.clone()
        self.type, self.sigma = d(b.type), d(b.sigma)
        self.retract = torch.full((b.n,), 1 << 20, dtype=torch.int32, device=device)
        q = int(b.vac_ax.sum())
        cap = int(min(q, int(b.vac_de.sum()))) + 1024
        self.ctx = R.relearn_create_batched(b.n, cap, b.num_networks, q + 1024,
                                            device=device.index)
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        self.h = {k: pin(getattr(b, k)) for k in ("x", "y", "z", "vac_ax", "vac_de", "type")}
        self.h_out = torch.empty(b.n, dtype=torch.int32).pin_memory()
        self.group = 0
        self.graph = None

    def step(self, flags=0, group=None):
        R, b = self.R, self.b
        self.vac_ax.copy_(self.vac_ax0)
        self.vac_de.copy_(self.vac_de0)
        R.relearn_build_octree_batch(self.ctx, b.offsets, self.x, self.y, self.z)
        p = R.params(0.0, b.theta, b.seed, 1, flags, self.group if group is None else group,
                     net_sigma=self.sigma)
        R.relearn_update_connectivity(self.ctx, p, self.vac_ax, self.vac_de, self.type)
        p = R.params(0.0, b.theta, b.seed, 999, 0, 0, net_sigma=self.sigma)
        R.relearn_delete_synapses(self.ctx, p, self.retract, self.retract, self.vac_ax,
                                  self.vac_de)

    def trial(self, group):
        """One direct (uncaptured) step with the search kernel timed: kernel ms."""
        self.R.relearn_collect_search_times(self.ctx)
        self.step(self.R.FLAG_TIMING, group)
        self.torch.cuda.synchronize()
        ms, n = self.R.relearn_collect_search_times(self.ctx)
        return ms / max(n, 1)

    def capture(self):
        torch = self.torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        torch.cuda.synchronize()

    def counters(self):
        s = self.R.relearn_get_last_stats(self.ctx)
        return s["searches_total"], s["evals_total"]

    def timed(self, steps, e2e=False):
        torch = self.torch
        st = torch.cuda.current_stream()
        total = 0.0
        q0, e0 = self.counters()
        l0 = self.R.relearn_launch_count()
        for _ in range(steps):
            self.flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            c = torch.cuda.Event(enable_timing=True)
            a.record(st)
            if e2e:
                for k in ("x", "y", "z", "type"):
                    getattr(self, k).copy_(self.h[k], non_blocking=True)
                self.vac_ax0.copy_(self.h["vac_ax"], non_blocking=True)
                self.vac_de0.copy_(self.h["vac_de"], non_blocking=True)
            self.graph.replay()
            if e2e:
                self.h_out.copy_(self.vac_ax, non_blocking=True)
            c.record(st)
            torch.cuda.synchronize()
            total += a.elapsed_time(c)
        q1, e1 = self.counters()
        return {"ms": total, "searches": q1 - q0, "evals": e1 - e0,
                "launches_host": self.R.relearn_launch_count() - l0}

    def h2d_bytes(self):
        return 21 * self.b.n

    def d2h_bytes(self):
        return 4 * self.b.n


def batch_cpu_baseline(b, sample=1 << 15):
    """The FP64 oracle on the host cores, on the batch's largest network: its tree build,
    bottom-up update and a random sample of its searches, scaled to all of its searches."""
    import oracle
    oracle.build()
    threads = (os.cpu_count() or 1) if oracle.openmp_available() else 1
    k = int(np.argmax(np.diff(b.offsets)))
    net = b.network(k)
    lo = int(b.offsets[k])
    t0 = time.perf_counter()
    t = oracle.Tree(net.x, net.y, net.z, id_base=lo)
    t.reduce(net.vac_de)
    t1 = time.perf_counter()
    qi, qe = oracle.queries(net.vac_ax)
    sel = np.sort(np.random.default_rng(0).choice(len(qi), min(sample, len(qi)), replace=False))
    t2 = time.perf_counter()
    t.search_batch(net.sigma, b.theta, b.seed, 1, qi[sel], qe[sel], threads=threads)
    t3 = time.perf_counter()
    est = (t1 - t0) + (t3 - t2) * len(qi) / len(sel)
    return {"value": len(qi) / est, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"largest network of the batch (n={net.n}): octree build + bottom-up "
                      f"update ({t1 - t0:.2f} s) + {len(sel)} of its {len(qi)} searches "
                      f"({t3 - t2:.2f} s), scaled to all of its searches"}


def run_batch(args):
    import torch
    from paper_2509_26193_gb300 import autotune
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local if ws > 1 else torch.cuda.current_device())
    torch.cuda.set_device(device)
    b = batch_workload(args.networks)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = batch_cpu_baseline(b)
    run = BatchRunner(b, device)
    run.step()
    torch.cuda.synchronize()
    if args.group:
        best, table = args.group, {}
    else:
        best, table = autotune.tune(run.trial)
    run.group = best
    # launches of one step, counted on direct calls (a graph replay makes the same ones)
    l0 = run.R.relearn_launch_count()
    run.step()
    torch.cuda.synchronize()
    launches_per_step = run.R.relearn_launch_count() - l0
    # search kernel time of one step with the chosen width (for the roofline)
    ks = [run.trial(best) for _ in range(3)]
    q0, e0 = run.counters()
    run.step()
    torch.cuda.synchronize()
    q1, e1 = run.counters()
    run.capture()
    warm(run.graph.replay, max(args.warmup, 3))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(device.index)
    clocks.start()
    res = run.timed(args.steps)
    clk = clocks.stop()
    units, secs = aggregate(res["searches"], res["ms"] / 1000.0, ws, device)
    e2e = None
    if not args.no_e2e:
        ck2 = ClockSampler(device.index)
        ck2.start()
        r2 = run.timed(args.steps, e2e=True)
        clk2 = ck2.stop()
        u2, s2 = aggregate(r2["searches"], r2["ms"] / 1000.0, ws, device)
        e2e = {"value": u2 / s2, "unit": UNIT, "h2d_bytes_per_step": run.h2d_bytes(),
               "d2h_bytes_per_step": run.d2h_bytes(), "clocks": clk2}
    if ws > 1:
        dist.barrier()
        if rank != 0:
            dist.destroy_process_group()
            return
    k_ms = min(ks)
    evals = e1 - e0
    peak_tflops = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = FLOPS_PER_EVAL * evals / (k_ms / 1000.0) / 1e12
    roof = {"bound": "alu", "kernel": "bh_search_kernel", "achieved": achieved,
            "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "traffic": None,
            "peak_source": f"derived: {SM_COUNT} SMs x {FP32_LANES} FP32 lanes x 2 flop/FMA x "
                           f"{SM_MAX_MHZ:.0f} MHz (FP32 pipe)",
            "work": f"{FLOPS_PER_EVAL} flop per node evaluation x {evals} evaluations in one "
                    f"launch (one step, timed uncaptured with CUDA events)",
            "kernel_ms_per_launch": k_ms,
            "kernel_share_of_step": k_ms / (res["ms"] / args.steps)}
    line = {"metric": BATCH_METRIC, "value": units / secs, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": batch_config(b, {
                "parallelism": "replicas" if ws > 1 else "single GPU",
                "searches_per_step": res["searches"] / args.steps,
                "evals_per_search": evals / max(q1 - q0, 1),
                "search_group": best, "autotune_ms": table,
                "graph": "build + update + deletion captured once, replayed per step"}),
            "clocks": clk, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# -------------------------------------------------------- differentiable form
DIFF_METRIC = ("neuron-searches/sec, differentiable form: expected synapse length over the "
               "root frontier and its adjoint at 2^18 neurons; % of GB300 roofline")
FLOPS_PER_CAND_FWD, FLOPS_PER_CAND_BWD = 22, 26


def diff_cpu_baseline(net):
    """The FP64 oracle's forward and gradient on the whole 2^18 network, host cores."""
    import oracle
    oracle.build()
    threads = (os.cpu_count() or 1) if oracle.openmp_available() else 1
    t0 = time.perf_counter()
    t = oracle.Tree(net.x, net.y, net.z)
    t.reduce(net.vac_de)
    oracle.mean_length(t, net.sigma, net.theta, net.vac_ax, net.vac_de, grad=True,
                       threads=threads)
    secs = time.perf_counter() - t0
    units = int(net.vac_ax[net.vac_ax > 0].sum())
    return {"value": units / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the whole 2^18 network: tree build, bottom-up update, forward and "
                      f"FP64 gradient ({secs:.1f} s)"}


def run_diff(args):
    import torch
    from paper_2509_26193_gb300 import build, relearn as R, workloads
    from paper_2509_26193_gb300.differentiable import calibrate_sigma, mean_synapse_length
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local if ws > 1 else torch.cuda.current_device())
    torch.cuda.set_device(device)
    net = workloads.differentiable_cube()
    build.build()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    x, y, z = (d(a).requires_grad_(True) for a in (net.x, net.y, net.z))
    va, vd = d(net.vac_ax), d(net.vac_de)
    sigma = torch.tensor([net.sigma], dtype=torch.float32, device=device, requires_grad=True)
    ctx = R.relearn_create(net.n, 64, device=device.index)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h = {k: pin(getattr(net, k)) for k in ("x", "y", "z", "vac_ax", "vac_de")}
    h_out = torch.empty((3, net.n), dtype=torch.float32).pin_memory()
    units_per_step = int(net.vac_ax[net.vac_ax > 0].sum())

    def step(e2e=False):
        if e2e:
            with torch.no_grad():
                for t, k in ((x, "x"), (y, "y"), (z, "z"), (va, "vac_ax"), (vd, "vac_de")):
                    t.copy_(h[k], non_blocking=True)
        for t in (x, y, z, sigma):
            t.grad = None
        m = mean_synapse_length(ctx, x, y, z, sigma, va, vd, net.theta)
        m.backward()
        if e2e:
            for k, t in enumerate((x, y, z)):
                h_out[k].copy_(t.grad, non_blocking=True)
        return m

    def timed(steps, e2e=False):
        st = torch.cuda.current_stream()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            step(e2e)
            b.record(st)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot

    warm(step, max(args.warmup, 3))
    m = step()
    torch.cuda.synchronize()
    mean0 = float(m.detach())
    e0 = R.relearn_get_last_stats(ctx)["length_evals_total"]
    l0 = R.relearn_launch_count()
    clocks = ClockSampler(device.index)
    clocks.start()
    ms = timed(args.steps)
    clk = clocks.stop()
    launches = R.relearn_launch_count() - l0
    evals = R.relearn_get_last_stats(ctx)["length_evals_total"] - e0
    units, secs = aggregate(units_per_step * args.steps, ms / 1000.0, ws, device)
    e2e = None
    if not args.no_e2e:
        ck2 = ClockSampler(device.index)
        ck2.start()
        ms2 = timed(args.steps, e2e=True)
        clk2 = ck2.stop()
        u2, s2 = aggregate(units_per_step * args.steps, ms2 / 1000.0, ws, device)
        e2e = {"value": u2 / s2, "unit": UNIT, "h2d_bytes_per_step": 20 * net.n,
               "d2h_bytes_per_step": 12 * net.n, "clocks": clk2}
    # sigma calibration: 50 Adam steps toward a 600 um mean length
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sig, means = calibrate_sigma(ctx, x.detach(), y.detach(), z.detach(), va, vd, net.sigma,
                                 600.0, steps=50)
    torch.cuda.synchronize()
    cal_s = time.perf_counter() - t0
    if ws > 1:
        dist.barrier()
        if rank != 0:
            dist.destroy_process_group()
            return
    # the forward and adjoint calls alone (C ABI, CUDA events): the roofline's time
    R.relearn_build_octree(ctx, x.detach(), y.detach(), z.detach())
    prm = R.params(1.0, net.theta, 0, 0, net_sigma=sigma.detach())
    mean_t = torch.empty(1, dtype=torch.float64, device=device)
    gbuf = [torch.empty(net.n, dtype=torch.float32, device=device) for _ in range(3)]
    k0 = R.relearn_get_last_stats(ctx)["length_evals_total"]
    f_ms = b_ms = 0.0
    for _ in range(args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        R.relearn_mean_length(ctx, prm, va, vd, mean_t)
        ev[1].record()
        R.relearn_mean_length_backward(ctx, va, vd, *gbuf)
        ev[2].record()
        torch.cuda.synchronize()
        f_ms += ev[0].elapsed_time(ev[1])
        b_ms += ev[1].elapsed_time(ev[2])
    kevals = R.relearn_get_last_stats(ctx)["length_evals_total"] - k0
    # the oracle last: its OpenMP threads would compete with the host loop above
    cpu = None if ws > 1 or args.no_cpu_baseline else diff_cpu_baseline(net)
    peak_tflops = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    flops = kevals / 2 * (FLOPS_PER_CAND_FWD + FLOPS_PER_CAND_BWD)
    achieved = flops / ((f_ms + b_ms) / 1000.0) / 1e12
    roof = {"bound": "alu", "kernel": "length_kernel (forward + backward)", "achieved": achieved,
            "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "traffic": None,
            "peak_source": f"derived: {SM_COUNT} SMs x {FP32_LANES} FP32 lanes x 2 flop/FMA x "
                           f"{SM_MAX_MHZ:.0f} MHz (FP32 pipe)",
            "work": f"{FLOPS_PER_CAND_FWD} flop per candidate forward + {FLOPS_PER_CAND_BWD} "
                    f"backward x {kevals // 2 // args.steps} candidates per pass, over the "
                    f"forward and adjoint "
                    f"calls' time (CUDA events; their few small kernels included)",
            "forward_ms": f_ms / args.steps, "backward_ms": b_ms / args.steps,
            "kernel_share_of_step": (f_ms + b_ms) / ms}
    line = {"metric": DIFF_METRIC, "value": units / secs, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "differentiable_cube n=262144 (uniform 4 mm cube, Poisson(2) "
                                   "vacancies 0..8, 20% inhibitory)",
                       "n": net.n, "sigma_um": net.sigma, "theta": net.theta,
                       "step": "autograd forward (build + bottom-up update + expected length) "
                               "+ hand-written adjoint (sigma and positions)",
                       "unit": "searches covered = sum of vac_ax over sources, per fwd+bwd",
                       "l2": "256 MB flush between steps",
                       "mean_length_um": mean0,
                       "candidates_per_source_pass": evals / 2 / args.steps /
                       max(int((net.vac_ax > 0).sum()), 1),
                       "calibration": {"steps": 50, "target_um": 600.0,
                                       "sigma_final_um": float(sig[-1]),
                                       "mean_final_um": float(means[-1]),
                                       "seconds": cal_s}},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "diff":
        run_diff(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
