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

Roofline of the search (the dominant kernels): the algorithmic work is the
method's, per search: E node evaluations on the search's path (root frontier and
restarts, as the oracle counts them), 12 FP32 operations each, three of them fused
multiply-adds (15 flop), plus one ex2; 16 bytes per evaluation and 8 per
expansion from L2. E is counted by the library's diagnostics (equal to the
oracle's per search where the paths agree) in one untimed step. The peaks are
measured on the GPU at hand by the library's probe kernels (FP32 FMA chains, ex2
chains, L2 reads), with the SM clock sampled during them.

The default run also measures, as sub-objects of the same line: the theta sweep
(0.2 and 0.5) on the same network, the 2^24-neuron cortical slab (one update with
the octree rebuilt inside the timing), the batched form (256 networks) and the
differentiable form (2^18 neurons). --main-only skips them.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.

--workload batch|diff|slab prints the line of that form alone (see run_batch,
run_diff, run_slab).
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
# the method's arithmetic per node evaluation: d^2 (3 sub + 3 FMA), criterion (2 mul +
# compare), shifted exponent (sub + mul), count multiply, running sum: 12 FP32
# operations, three of them FMAs (2 flop each) = 15 flop; one ex2
OPS_PER_EVAL, FLOPS_PER_EVAL = 12, 15
L2_BYTES_PER_EVAL, L2_BYTES_PER_EXPANSION = 16, 8


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
    ap.add_argument("--workload", choices=["clusters", "batch", "diff", "slab"],
                    default="clusters")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="run the step as direct calls instead of one captured CUDA graph")
    ap.add_argument("--regroup", action="store_true",
                    help="two-phase search: restarts regrouped by subtree (RELEARN_FLAG_REGROUP)")
    ap.add_argument("--networks", type=int, default=256)
    ap.add_argument("--main-only", action="store_true",
                    help="skip the theta sweep, the slab and the batched/differentiable forms")
    ap.add_argument("--launch-list", action="store_true",
                    help="run two direct steps of the workload (the first a warm-up) and exit: "
                         "the command profilers capture (prints the launches of one step)")
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


def profile_counters():
    """Counters of the search launch pair from the committed ncu summary (DRAM bytes
    per launch, issue-active share of the first update), or {} when the kernel
    sources changed since those counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "bh_search_traffic_gaussian_clusters_2p20.md")
    if not os.path.exists(path):
        return {}
    h = hashlib.sha256()
    for f in ("search.cu", "device.cuh", "octree.cu"):
        with open(os.path.join(ROOT, "paper_2509_26193_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    fields = dict(line.split(": ", 1) for line in open(path).read().splitlines()
                  if ": " in line and line.split(": ", 1)[0].replace("-", "").isalnum())
    if fields.get("sources-sha256", "").strip() != h.hexdigest():
        return {}
    out = {}
    for key, name in (("traffic-bytes-per-launch", "traffic"),
                      ("issue-active-first-update", "issue_active"),
                      ("instructions-first-update", "instructions")):
        if key in fields:
            out[name] = float(fields[key])
    return out


def workload_config(net, theta):
    """The workload as both arms name it (static; measured details go elsewhere)."""
    return {"workload": f"gaussian_clusters n={net.n} (64 clusters, std 300 um, 10 mm cube, "
                        f"Poisson(2) vacancies 0..8, 20% inhibitory)",
            "n": net.n, "sigma_um": net.sigma, "theta": theta,
            "updates_per_step": UPDATES_PER_STEP,
            "step": "build + 10 x (update + spike delivery) + full deletion",
            "l2": "flushed between steps (256 MB write)"}


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
        self.path = None

    def start(self):
        import tempfile
        try:
            fd, self.path = tempfile.mkstemp(prefix="relearn_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
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
        with open(self.path) as fh:
            lines = fh.read().splitlines()
        os.unlink(self.path)
        for line in lines:
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


# ---------------------------------------------------------------- ALU peaks
def measure_alu_peaks(device, seconds=0.1):
    """The rates that bound the search, measured on this GPU by the library's probe
    kernels (relearn_peak_probe), each timed alone with CUDA events for about
    `seconds`: FP32 FMA (scalar and packed f32x2 chains), ex2 on the
    special-function unit, and L2 reads of a 64 MB buffer. The SM clock is sampled
    while they run; derived figures (unit counts x that clock) are given beside."""
    import torch
    from paper_2509_26193_gb300 import relearn as R
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    small = torch.zeros(1 << 20, dtype=torch.float32, device=device)
    big = torch.zeros(1 << 24, dtype=torch.float32, device=device)  # 64 MB, inside L2
    ck = ClockSampler(device.index)
    ck.start()
    out = {}
    for name, kind, buf in (("fma", R.PROBE_FMA, small), ("fma2", R.PROBE_FMA2, small),
                            ("ex2", R.PROBE_EX2, small), ("l2", R.PROBE_L2, big)):
        iters = 4
        while True:  # grow the launch until it runs for `seconds`
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ops = R.relearn_peak_probe(kind, iters, buf)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            if ms >= 1000 * seconds or iters > 1 << 30:
                break
            iters = int(iters * max(2.0, 1.2 * 1000 * seconds / max(ms, 1e-3)))
        out[name] = ops / (ms / 1000.0)
    clk = ck.stop()
    mhz = clk.get("sm_mhz") or 0.0
    fma = max(out["fma"], out["fma2"])
    return {"fp32_tflops": 2 * fma / 1e12, "fp32_tops": fma / 1e12,
            "fma_scalar_per_s": out["fma"], "fma_packed_per_s": out["fma2"],
            "ex2_per_s": out["ex2"], "l2_read_gbs": out["l2"] / 1e9,
            "sms": sms, "clocks": clk,
            "derived_at_sampled_clock": {
                "fp32_tflops": sms * 128 * 2 * mhz * 1e6 / 1e12,
                "issue_warp_inst_per_s": sms * 4 * mhz * 1e6,
                "ex2_per_clock_per_sm": out["ex2"] / (sms * mhz * 1e6) if mhz else None},
            "how": "relearn_peak_probe: 4 blocks of 256 threads per SM; FMA and ex2 as "
                   "independent dependency chains, L2 as 16-byte ld.global.cg reads of a 64 MB "
                   "buffer; each launch timed alone with CUDA events"}


def search_roofline(kernel_ms, launches, evals_alg, evals_dedup, expansions, pk, counters,
                    label):
    """Roofline of the search launches (see the module docstring)."""
    secs = kernel_ms / 1000.0
    flops = FLOPS_PER_EVAL * evals_alg
    achieved = flops / secs / 1e12 if secs > 0 else 0.0
    roof = {"bound": "alu", "kernel": label, "achieved": achieved,
            "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
            "frac": achieved / pk["fp32_tflops"],
            "traffic": counters.get("traffic"),
            "peak_source": f"measured: FP32 FMA chains on this GPU ({pk['fp32_tops']:.1f} T FMA/s"
                           f" x 2 flop; SM clock {pk['clocks'].get('sm_mhz')} MHz during the "
                           f"probe)",
            "work": f"{FLOPS_PER_EVAL} flop ({OPS_PER_EVAL} FP32 operations, 3 of them FMAs) x "
                    f"{evals_alg:.4g} node evaluations (the oracle's count per search: root "
                    f"frontier and restarts) in {launches} launches",
            "kernel_ms_per_launch": kernel_ms / max(launches, 1)}
    ex2 = evals_dedup / secs if secs > 0 else 0.0
    l2 = (L2_BYTES_PER_EVAL * evals_alg + L2_BYTES_PER_EXPANSION * expansions) / secs / 1e9 \
        if secs > 0 else 0.0
    ops = OPS_PER_EVAL * evals_alg / secs / 1e12 if secs > 0 else 0.0
    roof["secondary"] = {
        "fp32_pipe_ops": {"achieved": ops, "peak": pk["fp32_tops"], "unit": "T FP32 ops/s",
                          "frac": ops / pk["fp32_tops"],
                          "work": f"{OPS_PER_EVAL} FP32 operations per evaluation (an FMA "
                                  f"counts once: the pipe's issue rate)"},
        "dedup": {"achieved": FLOPS_PER_EVAL * evals_dedup / secs / 1e12 if secs else 0.0,
                  "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
                  "frac": FLOPS_PER_EVAL * evals_dedup / secs / 1e12 / pk["fp32_tflops"]
                  if secs else 0.0,
                  "work": f"{evals_dedup:.4g} evaluations the kernels made (a source's root "
                          f"frontier once for all its searches)"},
        "mufu_ex2": {"achieved": ex2 / 1e12, "peak": pk["ex2_per_s"] / 1e12, "unit": "T ex2/s",
                     "frac": ex2 / pk["ex2_per_s"],
                     "work": "one ex2 per evaluation the kernels made"},
        "l2": {"achieved": l2, "peak": pk["l2_read_gbs"], "unit": "GB/s",
               "frac": l2 / pk["l2_read_gbs"],
               "work": f"{L2_BYTES_PER_EVAL} B per evaluation + {L2_BYTES_PER_EXPANSION} B per "
                       f"expansion, algorithmic"}}
    if "issue_active" in counters:
        roof["secondary"]["issue_active_first_update"] = {
            "frac": counters["issue_active"] / 100.0,
            "source": "ncu smsp__issue_active of the first update's launch (profiles/)"}
    return roof


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

    def diag_step(self):
        """One untimed step with the search diagnostics on: the oracle-basis node
        evaluations (per search: root frontier + restarts) summed over its updates."""
        R = self.R
        self.vac_ax.copy_(self.vac_ax0)
        self.vac_de.copy_(self.vac_de0)
        R.relearn_build_octree(self.ctx, self.x, self.y, self.z)
        q0, e0, w0 = self.counters()
        evals = 0
        for u in range(UPDATES_PER_STEP):
            p = R.params(self.net.sigma, self.theta, self.net.seed, 500000 + u,
                         R.FLAG_DIAG | self.extra_flags, self.group)
            R.relearn_update_connectivity(self.ctx, p, self.vac_ax, self.vac_de, self.type)
            evals += int(R.relearn_get_search_diag(self.ctx)["evals"].astype(np.int64).sum())
        q1, e1, w1 = self.counters()
        p = R.params(self.net.sigma, self.theta, self.net.seed, 500999)
        R.relearn_delete_synapses(self.ctx, p, self.retract, self.retract, self.vac_ax,
                                  self.vac_de)
        self.torch.cuda.synchronize()
        # the library counts evaluations and walk steps only in counted (here: diagnostic)
        # updates; the timed steps run uncounted
        return {"searches": q1 - q0, "evals_alg": evals, "evals_dedup": e1 - e0,
                "walk_steps": w1 - w0}

    def build_graph_ms(self, reps=20):
        """The octree build (a1-a3) alone, captured in a CUDA graph and replayed: its
        device time without the host's launch gaps."""
        torch, R = self.torch, self.R
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            R.relearn_build_octree(self.ctx, self.x, self.y, self.z)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            R.relearn_build_octree(self.ctx, self.x, self.y, self.z)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def first_update_graph_ms(self, reps=5):
        """Phase times of the first update from the library's events inside a captured
        and replayed update (initial vacancies, octree build, one update without
        diagnostics): device time without the host's launch gaps between the small
        kernels. A deletion of every synapse after each replay (outside the graph)
        leaves the store empty for the next."""
        torch, R = self.torch, self.R
        p = R.params(self.net.sigma, self.theta, self.net.seed, 0,
                     R.FLAG_TIMING | self.extra_flags, self.group)
        pdel = R.params(self.net.sigma, self.theta, self.net.seed, 999)

        def body():
            self.vac_ax.copy_(self.vac_ax0)
            self.vac_de.copy_(self.vac_de0)
            R.relearn_build_octree(self.ctx, self.x, self.y, self.z)
            R.relearn_update_connectivity(self.ctx, p, self.vac_ax, self.vac_de, self.type)

        def clear():
            R.relearn_delete_synapses(self.ctx, pdel, self.retract, self.retract, self.vac_ax,
                                      self.vac_de)

        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            body()
            clear()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            body()
        keys = ("ms_reduce", "ms_search_kernel", "ms_accept", "ms_apply", "ms_total")
        acc = dict.fromkeys(keys, 0.0)
        for _ in range(reps):
            g.replay()
            torch.cuda.synchronize()
            st = R.relearn_get_last_stats(self.ctx)
            for k in keys:
                acc[k] += st[k]
            clear()
        torch.cuda.synchronize()
        R.relearn_collect_search_times(self.ctx)  # drop the replays' search events
        return {k: v / reps for k, v in acc.items()}

    def close(self):
        self.ctx.close()

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
        q0 = self.counters()[0]
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
        return {"ms": total_ms, "searches": self.counters()[0] - q0}

    def timed(self, steps, e2e):
        torch = self.torch
        st = torch.cuda.current_stream()
        total_ms = 0.0
        q0 = self.counters()[0]
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
        return {"ms": total_ms, "searches": self.counters()[0] - q0, "kernel_ms": k_ms,
                "kernel_launches": k_n, "launches": launches}


def first_update_profile(runner):
    """Phase times of the first (largest) update of a step, for the breakdown, and its
    requests (diagnostics on) for the comparison with the oracle's sample."""
    R = runner.R
    torch = runner.torch
    runner.vac_ax.copy_(runner.vac_ax0)
    runner.vac_de.copy_(runner.vac_de0)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record()
    R.relearn_build_octree(runner.ctx, runner.x, runner.y, runner.z)  # a1-a3
    b1.record()
    p = R.params(runner.net.sigma, runner.theta, runner.net.seed, 0,
                 runner.extra_flags | R.FLAG_DIAG, runner.group)
    s = R.relearn_update_connectivity(runner.ctx, p, runner.vac_ax, runner.vac_de, runner.type,
                                      stats=True)
    s["ms_build"] = b0.elapsed_time(b1)
    s["targets"], _ = R.relearn_get_requests(runner.ctx)
    p = R.params(runner.net.sigma, runner.theta, runner.net.seed, 999)
    R.relearn_delete_synapses(runner.ctx, p, runner.retract, runner.retract, runner.vac_ax,
                              runner.vac_de)
    runner.torch.cuda.synchronize()
    return s


# ------------------------------------------------------------------ CPU side
def cpu_baseline(net, theta, sample=1 << 17, sample_1=1 << 12):
    """The FP64 oracle on the host cores: tree build + bottom-up update + a random
    sample of the first update's searches, extrapolated to the whole update; once with
    OpenMP over the searches on every core and once single-threaded. The sample's
    targets and margins are kept for the comparison with the GPU's requests."""
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
    tgt, diag = t.search_batch(net.sigma, theta, net.seed, 0, qi[sel], qe[sel], threads=threads)
    t4 = time.perf_counter()
    sel1 = sel[:sample_1]
    t.search_batch(net.sigma, theta, net.seed, 0, qi[sel1], qe[sel1], threads=1)
    t5 = time.perf_counter()
    t.close()
    q = len(qi)
    est = (t1 - t0) + (t2 - t1) + (t4 - t3) * q / len(sel)
    est1 = (t1 - t0) + (t2 - t1) + (t5 - t4) * q / len(sel1)
    base = {"value": q / est, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"2^20 octree build + bottom-up update + {len(sel)} of the first update's "
                      f"{q} searches (random sample), search time scaled to all {q}; "
                      f"build {t1 - t0:.2f} s, update {t2 - t1:.2f} s, sample {t4 - t3:.2f} s",
            "single_thread": {"value": q / est1, "unit": UNIT, "cores": 1,
                              "sample": f"the same build and update (serial) + {len(sel1)} of "
                                        f"the sampled searches on one thread "
                                        f"({t5 - t4:.2f} s), scaled to all {q}"},
            "evals_per_search": float(diag["evals"].mean()),
            "expansions_per_search": float(diag["expansions"].mean())}
    return base, {"sel": sel, "targets": tgt, "diag": diag}


def parity_sample(gpu_targets, orc):
    """The GPU's first-update requests against the oracle's on the baseline's sample:
    the exemption shares and the mismatches (the tests assert the same rule)."""
    if orc is None:
        return None
    g = gpu_targets[orc["sel"]]
    d = orc["diag"]
    diff = g != orc["targets"]
    out = {"searches": int(len(g)), "differ": int(diff.sum())}
    for tol in (1e-5, 1e-6):
        ex = (d["margin_ac"] < tol) | (d["margin_draw"] < tol)
        out[f"exempt_share_{tol:g}"] = float(ex.mean())
        out[f"differ_outside_exemption_{tol:g}"] = int((diff & ~ex).sum())
    return out


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
        t.close()
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


def measure_clusters(net, theta, device, args, pk, counters, regroup=False, e2e=True,
                     profile=True, xe=None):
    """The clustered step at one theta: timed graph replays (and the end-to-end
    variant), the search kernels' CUDA-event times from direct steps, the algorithmic
    work from one diagnostics step. Returns a dict (and the runner's first-update
    requests when profile is set)."""
    import torch
    from paper_2509_26193_gb300 import relearn as R
    run = Runner(net, theta, device, args.group, R.FLAG_REGROUP if regroup else 0)
    prof = first_update_profile(run) if profile else None
    warm(run.step, max(args.warmup, 3))
    torch.cuda.synchronize()
    dg = run.diag_step()
    build_ms = run.build_graph_ms() if profile else None
    upd_graph = run.first_update_graph_ms() if profile else None
    if args.graph:
        # search-kernel times (library events) come from direct steps; the step time
        # from graph replays of the same step
        res_k = run.timed(args.steps, e2e=False)
        run.capture()
        warm(run.graph.replay, max(args.warmup, 3))
        torch.cuda.synchronize()
    clocks = ClockSampler(device.index)
    clocks.start()
    res = run.timed_graph(args.steps, e2e=False) if args.graph else run.timed(args.steps, False)
    clk = clocks.stop()
    if args.graph:
        res.update({k: res_k[k] for k in ("kernel_ms", "kernel_launches", "launches")})
    out = {"res": res, "clocks": clk, "diag": dg, "prof": prof, "runner": run,
           "build_graph_ms": build_ms, "first_update_graph": upd_graph}
    if e2e and not args.no_e2e:
        if not args.graph:
            run.step(e2e=True)
        torch.cuda.synchronize()
        ck2 = ClockSampler(device.index)
        ck2.start()
        r2 = run.timed_graph(args.steps, e2e=True) if args.graph else run.timed(args.steps, True)
        out["e2e"] = {"res": r2, "clocks": ck2.stop()}
    # work of the timed region: the oracle-basis evaluations per search (diagnostics
    # step) x the region's searches; expansions from the oracle's ratio X / E (xe)
    evals_alg = dg["evals_alg"] / max(dg["searches"], 1) * res["searches"]
    evals_made = dg["evals_dedup"] / max(dg["searches"], 1) * res["searches"]
    out["roofline"] = search_roofline(
        res["kernel_ms"], res["kernel_launches"], evals_alg, evals_made,
        (xe or 0.0) * evals_alg, pk, counters,
        "search (bh_search_kernel + bh_split_kernel, one launch pair per update)")
    if xe is None:
        out["roofline"]["secondary"]["l2"]["work"] += " (expansions not counted: no oracle sample)"
    out["roofline"]["kernel_share_of_step"] = res["kernel_ms"] / res["ms"]
    return out


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
    cpu, orc_sample = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, orc_sample = cpu_baseline(net, args.theta)  # before the GPU work
    from paper_2509_26193_gb300 import build
    build.build()
    pk = measure_alu_peaks(device)
    counters = profile_counters()
    if ws > 1:
        dist.barrier()
    xe = cpu["expansions_per_search"] / max(cpu["evals_per_search"], 1e-9) if cpu else None
    m = measure_clusters(net, args.theta, device, args, pk, counters, regroup=args.regroup,
                         xe=xe)
    res, clk, run = m["res"], m["clocks"], m["runner"]
    if ws > 1:
        dist.barrier()
    units, secs = aggregate(res["searches"], res["ms"] / 1000.0, ws, device)
    e2e = None
    if "e2e" in m:
        r2 = m["e2e"]["res"]
        u2, s2 = aggregate(r2["searches"], r2["ms"] / 1000.0, ws, device)
        e2e = {"value": u2 / s2, "unit": UNIT, "h2d_bytes_per_step": run.h2d_bytes(),
               "d2h_bytes_per_step": run.d2h_bytes(), "clocks": m["e2e"]["clocks"]}
    if ws > 1:
        dist.barrier()
    if rank != 0:
        run.close()
        dist.destroy_process_group()
        return
    prof = m["prof"]
    dg = m["diag"]
    roof = m["roofline"]
    details = {
        "parallelism": "replicas" if ws > 1 else "single GPU",
        "searches_per_step": res["searches"] / args.steps,
        "first_update": {"searches": prof["searches"], "formed": prof["formed"],
                         "ms_total": prof["ms_total"], "ms_reduce": prof["ms_reduce"],
                         "ms_search": prof["ms_search"],
                         "ms_search_kernel": prof["ms_search_kernel"],
                         "ms_accept": prof["ms_accept"], "ms_apply": prof["ms_apply"],
                         "ms_build_a1_a3": prof["ms_build"],
                         "ms_build_a1_a3_graph": m["build_graph_ms"],
                         "graph_replay": m["first_update_graph"],
                         "searches_per_s": prof["searches"] / (prof["ms_total"] / 1e3)},
        "evals_per_search_algorithmic": dg["evals_alg"] / max(dg["searches"], 1),
        "evals_per_search_made": dg["evals_dedup"] / max(dg["searches"], 1),
        "search_group": args.group or "default",
        "restarts": "regrouped by subtree" if args.regroup else "inline",
        "execution": "one CUDA graph replay per step" if args.graph else
                     "direct calls (one C-ABI call per operation)",
        "launches_per_step": res["launches"] / args.steps,
        "walk_steps_per_search": dg["walk_steps"] / max(dg["searches"], 1),
        "parity_sample": parity_sample(prof["targets"], orc_sample),
        "alu_peaks": pk}
    line = {"metric": METRIC, "value": units / secs, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": res["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(net, args.theta),
            "clocks": clk, "e2e": e2e, "gpu_launches": res["launches"],
            "roofline": roof, "cpu_baseline": cpu, "details": details}
    run.close()
    del run, m
    torch.cuda.empty_cache()
    if ws == 1 and not args.main_only:
        line.update(extras(args, net, device, pk, counters, xe))
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def extras(args, net, device, pk, counters, xe=None):
    """The other configurations and forms, each measured in the same process."""
    import torch
    out = {"theta_sweep": {}, "forms": {}}
    for theta in (0.2, 0.5):
        t0 = time.perf_counter()
        m = measure_clusters(net, theta, device, args, pk, counters, e2e=False, profile=False,
                             xe=xe)
        r = m["res"]
        out["theta_sweep"][str(theta)] = {
            "value": r["searches"] / (r["ms"] / 1000.0), "unit": UNIT,
            "ms_per_step": r["ms"] / args.steps, "steps": args.steps,
            "searches_per_step": r["searches"] / args.steps, "clocks": m["clocks"],
            "roofline": {k: m["roofline"][k] for k in ("achieved", "peak", "unit", "frac")},
            "evals_per_search_algorithmic": m["diag"]["evals_alg"] / max(m["diag"]["searches"], 1),
            "seconds": time.perf_counter() - t0}
        m["runner"].close()
        del m
        torch.cuda.empty_cache()
    for name, fn in (("slab_2p24", run_slab), ("batched", run_batch),
                     ("differentiable", run_diff)):
        t0 = time.perf_counter()
        line = fn(args, embedded=True, pk=pk)
        keep = {k: line.get(k) for k in ("metric", "value", "unit", "ms_per_step", "steps",
                                         "config", "clocks", "e2e", "roofline", "cpu_baseline",
                                         "details")}
        keep["seconds"] = time.perf_counter() - t0
        if name == "slab_2p24":
            out[name] = keep
        else:
            out["forms"][name] = keep
        torch.cuda.empty_cache()
    return out


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
        q0 = self.counters()[0]
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
        return {"ms": total, "searches": self.counters()[0] - q0,
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


def run_batch(args, embedded=False, pk=None):
    import torch
    from paper_2509_26193_gb300 import autotune
    ws, rank, local = (1, 0, 0) if embedded else dist_env()
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
    if pk is None:
        from paper_2509_26193_gb300 import build
        build.build()
        pk = measure_alu_peaks(device)
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
    run.step(run.R.FLAG_DIAG)  # the oracle-basis evaluations per search
    torch.cuda.synchronize()
    q1, e1 = run.counters()
    evals_alg = int(run.R.relearn_get_search_diag(run.ctx)["evals"].astype(np.int64).sum())
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
    run.ctx.close()
    if ws > 1:
        dist.barrier()
        if rank != 0:
            dist.destroy_process_group()
            return None
    k_ms = min(ks)
    roof = search_roofline(k_ms, 1, evals_alg, e1 - e0, 0.0, pk, {},
                           "bh_search_kernel (batched: every network's searches in one launch)")
    roof["secondary"]["l2"]["work"] += " (expansions not counted)"
    roof["kernel_share_of_step"] = k_ms / (res["ms"] / args.steps)
    line = {"metric": BATCH_METRIC, "value": units / secs, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": batch_config(b),
            "details": {"parallelism": "replicas" if ws > 1 else "single GPU",
                        "searches_per_step": res["searches"] / args.steps,
                        "evals_per_search_algorithmic": evals_alg / max(q1 - q0, 1),
                        "evals_per_search_made": (e1 - e0) / max(q1 - q0, 1),
                        "search_group": best, "autotune_ms": table,
                        "graph": "build + update + deletion captured once, replayed per step"},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "cpu_baseline": cpu}
    if not embedded:
        line["details"]["alu_peaks"] = pk
        print(json.dumps(line), flush=True)
        if ws > 1:
            dist.destroy_process_group()
    return line


# ------------------------------------------------------------------ the slab
SLAB_METRIC = ("neuron-searches/sec per connectivity update, 2^24-neuron cortical slab, "
               "octree rebuilt inside the timing; % of GB300 roofline")


def run_slab(args, embedded=False, pk=None):
    """2^24 neurons in a 10-layer slab (20 x 20 x 2.5 mm, Poisson(1) vacancies,
    sigma = 1000 um, theta = 0.3). One step = octree build + one connectivity update
    (timed together) + full deletion (untimed, returns the network to empty)."""
    import torch
    from paper_2509_26193_gb300 import build, relearn as R, workloads
    ws, rank, local = (1, 0, 0) if embedded else dist_env()
    device = torch.device("cuda", local if ws > 1 else torch.cuda.current_device())
    torch.cuda.set_device(device)
    build.build()
    if pk is None:
        pk = measure_alu_peaks(device)
    net = workloads.cortical_slab()
    q = int(net.vac_ax.sum())
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    x, y, z = d(net.x), d(net.y), d(net.z)
    va0, vd0, typ = d(net.vac_ax), d(net.vac_de), d(net.type)
    va, vd = va0.clone(), vd0.clone()
    retract = torch.full((net.n,), 1 << 20, dtype=torch.int32, device=device)
    ctx = R.relearn_create(net.n, q + 1024, 0, device=device.index)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    steps = max(1, min(args.steps, 3))
    state = {"k": 0}

    def one(flags=0, timed=True):
        va.copy_(va0)
        vd.copy_(vd0)
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        R.relearn_build_octree(ctx, x, y, z)
        p = R.params(net.sigma, net.theta, net.seed, 10 * state["k"], flags)
        R.relearn_update_connectivity(ctx, p, va, vd, typ)
        b.record()
        p = R.params(net.sigma, net.theta, net.seed, 10 * state["k"] + 9)
        R.relearn_delete_synapses(ctx, p, retract, retract, va, vd)
        torch.cuda.synchronize()
        state["k"] += 1
        return a.elapsed_time(b)

    one()  # warm-up
    s0 = R.relearn_get_last_stats(ctx)
    one(R.FLAG_DIAG)
    evals_alg = int(R.relearn_get_search_diag(ctx)["evals"].astype(np.int64).sum())
    R.relearn_collect_search_times(ctx)
    s1 = R.relearn_get_last_stats(ctx)
    k_ms = [one(R.FLAG_TIMING) for _ in range(steps)]
    kms, kn = R.relearn_collect_search_times(ctx)
    ck = ClockSampler(device.index)
    ck.start()
    ms = [one() for _ in range(steps)]
    clk = ck.stop()
    ctx.close()
    searches = s1["searches_total"] - s0["searches_total"]
    evals_dedup = s1["evals_total"] - s0["evals_total"]
    roof = search_roofline(kms / max(kn, 1), 1, evals_alg, evals_dedup, 0.0, pk, {},
                           "search (bh_search_kernel + bh_split_kernel, one launch pair)")
    roof["secondary"]["l2"]["work"] += " (expansions not counted)"
    tot = sum(ms)
    line = {"metric": SLAB_METRIC, "value": searches * steps / (tot / 1000.0), "unit": UNIT,
            "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": tot / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "cortical_slab n=16777216 (20 x 20 x 2.5 mm, 10 layers, "
                                   "Poisson(1) vacancies, 20% inhibitory)",
                       "n": net.n, "sigma_um": net.sigma, "theta": net.theta,
                       "step": "octree build + one connectivity update (timed); full deletion "
                               "after the timed region",
                       "l2": "256 MB flush before every step; inputs larger than L2"},
            "details": {"searches_per_step": searches,
                        "evals_per_search_algorithmic": evals_alg / max(searches, 1),
                        "evals_per_search_made": evals_dedup / max(searches, 1),
                        "timed_with_search_events_ms": sum(k_ms) / steps},
            "clocks": clk, "e2e": None, "roofline": roof, "cpu_baseline": None}
    if not embedded:
        print(json.dumps(line), flush=True)
    return line


# -------------------------------------------------------- differentiable form
DIFF_METRIC = ("neuron-searches/sec, differentiable form: expected synapse length over the "
               "root frontier and its adjoint at 2^18 neurons; % of GB300 roofline")
# flop per frontier candidate (an FMA counts 2): forward d^2 8, criterion 3, attraction
# 3, S += a 1, a d and a D 4 (19; sqrt and ex2 on the special-function unit); adjoint
# d^2 8, criterion 3, attraction 3, q 1, d - l 1, covariance 4, D - Dbar 1, kappa 4,
# kappa r 3, direct term 3, node adjoint 3 (33; sqrt, rcp and ex2 on that unit)
FLOPS_PER_CAND_FWD, FLOPS_PER_CAND_BWD = 19, 33


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


def run_diff(args, embedded=False, pk=None):
    import torch
    from paper_2509_26193_gb300 import build, relearn as R, workloads
    from paper_2509_26193_gb300.differentiable import calibrate_sigma, mean_synapse_length
    ws, rank, local = (1, 0, 0) if embedded else dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local if ws > 1 else torch.cuda.current_device())
    torch.cuda.set_device(device)
    net = workloads.differentiable_cube()
    build.build()
    if pk is None:
        pk = measure_alu_peaks(device)
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
    # sigma calibration: 50 Adam steps toward a 600 um mean length (two untimed steps
    # first: the first optimizer step of a process pays a one-time start-up cost)
    calibrate_sigma(ctx, x.detach(), y.detach(), z.detach(), va, vd, net.sigma, 600.0, steps=2)
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
    ctx.close()
    flops = kevals / 2 * (FLOPS_PER_CAND_FWD + FLOPS_PER_CAND_BWD)
    achieved = flops / ((f_ms + b_ms) / 1000.0) / 1e12
    roof = {"bound": "alu", "kernel": "length_kernel (forward + backward)", "achieved": achieved,
            "peak": pk["fp32_tflops"], "unit": "TFLOP/s", "frac": achieved / pk["fp32_tflops"],
            "traffic": None,
            "peak_source": f"measured: FP32 FMA chains on this GPU ({pk['fp32_tops']:.1f} T FMA/s"
                           f" x 2 flop)",
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
                       "l2": "256 MB flush between steps"},
            "details": {"mean_length_um": mean0,
                        "candidates_per_source_pass": evals / 2 / args.steps /
                        max(int((net.vac_ax > 0).sum()), 1),
                        "calibration": {"steps": 50, "target_um": 600.0,
                                        "sigma_final_um": float(sig[-1]),
                                        "mean_final_um": float(means[-1]),
                                        "seconds": cal_s}},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "cpu_baseline": cpu}
    if not embedded:
        print(json.dumps(line), flush=True)
        if ws > 1:
            dist.destroy_process_group()
    return line


def run_launch_list(args):
    """Two direct (uncaptured) steps, no timing: the second step's kernels are the ones
    a launch list or a per-kernel capture takes (skip the first step's launches)."""
    import torch
    from paper_2509_26193_gb300 import build, relearn as R
    build.build()
    device = torch.device("cuda", torch.cuda.current_device())
    if args.workload == "batch":
        run = BatchRunner(batch_workload(args.networks), device)
        step = run.step
    elif args.workload == "diff":
        from paper_2509_26193_gb300 import workloads
        from paper_2509_26193_gb300.differentiable import mean_synapse_length
        net = workloads.differentiable_cube()
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        x, y, z = (d(a).requires_grad_(True) for a in (net.x, net.y, net.z))
        va, vd = d(net.vac_ax), d(net.vac_de)
        sigma = torch.tensor([net.sigma], dtype=torch.float32, device=device,
                             requires_grad=True)
        ctx = R.relearn_create(net.n, 64)

        def step():
            mean_synapse_length(ctx, x, y, z, sigma, va, vd, net.theta).backward()
    else:
        run = Runner(workload(args.n), args.theta, device, args.group,
                     R.FLAG_REGROUP if args.regroup else 0)
        step = lambda: run.step(timing=False)
    counts = []
    for _ in range(2):
        l0 = R.relearn_launch_count()
        step()
        torch.cuda.synchronize()
        counts.append(R.relearn_launch_count() - l0)
    print(json.dumps({"launch_list": args.workload, "launches_per_step": counts}), flush=True)


def main():
    args = parse()
    if args.launch_list:
        run_launch_list(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "diff":
        run_diff(args)
    elif args.workload == "slab":
        run_slab(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
