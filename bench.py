#!/usr/bin/env python3
"""Benchmark: cooperative BFS on an R-MAT scale-22 graph (one GB300).

Workload (the headline configuration, the largest single-GPU graph of the measurement
plan and the one the HBM-roofline target is stated on): directed R-MAT, scale 22, edge
factor 16, a/b/c/d = 0.57/0.19/0.19/0.05, seed 22, self-loops and duplicates removed;
source = highest out-degree vertex.  One step = one complete traversal (init kernel +
persistent cooperative kernel, its scheduler polling for offer_kill / request_fork) with
the graph already resident in HBM.  value = GTEPS = E_s / t, E_s = out-edges of reached
vertices.

Also on the same JSON line: the roofline of the persistent kernel (algorithmic bytes
4V + 20 V_r + 8 E_s per launch over its CUDA-event duration against the measured HBM
copy bandwidth), the end-to-end number through the C ABI with host buffers (H2D of the
CSR, D2H of the levels inside the timed region), the CPU oracle timed on this host,
clock samples taken during the timed region, parity of the last timed step's output
against the oracle, and secondary figures (skipped with --no-extras): frontier SSSP on
R-MAT scale 20 with its own roofline, e2e and oracle baseline, the non-cooperative
baseline's overhead ratio and random kill/fork schedules, the co-runner (fp32 saxpy on
half the SMs every 16.7 ms) with and without cooperation, gather time under each kill
mode, the topology-driven SSSP, the work-stealing octree, the batched and served forms,
the 256x256 grid BFS (barrier-latency bound) and empty-barrier latency.

--impl reference times the CPU oracle (FIFO-queue BFS, one core) on the same workload:
the slow reference arm.

Multi-GPU (--gpus N under torchrun): replicas only -- every rank runs the same
workload on its own GPU; value = all ranks' edges / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BFS/SSSP GTEPS (1 GB300, % HBM roofline); barrier us; co-runner p99 latency"
WORKLOADS = {
    # name: (graph kind, scale, graph seed, weight seed, traversal)
    "rmat22-bfs": ("rmat", 22, 22, None, "bfs"),    # the headline configuration
    "rmat20-sssp": ("rmat", 20, 20, 21, "sssp"),
    "grid256-bfs": ("grid", 256, None, None, "bfs"),
}

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the persistent kernel, per
# workload, from the ncu captures summarised in profiles/; an entry is used only while
# the kernel sources still have the digest it was taken on (otherwise null).
TRAFFIC = {
    "rmat22-bfs": {"sources_sha": "1f6f5f36c732ece4", "bytes": 391598592},
    "rmat20-sssp": {"sources_sha": "1f6f5f36c732ece4", "bytes": 201957120},
}


def sources_sha() -> str:
    h = hashlib.sha256()
    for rel in ("paper_1707_01989_gb300/csrc/coop.cu", "paper_1707_01989_gb300/csrc/coop_runtime.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region: the
    sampler is running (its first sample in) before the region starts, samples every
    `every_ms` (20 ms by default, for timed regions of tens of milliseconds), and only
    samples taken from the region's start on are summarised.  Latency measurements that
    run for seconds sample every 200 ms: each query takes the driver's locks, which a
    CUDA call made meanwhile (a launch, a synchronise) waits for."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, every_ms: int = 20):
        self.dev = device_index
        self.every_ms = int(every_ms)
        self.proc = None
        self.lines = []  # (host time, line)
        self.t0 = 0.0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.every_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            t_wait = time.perf_counter()
            while not self.lines and time.perf_counter() - t_wait < 3.0 and self.proc.poll() is None:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        self.t0 = time.perf_counter()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            time.sleep(min(0.25, 1.5 * self.every_ms / 1e3))  # one more sample after the region
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for t, ln in self.lines if t >= self.t0] or [ln for _, ln in self.lines[-1:]]
        for ln in inside:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


HEADLINE = "rmat22-bfs"


def load_workload(name=HEADLINE):
    """(graph, weights or None, source, traversal) of a named workload."""
    import graphgen as gg
    kind, scale, seed, wseed, trav = WORKLOADS[name]
    if kind == "grid":
        return gg.grid(scale, scale), None, 0, trav
    g = gg.rmat(scale, 16, seed=seed)
    w = gg.weights(g, wseed) if wseed is not None else None
    return g, w, gg.max_out_degree_vertex(g), trav


def reached_work(g, reached_mask):
    import numpy as np
    deg = np.diff(g.row_off.astype(np.int64))
    return int(reached_mask.sum()), int(deg[reached_mask].sum())


def oracle_run(g, w, src, trav):
    import oracle
    return oracle.dijkstra(g, w, src) if trav == "sssp" else oracle.bfs(g, src)


def reached_of(out, trav):
    import numpy as np
    return (out != np.uint32(0xFFFFFFFF)) if trav == "sssp" else (out >= 0)


def algorithmic_bytes(V, vr, es, trav):
    """Bytes a work-efficient traversal must touch (per launch): init of the output array,
    per reached vertex its queue write+read, row offsets and result update, per scanned
    edge its column (+ weight) and the target's state."""
    return 4 * V + 24 * vr + 12 * es if trav == "sssp" else 4 * V + 20 * vr + 8 * es


def time_cpu_oracle(g, w, src, trav, budget_s=10.0, max_runs=8):
    """Time the oracle as it stands (one core), whole traversals until the budget is spent."""
    times, out = [], None
    t_start = time.perf_counter()
    while len(times) < max_runs and (len(times) == 0 or (time.perf_counter() - t_start) < budget_s):
        t0 = time.perf_counter()
        out = oracle_run(g, w, src, trav)
        times.append(time.perf_counter() - t0)
    return out, times


def config_of(name, g, extra=None):
    kind, scale, seed, wseed, trav = WORKLOADS[name]
    c = {"workload": name, "graph": kind, "V": g.num_vertices, "E": g.num_edges, "traversal": trav}
    if kind == "rmat":
        c.update({"scale": scale, "edge_factor": 16, "abcd": [0.57, 0.19, 0.19, 0.05], "seed": seed})
        if wseed is not None:
            c.update({"weights": "uint32 U[1,255]", "weight_seed": wseed})
    else:
        c.update({"grid": f"{scale}x{scale}", "neighbourhood": 4})
    if extra:
        c.update(extra)
    return c


def measure(coop, ctx, dev, stream, flush, name, steps, warmup, world=1, cpu_budget=None, clocks=None):
    """One workload's figures: device-timed GTEPS over `steps` traversals (L2 flushed
    between them, inputs resident), the persistent kernel's roofline, the end-to-end rate
    through the C ABI with the inputs copied from pinned host memory and the result copied
    back inside the timed region, parity of the last timed step's output against the
    oracle, and (cpu_budget given) the oracle timed on one host core.  `clocks` (a
    ClockSampler) samples the SM clock during the device-timed steps."""
    import contextlib
    import numpy as np
    import torch
    g, w, src, trav = load_workload(name)
    V, E = g.num_vertices, g.num_edges
    ro_h = torch.from_numpy(np.array(g.row_off)).pin_memory()
    col_h = torch.from_numpy(np.array(g.col)).pin_memory()
    w_h = torch.from_numpy(w.view(np.int32)).pin_memory() if w is not None else None
    ro, col = ro_h.to(dev), col_h.to(dev)
    wt = w_h.to(dev) if w_h is not None else None
    out_d = torch.empty(V, dtype=torch.int32, device=dev)
    out_h = torch.empty(V, dtype=torch.int32).pin_memory()
    csr = coop.make_csr(ro, col)
    threads = coop.coop_query(ctx)["threads_per_cta"]

    if trav == "sssp":
        def step():
            coop.coop_sssp(ctx, csr, wt, src, out_d, stream=stream)
    else:
        def step():
            coop.coop_bfs(ctx, csr, src, out_d, stream=stream)

    def result():
        r = out_d.cpu().numpy()
        return r.view(np.uint32) if trav == "sssp" else r

    for _ in range(warmup):
        step()
    stream.synchronize()
    st = coop.coop_get_stats(ctx)
    vr, es = reached_work(g, reached_of(result(), trav))
    out_d.fill_(-2)  # the timed steps must write every element again
    torch.cuda.synchronize(dev)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize(dev)
    step_ms, kern_us = [], []
    with (clocks if clocks is not None else contextlib.nullcontext()):
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_us.append(coop.coop_get_stats(ctx).kernel_us)
    torch.cuda.synchronize(dev)
    last = result()  # the last timed step's output, checked against the oracle below
    t_step = job_time(statistics.mean(step_ms) / 1e3, world, dev)
    value = whole_job_rate(es, world, t_step)

    # roofline of the dominant kernel (the persistent traversal kernel)
    hbm, peak_kind = peaks()
    B = algorithmic_bytes(V, vr, es, trav)
    k_s = statistics.mean(kern_us) / 1e6
    achieved = B / k_s / 1e9
    traffic = None
    tr = TRAFFIC.get(name)
    if tr and tr.get("sources_sha") == sources_sha():
        traffic = tr["bytes"]

    # end to end through the C ABI with host buffers: H2D inputs, traversal, D2H result
    h2d = (V + 1) * 4 + E * 4 + (E * 4 if wt is not None else 0)
    d2h = V * 4
    e2e_ms = []
    for i in range(warmup + steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        with torch.cuda.stream(stream):
            ro.copy_(ro_h, non_blocking=True)
            col.copy_(col_h, non_blocking=True)
            if wt is not None:
                wt.copy_(w_h, non_blocking=True)
        step()
        with torch.cuda.stream(stream):
            out_h.copy_(out_d, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_val = whole_job_rate(es, world, job_time(statistics.mean(e2e_ms) / 1e3, world, dev))
    e2e_out = out_h.numpy().view(np.uint32) if trav == "sssp" else out_h.numpy()

    res = {
        "value": round(value, 4), "ms_per_step": round(t_step * 1e3, 4),
        "dtype": "u32" if trav == "sssp" else "int32",
        "config": config_of(name, g, {
            "V_reached": vr, "E_s": es, "source": src, "parallelism": "replicas",
            "l2": "flushed between steps (512 MB write)", "ctas": st.max_active, "threads_per_cta": threads}),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": f"coop_traverse<{trav.upper()}>", "kernel_us": round(k_s * 1e6, 2),
                     "algorithmic_bytes": B},
        "e2e": {"value": round(e2e_val, 4), "unit": "GTEPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "stats": {"levels": st.levels, "barriers": st.barriers, "frontier_total": st.frontier_total,
                  "edges_expanded": st.edges_scanned, "work_inflation": round(st.edges_scanned / max(es, 1), 3)},
    }
    ref = None
    if cpu_budget is not None:
        ref, times = time_cpu_oracle(g, w, src, trav, budget_s=cpu_budget)
        res["parity_last_step"] = bool(np.array_equal(ref, last)) and bool(np.array_equal(ref, e2e_out))
        algo = "binary-heap Dijkstra" if trav == "sssp" else "FIFO-queue BFS"
        res["cpu_baseline"] = {
            "value": round(es / statistics.mean(times) / 1e9, 6), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} full {algo} traversal(s) of the {name} workload on 1 host core "
                      f"({os.cpu_count()} cores present)"}
    res["_graph"] = (g, src, ro, col, csr, ref)  # reused by the secondary figures on the same graph
    return res


def job_time(t_local: float, world: int, device) -> float:
    """Seconds of the whole job: the slowest rank's time (MAX all-reduce, then a barrier)."""
    if world <= 1:
        return t_local
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(tt.item())


def whole_job_rate(units_per_rank: int, world: int, t_job: float) -> float:
    """G-units per second of the whole job: every rank processes its own replica."""
    return units_per_rank * world / t_job / 1e9


def run_reference(args):
    """--impl reference: the CPU oracle on the same workload (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g, w, src, trav = load_workload(args.workload)
    for _ in range(args.warmup):
        oracle_run(g, w, src, trav)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = oracle_run(g, w, src, trav)
        times.append(time.perf_counter() - t0)
    _, es = reached_work(g, reached_of(out, trav))
    t = statistics.mean(times)
    val = es / t / 1e9
    algo = "binary-heap Dijkstra" if trav == "sssp" else "FIFO-queue BFS"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 6), "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if trav == "sssp" else "int32", "data": "synthetic",
        "config": config_of(args.workload, g, {"source": src}),
        "cpu_baseline": {"value": round(val, 6), "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full {algo} traversals of the {args.workload} workload"},
        "e2e": {"value": round(val, 6), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--extras", default="all",
                    help="comma-separated secondary figures to run (default all): " + ", ".join(EXTRAS))
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--threads", type=int, default=0, help="worker threads per CTA (0 = library default)")
    args = ap.parse_args()
    selected_extras(args.extras)  # an unknown name fails before any work
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1707_01989_gb300 as coop

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    args.warmup = max(3, args.warmup)

    ctx = coop.coop_init(local, 0, args.threads)
    coop.coop_set_timing(ctx, True)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    clocks = ClockSampler(local)
    m = measure(coop, ctx, dev, stream, flush, args.workload, args.steps, args.warmup, world,
                args.cpu_budget if rank == 0 else None, clocks)
    if rank == 0:
        extras = {}
        if not args.no_extras:
            extras = secondary(coop, ctx, dev, stream, flush, args, m)
        extras["parity_vs_oracle"] = m["parity_last_step"]
        line = {
            "metric": METRIC, "value": m["value"], "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": m["dtype"], "data": "synthetic",
            "config": m["config"], "roofline": m["roofline"], "e2e": m["e2e"],
            "gpu_launches": 2 * args.steps, "clocks": clocks.summary(), "cpu_baseline": m["cpu_baseline"],
            "stats": m["stats"], "extras": extras,
        }
        print(json.dumps(line), flush=True)
    m.pop("_graph", None)
    coop.coop_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()
    return 0


def random_schedules(coop, ctx, csr, src, lv, ref, stream, es, seeds=(0, 1, 2, 3), p_kill=0.5, p_fork=1.0):
    """R-MAT 22 BFS under seeded random kill/fork schedules: bit-exact flag and throughput.
    With these probabilities every seed both kills and forks within the graph's five
    resizing barriers."""
    import numpy as np
    res = []
    for seed in seeds:
        coop.coop_set_schedule(ctx, seed, p_kill, p_fork)
        t0 = time.perf_counter()
        st = coop.coop_bfs(ctx, csr, src, lv, stream=stream, stats=True)
        dt = time.perf_counter() - t0
        res.append({"seed": seed, "bit_exact": bool(np.array_equal(lv.cpu().numpy(), ref)), "kills": st.kills,
                    "forks": st.forks, "joined": st.joined, "min_active": st.min_active,
                    "kernel_us": round(st.kernel_us, 1),
                    "gteps_kernel": round(es / (st.kernel_us / 1e6) / 1e9, 2), "host_ms": round(dt * 1e3, 2)})
    coop.coop_set_schedule(ctx, 0, 0.0, 0.0)
    return res


class gil_handover:
    """The co-runner's host thread and the thread launching traversals share one Python
    interpreter; a thread coming back from a library call waits for the other to give up
    the interpreter lock, by default up to 5 ms.  While a co-runner is timed the hand-over
    interval is 10 us, so that the latency measured is the system's, not the harness's
    (a co-runner in its own process or native thread has no such wait)."""

    def __enter__(self):
        self.old = sys.getswitchinterval()
        sys.setswitchinterval(1e-5)

    def __exit__(self, *exc):
        sys.setswitchinterval(self.old)


def corunner(coop, ctx, dev, csr, src, lv, stream, period_s=1.0 / 60.0, duration_s=6.0, work=None, n_solo=360):
    """Cooperative multitasking: a periodic fp32 saxpy over 64 MB (x and y, 16.7 ms period)
    that claims half the SMs from back-to-back R-MAT 22 BFS traversals.

    Latency of one co-runner job = host time from coop_request_resources (the gather) to
    the saxpy's completion; solo = the same path with no traversal in flight.  The
    traversals' throughput with and without the co-runner gives the cooperative kernel's
    slowdown (the analogue of the paper's Sec. 5.4 measurements)."""
    import torch
    N = coop.coop_query(ctx)["max_ctas"]
    half = N // 2
    n_el = 16 * 1024 * 1024
    x = torch.rand(n_el, device=dev)
    y = torch.rand(n_el, device=dev)
    cs = torch.cuda.Stream(device=dev, priority=-1)
    for _ in range(3):
        coop.coop_saxpy(half, 2.0, x, y, stream=cs)
    cs.synchronize()

    def job():
        t0 = time.perf_counter()
        got = coop.coop_request_resources(ctx, half, timeout_us=2_000_000)
        t1 = time.perf_counter()
        coop.coop_saxpy(half, 2.0, x, y, stream=cs)
        cs.synchronize()
        t2 = time.perf_counter()
        coop.coop_release(ctx, got)
        return (t2 - t0) * 1e3, (t1 - t0) * 1e3

    solo = [job()[0] for _ in range(n_solo)]  # as many as the co-run's jobs: the same p99 estimator
    # solo with x and y out of L2 (a 512 MB write before each job, not timed): the state a
    # co-run job finds them in, since the traversals stream the 278 MB graph through L2
    wipe = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    solo_cold = []
    for _ in range(n_solo // 4):
        wipe.zero_()
        torch.cuda.synchronize(dev)
        solo_cold.append(job()[0])
    del wipe
    # traversal throughput alone
    coop.coop_bfs(ctx, csr, src, lv, stream=stream)
    stream.synchronize()
    t0 = time.perf_counter()
    n_alone = 0
    while time.perf_counter() - t0 < 0.5:
        coop.coop_bfs(ctx, csr, src, lv, stream=stream)
        n_alone += 1
    stream.synchronize()
    per_alone = (time.perf_counter() - t0) / n_alone
    # traversals back to back while the co-runner ticks every period
    lat, gat = [], []
    missed = [0]
    stop = threading.Event()

    def ticker():
        # frame-paced: a job starts on a tick of the period; one that overruns its period
        # skips the ticks it missed (no catch-up burst of back-to-back jobs)
        nxt = time.perf_counter()
        while not stop.is_set():
            l, g = job()
            lat.append(l)
            gat.append(g)
            nxt += period_s
            now = time.perf_counter()
            while nxt < now:
                nxt += period_s
                missed[0] += 1
            time.sleep(max(0.0, nxt - now))

    th = threading.Thread(target=ticker)
    coop.coop_get_request_log(ctx, clear=True)
    with gil_handover():
        t0, c0 = time.perf_counter(), time.process_time()
        th.start()
        n_co = 0
        while time.perf_counter() - t0 < duration_s:
            coop.coop_bfs(ctx, csr, src, lv, stream=stream)
            n_co += 1
        stream.synchronize()
        per_co = (time.perf_counter() - t0) / n_co
        stop.set()
        th.join()
        cores = (time.process_time() - c0) / (time.perf_counter() - t0)
    coop.coop_sync(ctx)
    reqs = coop.coop_get_request_log(ctx, clear=True)
    slowest = sorted(reqs, key=lambda r: -r["gather_us"])[:3]
    dev_gather = [r["gather_us"] / 1e3 for r in reqs]
    run = [l - g for l, g in zip(lat, gat)]

    def pct(v, q):
        v = sorted(v)
        return round(v[min(len(v) - 1, int(round(q * (len(v) - 1))))], 4)

    return {"period_ms": round(period_s * 1e3, 2), "claimed_ctas": half, "of_ctas": N, "jobs": len(lat),
            "ticks_missed": missed[0],
            "latency_ms_p50": pct(lat, 0.5), "latency_ms_p99": pct(lat, 0.99),
            "solo_ms_p50": pct(solo, 0.5), "solo_ms_p99": pct(solo, 0.99),
            "p99_vs_solo": round(pct(lat, 0.99) / pct(solo, 0.99), 3),
            "solo_cold_ms_p50": pct(solo_cold, 0.5), "solo_cold_ms_p99": pct(solo_cold, 0.99),
            "p99_vs_solo_cold": round(pct(lat, 0.99) / pct(solo_cold, 0.99), 3),
            "gather_ms_p50": pct(gat, 0.5), "gather_ms_p99": pct(gat, 0.99),
            # the library's own clock around the gather (no interpreter), and the rest of a
            # job: the saxpy on the lent SMs beside the traversal, launch and synchronise
            "gather_ms_lib_p50": pct(dev_gather or [0.0], 0.5), "gather_ms_lib_p99": pct(dev_gather or [0.0], 0.99),
            "run_ms_p50": pct(run, 0.5), "run_ms_p99": pct(run, 0.99),
            "deadline_ms": 2.0, "deadline_met_frac": round(sum(l <= 2.0 for l in lat) / max(1, len(lat)), 4),
            "host_cores_busy": round(cores, 2),  # this process's CPU time / wall time while co-running
            "traversal_ms_alone": round(per_alone * 1e3, 4), "traversal_ms_corun": round(per_co * 1e3, 4),
            "coop_slowdown": round(per_co / per_alone, 4),
            # per-request records of the three slowest gathers: M when posted and granted
            "slowest_gathers": [{k: round(v, 1) for k, v in r.items()} for r in slowest],
            **({} if work is None else {
                # host-timed back-to-back traversals (launch gaps included)
                "gteps_alone": round(work[0] / per_alone / 1e9, 3), "gteps_corun": round(work[0] / per_co / 1e9, 3),
                "hbm_frac_alone": round(work[1] / per_alone / 1e9 / work[2], 4),
                "hbm_frac_corun": round(work[1] / per_co / 1e9 / work[2], 4)})}


def preemption(coop, ctx, dev, stream, period_s=1.0 / 60.0, duration_s=1.0):
    """Co-runner latency with and without cooperation, on back-to-back 256x256 grid BFS
    traversals (about 3 ms each, 511 resizing barriers).

    Without cooperation (the non-cooperative baseline kernel, the co-runner only on a
    high-priority stream) the co-runner's CTAs start when a traversal ends and frees its
    SMs: CTAs are not preempted.  With cooperation the co-runner asks for half the CTAs
    (coop_request_resources), the traversal gives them up at its next kill point, and
    the co-runner runs beside it.  Latency = host time from the co-runner's request (or
    launch) to its completion; solo = the same with no traversal in flight."""
    import numpy as np
    import torch
    import graphgen as gg
    g = gg.grid(256, 256)
    ro = torch.from_numpy(np.array(g.row_off)).to(dev)
    col = torch.from_numpy(np.array(g.col)).to(dev)
    lv = torch.empty(g.num_vertices, dtype=torch.int32, device=dev)
    csr = coop.make_csr(ro, col)
    N = coop.coop_query(ctx)["max_ctas"]
    half = N // 2
    n_el = 16 * 1024 * 1024
    x = torch.rand(n_el, device=dev)
    y = torch.rand(n_el, device=dev)
    cs = torch.cuda.Stream(device=dev, priority=-1)
    for _ in range(3):
        coop.coop_saxpy(half, 2.0, x, y, stream=cs)
    cs.synchronize()

    def plain_job():
        t0 = time.perf_counter()
        coop.coop_saxpy(half, 2.0, x, y, stream=cs)
        cs.synchronize()
        return (time.perf_counter() - t0) * 1e3

    def coop_job():
        t0 = time.perf_counter()
        got = coop.coop_request_resources(ctx, half, timeout_us=2_000_000)
        coop.coop_saxpy(half, 2.0, x, y, stream=cs)
        cs.synchronize()
        t1 = time.perf_counter()
        coop.coop_release(ctx, got)
        return (t1 - t0) * 1e3

    def run(traverse, job):
        lat = []
        stop = threading.Event()

        def ticker():
            nxt = time.perf_counter()
            while not stop.is_set():
                lat.append(job())
                nxt += period_s
                time.sleep(max(0.0, nxt - time.perf_counter()))

        traverse()
        stream.synchronize()
        th = threading.Thread(target=ticker)
        t0 = time.perf_counter()
        th.start()
        n = 0
        while time.perf_counter() - t0 < duration_s:
            traverse()
            n += 1
        stream.synchronize()
        per = (time.perf_counter() - t0) / n
        stop.set()
        th.join()
        return lat, per

    def pct(v, q):
        v = sorted(v)
        return round(v[min(len(v) - 1, int(round(q * (len(v) - 1))))], 4)

    solo = [plain_job() for _ in range(30)]
    lat_plain, per_plain = run(lambda: coop.coop_bfs_baseline(ctx, csr, 0, lv, stream=stream), plain_job)
    lat_coop, per_coop = run(lambda: coop.coop_bfs(ctx, csr, 0, lv, stream=stream), coop_job)
    coop.coop_sync(ctx)
    return {"graph": "grid 256x256 BFS, back to back", "period_ms": round(period_s * 1e3, 2), "claimed_ctas": half,
            "solo_ms_p50": pct(solo, 0.5), "solo_ms_p99": pct(solo, 0.99),
            "no_coop": {"jobs": len(lat_plain), "latency_ms_p50": pct(lat_plain, 0.5),
                        "latency_ms_p99": pct(lat_plain, 0.99), "traversal_ms": round(per_plain * 1e3, 4)},
            "coop": {"jobs": len(lat_coop), "latency_ms_p50": pct(lat_coop, 0.5),
                     "latency_ms_p99": pct(lat_coop, 0.99), "traversal_ms": round(per_coop * 1e3, 4)},
            "p99_no_coop_vs_coop": round(pct(lat_plain, 0.99) / pct(lat_coop, 0.99), 3)}


# The graphics workload classes of Sec. 5.5's Table 3: period P, duration E (ms) and the
# share of the CTAs the non-cooperative task claims.
TABLE3_CLASSES = (("light", 70.0, 3.0, 4), ("medium", 40.0, 3.0, 4), ("heavy", 40.0, 10.0, 2))


def table3(coop, ctx, dev, stream, csr, src, lv, ref, duration_s=1.0, classes=TABLE3_CLASSES):
    """Sec. 5.5 / Table 3: the cooperative kernel's slowdown under periodic
    non-cooperative work, against kernel-level preemption.

    For each class (P, E, N/d) the non-cooperative task is a job of back-to-back saxpy
    launches on N/d CTAs sized to run E ms alone (its measured duration is D).  The
    cooperative kernel is back-to-back R-MAT 22 BFS traversals for `duration_s`; every P
    ms the task asks for N/d CTAs, runs, and gives them back.  Cooperative slowdown =
    traversal time with the task / without.  Non-cooperative: the baseline kernel
    (fixed CTAs, no scheduler) with the job on a high-priority stream -- its CTAs wait
    for a traversal to end and the next traversal cannot pass its first barrier until the
    job is done, so the compute kernel is effectively preempted for D every P; the model
    of the paper for that is P / (P - D).  Each run's last levels are checked against the
    oracle."""
    import numpy as np
    import torch
    N = coop.coop_query(ctx)["max_ctas"]
    n_el = 16 * 1024 * 1024
    x = torch.rand(n_el, device=dev)
    y = torch.rand(n_el, device=dev)
    cs = torch.cuda.Stream(device=dev, priority=-1)
    trav_coop = lambda: coop.coop_bfs(ctx, csr, src, lv, stream=stream)
    trav_plain = lambda: coop.coop_bfs_baseline(ctx, csr, src, lv, stream=stream)

    def job_alone(k, reps):
        t0 = time.perf_counter()
        for _ in range(reps):
            coop.coop_saxpy(k, 2.0, x, y, stream=cs)
        cs.synchronize()
        return (time.perf_counter() - t0) * 1e3

    def rate(traverse, secs):
        traverse()
        stream.synchronize()
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < secs:
            traverse()
            n += 1
        stream.synchronize()
        return (time.perf_counter() - t0) / n

    def corun(traverse, job, period_ms):
        lat, starts = [], []
        stop = threading.Event()

        def ticker():
            nxt = time.perf_counter()
            while not stop.is_set():
                starts.append(time.perf_counter())
                lat.append(job())
                nxt += period_ms / 1e3
                time.sleep(max(0.0, nxt - time.perf_counter()))

        traverse()
        stream.synchronize()
        th = threading.Thread(target=ticker)
        t0 = time.perf_counter()
        th.start()
        n = 0
        while time.perf_counter() - t0 < duration_s:
            traverse()
            n += 1
        stream.synchronize()
        per = (time.perf_counter() - t0) / n
        stop.set()
        th.join()
        exact = bool(np.array_equal(lv.cpu().numpy(), ref))
        gaps = np.diff(starts) * 1e3 if len(starts) > 1 else np.array([0.0])
        return per, lat, float(np.median(gaps)), exact

    def pct(v, q):
        v = sorted(v)
        return round(v[min(len(v) - 1, int(round(q * (len(v) - 1))))], 3)

    alone_coop = rate(trav_coop, 0.4)
    alone_plain = rate(trav_plain, 0.4)
    coop.coop_sync(ctx)
    rows = []
    for name, P, E, d in classes:
        k = N // d
        one = statistics.median(job_alone(k, 1) for _ in range(5))
        reps = max(1, int(round(E / max(one, 1e-3))))
        D = statistics.median(job_alone(k, reps) for _ in range(5))

        gather = []

        def coop_job():
            t0 = time.perf_counter()
            got = coop.coop_request_resources(ctx, k, timeout_us=2_000_000)
            gather.append((time.perf_counter() - t0) * 1e3)
            for _ in range(reps):
                coop.coop_saxpy(k, 2.0, x, y, stream=cs)
            cs.synchronize()
            t1 = time.perf_counter()
            coop.coop_release(ctx, got)
            return (t1 - t0) * 1e3

        def plain_job():
            return job_alone(k, reps)

        coop.coop_get_request_log(ctx, clear=True)
        per_c, lat_c, per_task_c, ok_c = corun(trav_coop, coop_job, P)
        coop.coop_sync(ctx)
        reqs = coop.coop_get_request_log(ctx, clear=True)
        slowest = max(reqs, key=lambda r: r["gather_us"]) if reqs else {}
        per_p, lat_p, per_task_p, ok_p = corun(trav_plain, plain_job, P)
        rows.append({
            "class": name, "period_ms": P, "task_ms": round(D, 3), "task_ctas": k, "task_launches": reps,
            "model_P_over_P_minus_D": round(P / (P - D), 3),
            "coop_slowdown": round(per_c / alone_coop, 3), "no_coop_slowdown": round(per_p / alone_plain, 3),
            "coop_task_latency_ms_p50": pct(lat_c, 0.5), "coop_task_latency_ms_p99": pct(lat_c, 0.99),
            "coop_task_latency_ms_max": pct(lat_c, 1.0), "coop_gather_ms_max": pct(gather or [0.0], 1.0),
            "slowest_request": {kk: round(v, 1) for kk, v in slowest.items()},
            "no_coop_task_latency_ms_p99": pct(lat_p, 0.99),
            "coop_task_period_ms": round(per_task_c, 2), "no_coop_task_period_ms": round(per_task_p, 2),
            "coop_deadline_met_frac": round(sum(l <= P for l in lat_c) / max(1, len(lat_c)), 3),
            "tasks": len(lat_c), "bit_exact": ok_c and ok_p})
    return {"graph": "R-MAT 22 BFS, back to back", "traversal_ms_alone": round(alone_coop * 1e3, 4),
            "baseline_traversal_ms_alone": round(alone_plain * 1e3, 4), "classes": rows}


def occupancy_trace(coop, ctx, dev, stream, period_s=0.0005, runs=40):
    """SM occupancy over time: active CTAs M at every resizing barrier of one traversal
    while a co-runner takes half the CTAs (saxpy over 64 MB) every `period_s` and gives
    them back -- the kernel shrinking to N/2 and growing back.  Grid 256x256 BFS (511
    barriers, about 6 us apart) and R-MAT 22 BFS (6 barriers).  Returns, per graph, the
    traversal among `runs` back-to-back ones with the most resize events: its trace
    as (t_us, M_after) at the barriers where M changed, and the number of barriers spent
    at each M."""
    import numpy as np
    import torch
    import graphgen as gg
    N = coop.coop_query(ctx)["max_ctas"]
    half = N // 2
    x = torch.rand(16 << 20, device=dev)
    y = torch.rand(16 << 20, device=dev)
    cs = torch.cuda.Stream(device=dev, priority=-1)
    out = {}
    for name, g, src in (("grid256_bfs", gg.grid(256, 256), 0), ("rmat22_bfs", gg.rmat(22, 16, seed=22), None)):
        src = gg.max_out_degree_vertex(g) if src is None else src
        ro = torch.from_numpy(np.array(g.row_off)).to(dev)
        col = torch.from_numpy(np.array(g.col)).to(dev)
        lv = torch.empty(g.num_vertices, dtype=torch.int32, device=dev)
        csr = coop.make_csr(ro, col)
        stop = threading.Event()

        def ticker():
            nxt = time.perf_counter()
            while not stop.is_set():
                got = coop.coop_request_resources(ctx, half, timeout_us=2_000_000)
                coop.coop_saxpy(half, 2.0, x, y, stream=cs)
                cs.synchronize()
                coop.coop_release(ctx, got)
                nxt += period_s
                time.sleep(max(0.0, nxt - time.perf_counter()))

        th = threading.Thread(target=ticker)
        th.start()
        best = None
        try:
            for _ in range(runs):
                st = coop.coop_bfs(ctx, csr, src, lv, stream=stream, stats=True)
                log = coop.coop_get_resize_log(ctx)
                events = sum(1 for r in log if r[3] or r[4])
                if best is None or events > best[0]:
                    best = (events, log, st)
        finally:
            stop.set()
            th.join()
        coop.coop_sync(ctx)
        _, log, st = best
        trace, m = [], None
        for r in log:  # (barrier, t_us, M_before, k, W, M_after, spawned, edges)
            if m is None or r[5] != m:
                trace.append((r[1], r[5]))
                m = r[5]
        dwell = {}
        for r in log:
            dwell[r[5]] = dwell.get(r[5], 0) + 1
        out[name] = {"N": N, "barriers": st.barriers, "kills": st.kills, "forks": st.forks, "joined": st.joined,
                     "min_active": st.min_active, "kernel_us": round(st.kernel_us, 1),
                     "trace_t_us_M": trace[:200], "barriers_at_M": dict(sorted(dwell.items()))}
        del ro, col, lv
    return out


def gather_by_kill_mode(coop, ctx, dev, stream, period_s=0.005, duration_s=0.6):
    """Gather time -- coop_request_resources(half the CTAs) until granted -- under each
    kill mode, on back-to-back traversals of R-MAT 22 BFS (6 wide levels) and of the
    256x256 grid BFS (511 narrow levels): the regular versus query barrier comparison of
    Sec. 5.4 ("Responsiveness"), plus the query barrier with kill points between chunks."""
    import numpy as np
    import torch
    import graphgen as gg
    N = coop.coop_query(ctx)["max_ctas"]
    half = N // 2
    modes = (("simple", coop.COOP_KILL_SIMPLE), ("query", coop.COOP_KILL_QUERY), ("chunk", coop.COOP_KILL_CHUNK))
    out = {}
    for gname, g, src in (("rmat22_bfs", gg.rmat(22, 16, seed=22), None), ("grid256_bfs", gg.grid(256, 256), 0)):
        src = gg.max_out_degree_vertex(g) if src is None else src
        ro = torch.from_numpy(np.array(g.row_off)).to(dev)
        col = torch.from_numpy(np.array(g.col)).to(dev)
        lv = torch.empty(g.num_vertices, dtype=torch.int32, device=dev)
        csr = coop.make_csr(ro, col)
        res = {}
        for mname, m in modes:
            coop.coop_set_kill_mode(ctx, m)
            gat = []
            stop = threading.Event()

            def ticker():
                nxt = time.perf_counter()
                while not stop.is_set():
                    t0 = time.perf_counter()
                    got = coop.coop_request_resources(ctx, half, timeout_us=2_000_000)
                    gat.append((time.perf_counter() - t0) * 1e3)
                    coop.coop_release(ctx, got)
                    nxt += period_s
                    time.sleep(max(0.0, nxt - time.perf_counter()))

            coop.coop_bfs(ctx, csr, src, lv, stream=stream)
            stream.synchronize()
            th = threading.Thread(target=ticker)
            t0 = time.perf_counter()
            th.start()
            n = 0
            while time.perf_counter() - t0 < duration_s:
                coop.coop_bfs(ctx, csr, src, lv, stream=stream)
                n += 1
            stream.synchronize()
            stop.set()
            th.join()
            coop.coop_sync(ctx)
            g_ms = sorted(gat)
            q = lambda f: round(g_ms[min(len(g_ms) - 1, int(round(f * (len(g_ms) - 1))))], 4)
            res[mname] = {"requests": len(g_ms), "gather_ms_p50": q(0.5), "gather_ms_p99": q(0.99),
                          "gather_ms_max": round(g_ms[-1], 4), "traversal_ms": round(duration_s / n * 1e3, 4)}
        coop.coop_set_kill_mode(ctx, coop.COOP_KILL_CHUNK)
        out[gname] = res
        del ro, col, lv
    out["claimed_ctas"] = half
    return out


def topology_driven(coop, ctx, dev, stream, flush, reps=3):
    """Table 1's two SSSP formulations on the headline graph: p-sssp (topology-driven,
    three barriers per iteration, every vertex scanned each iteration) against the
    frontier SSSP of the headline number."""
    import numpy as np
    import torch
    g, w, src, _ = load_workload("rmat20-sssp")
    ro = torch.from_numpy(np.array(g.row_off)).to(dev)
    col = torch.from_numpy(np.array(g.col)).to(dev)
    wt = torch.from_numpy(w.view(np.int32)).to(dev)
    d = torch.empty(g.num_vertices, dtype=torch.int32, device=dev)
    csr = coop.make_csr(ro, col)
    out = {}
    for name, f in (("p_sssp", coop.coop_sssp_topo), ("frontier_sssp", coop.coop_sssp)):
        f(ctx, csr, wt, src, d, stream=stream)
        ks, st = [], None
        for _ in range(reps):
            flush.zero_()
            st = f(ctx, csr, wt, src, d, stream=stream, stats=True)
            ks.append(st.kernel_us)
        kus = statistics.median(ks)
        out[name] = {"kernel_us": round(kus, 2), "gteps": round(st.reached_edges / (kus / 1e6) / 1e9, 3),
                     "barriers": st.barriers, "edges_relaxed": st.edges_scanned}
    ref = oracle_run(g, w, src, "sssp")
    out["p_sssp_bit_exact"] = bool(np.array_equal(d.cpu().numpy().view(np.uint32), ref))
    return out


def octree(coop, ctx, dev, stream, flush, n=1 << 22, leaf_cap=32, reps=3):
    """The work-stealing application (Table 1 octree): build time of an octree over n
    clustered points alone, then with the host taking half the CTAs every 5 ms (gather
    time of the loop-head offer_kill), checked against the oracle."""
    import numpy as np
    import torch
    import graphgen as gg
    from oracle import octree as ot
    pts = gg.points(n, 90, "clustered")
    x, y, z = (torch.from_numpy(a.view(np.int32)).to(dev) for a in pts)
    code = torch.empty(n, dtype=torch.int64, device=dev)
    begin = torch.empty(n, dtype=torch.int32, device=dev)
    count = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    nl = torch.empty(1, dtype=torch.int32, device=dev)
    run = lambda st: coop.coop_octree(ctx, x, y, z, leaf_cap, 21, code, begin, count, perm, nl, stream=stream,
                                      stats=st)
    run(False)
    ks, st = [], None
    for _ in range(reps):
        flush.zero_()
        st = run(True)
        ks.append(st.kernel_us)
    kus = statistics.median(ks)
    k = int(nl.item())
    c, b, cnt, pm = (a.cpu().numpy() for a in (code[:k], begin[:k], count[:k], perm))
    got = np.zeros(n, dtype=np.uint64)
    for cc, bb, kk in zip(c.view(np.uint64), b, cnt):
        got[pm[bb:bb + kk]] = cc
    t0 = time.perf_counter()
    exp = ot.leaf_code_of_points(*pts, leaf_cap, 21)
    cpu_s = time.perf_counter() - t0
    out = {"points": n, "leaf_cap": leaf_cap, "leaves": k, "kernel_us": round(kus, 1),
           "mpoints_per_s": round(n / (kus / 1e6) / 1e6, 1), "tasks": st.frontier_total, "steals": st.edges_scanned,
           "points_moved": st.reached_edges, "bit_exact": bool(np.array_equal(got, exp)),
           "oracle_s_1core": round(cpu_s, 3)}
    # gather under the work-stealing loop's offer_kill
    N = coop.coop_query(ctx)["max_ctas"]
    gat = []
    stop = threading.Event()

    def ticker():
        nxt = time.perf_counter()
        while not stop.is_set():
            t0 = time.perf_counter()
            got_c = coop.coop_request_resources(ctx, N // 2, timeout_us=2_000_000)
            gat.append((time.perf_counter() - t0) * 1e3)
            coop.coop_release(ctx, got_c)
            nxt += 0.005
            time.sleep(max(0.0, nxt - time.perf_counter()))

    th = threading.Thread(target=ticker)
    t0 = time.perf_counter()
    th.start()
    runs = 0
    while time.perf_counter() - t0 < 0.6:
        run(False)
        runs += 1
    stream.synchronize()
    stop.set()
    th.join()
    coop.coop_sync(ctx)
    g = sorted(gat)
    out["under_requests"] = {"runs": runs, "build_ms": round(0.6 / runs * 1e3, 3), "requests": len(g),
                             "gather_ms_p50": round(g[len(g) // 2], 4), "gather_ms_p99": round(g[int(0.99 * (len(g) - 1))], 4)}
    return out


def batched(coop, ctx, dev, stream, flush, n_inst=64, seed=3, steps=5):
    """Batched form: 64 independent R-MAT instances (scales uniform in 12..20, edge factor
    16), a BFS and an SSSP job each, run as one autotuned, CUDA-graph-captured launch,
    against one launch per job (the same 128 traversals issued back to back)."""
    import numpy as np
    import torch
    import graphgen as gg
    import oracle
    rng = np.random.default_rng(seed)
    scales = rng.integers(12, 21, size=n_inst)
    keep, jobs, outs = [], [], []
    es_total, edges_total = 0, 0
    singles = []
    for i, sc in enumerate(scales):
        g = gg.rmat(int(sc), 16, seed=1000 + i)
        w = gg.weights(g, 2000 + i)
        src = gg.max_out_degree_vertex(g)
        ro = torch.from_numpy(np.array(g.row_off)).to(dev)
        col = torch.from_numpy(np.array(g.col)).to(dev)
        wt = torch.from_numpy(w.view(np.int32)).to(dev)
        lv = torch.empty(g.num_vertices, dtype=torch.int32, device=dev)
        dist = torch.empty(g.num_vertices, dtype=torch.int32, device=dev)
        csr = coop.make_csr(ro, col)
        keep += [ro, col, wt, lv, dist, csr]
        jobs += [coop.make_job(csr, src, lv), coop.make_job(csr, src, dist, wt)]
        outs.append((g, w, src, lv, dist))
        singles.append((csr, src, lv, wt, dist))
        edges_total += g.num_edges
    b = coop.coop_batch_create(ctx, jobs, keep)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ctas = coop.coop_batch_tune(b, stream)
    tune_s = time.perf_counter() - t0

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    run = lambda: coop.coop_batch_run(b, stream, use_graph=True)
    run()
    ms_batch = timed(run, steps)
    stats = coop.coop_batch_get_stats(b)

    def one_per_job():
        for csr, src, lv, wt, dist in singles:
            coop.coop_bfs(ctx, csr, src, lv, stream=stream)
            coop.coop_sssp(ctx, csr, wt, src, dist, stream=stream)

    one_per_job()
    ms_single = timed(one_per_job, max(2, steps // 2))
    # parity of the batched results (run once more, then compare every job)
    run()
    torch.cuda.synchronize(dev)
    exact, algo = 0, 0
    for g, w, src, lv, dist in outs:
        l = lv.cpu().numpy()
        d = dist.cpu().numpy().view(np.uint32)
        exact += int(np.array_equal(l, oracle.bfs(g, src))) + int(np.array_equal(d, oracle.dijkstra(g, w, src)))
        deg = np.diff(g.row_off.astype(np.int64))
        vr, es = int((l >= 0).sum()), int(deg[l >= 0].sum())
        es_total += es * 2  # BFS and SSSP reach the same vertices
        algo += algorithmic_bytes(g.num_vertices, vr, es, "bfs") + algorithmic_bytes(g.num_vertices, vr, es, "sssp")
    hbm, _ = peaks()
    return {"instances": int(n_inst), "jobs": len(jobs), "scales": [int(x) for x in scales],
            "edges_total": int(edges_total), "E_s_total": int(es_total),
            "batch_ms": round(ms_batch, 3), "one_launch_per_job_ms": round(ms_single, 3),
            "gteps_batched": round(es_total / (ms_batch / 1e3) / 1e9, 3),
            "gteps_one_per_job": round(es_total / (ms_single / 1e3) / 1e9, 3),
            "speedup": round(ms_single / ms_batch, 3), "graph_captured": True,
            # every job's algorithmic bytes over the batch's time, against the HBM peak
            "algorithmic_bytes": int(algo), "hbm_frac": round(algo / (ms_batch / 1e3) / 1e9 / hbm, 4),
            "tuned_ctas_total": int(sum(ctas)), "tune_s": round(tune_s, 2),
            "jobs_bit_exact": exact, "all_ok": all(s.status == 0 for s in stats)}


def serving(coop, dev, n_graphs=32, rate=200.0, duration_s=3.0, slots=4, budget=60 << 30):
    """Serving: a Poisson stream of BFS / SSSP queries (50/50, random sources) on 32
    device-resident R-MAT graphs of scales 14..21, admitted by the server under a 60 GB
    HBM budget, with the periodic saxpy co-runner taking half the SMs every 16.7 ms.
    Also the saturation throughput (every query submitted at once) with `slots` slots
    against one query at a time (a single slot: one launch per query)."""
    import numpy as np
    import torch
    import graphgen as gg
    import oracle
    rng_g, rng_a, rng_s = (np.random.default_rng(x) for x in (4, 5, 6))
    scales = rng_g.integers(14, 22, size=n_graphs)
    graphs = []
    for i, sc in enumerate(scales):
        g = gg.rmat(int(sc), 16, seed=3000 + i)
        w = gg.weights(g, 4000 + i)
        ro = torch.from_numpy(np.array(g.row_off)).to(dev)
        col = torch.from_numpy(np.array(g.col)).to(dev)
        wt = torch.from_numpy(w.view(np.int32)).to(dev)
        graphs.append((g, w, ro, col, wt, coop.make_csr(ro, col)))
    maxV = max(x[0].num_vertices for x in graphs)
    n_q = int(rate * duration_s)
    gaps = rng_a.exponential(1.0 / rate, size=n_q)
    qs = []
    for i in range(n_q):
        gi = int(rng_s.integers(0, n_graphs))
        qs.append((gi, coop.COOP_JOB_BFS if rng_s.random() < 0.5 else coop.COOP_JOB_SSSP,
                   int(rng_s.integers(0, graphs[gi][0].num_vertices))))
    outs = [torch.empty(maxV, dtype=torch.int32, device=dev) for _ in range(64)]

    def make_server(k):
        sv = coop.coop_server_create(dev.index or 0, slots=k, hbm_budget_bytes=budget)
        for g, w, ro, col, wt, csr in graphs:
            coop.coop_server_add_graph(sv, csr, wt)
        return sv

    # open loop: Poisson arrivals with the co-runner alongside
    sv = make_server(slots)
    N = coop.coop_query(coop.coop_init(dev.index or 0))["max_ctas"]
    x = torch.rand(16 * 1024 * 1024, device=dev)
    y = torch.rand(16 * 1024 * 1024, device=dev)
    cs = torch.cuda.Stream(device=dev, priority=-1)
    for _ in range(3):
        coop.coop_saxpy(N // 2, 2.0, x, y, stream=cs)
    cs.synchronize()
    lat_co, stop = [], threading.Event()

    def ticker():
        nxt = time.perf_counter()
        while not stop.is_set():
            t0 = time.perf_counter()
            coop.coop_server_request_resources(sv, N // 2, timeout_us=2000,
                                               ok=(coop.COOP_OK, coop.COOP_ETIMEOUT))
            coop.coop_saxpy(N // 2, 2.0, x, y, stream=cs)
            cs.synchronize()
            coop.coop_server_release(sv, N // 2)
            lat_co.append((time.perf_counter() - t0) * 1e3)
            nxt += 1.0 / 60.0
            time.sleep(max(0.0, nxt - time.perf_counter()))

    import collections
    pending, done = collections.deque(), []
    th = threading.Thread(target=ticker)
    th.start()
    t_start = time.perf_counter()
    due = t_start
    for i, (gi, kind, src) in enumerate(qs):
        due += gaps[i]
        time.sleep(max(0.0, due - time.perf_counter()))
        if len(pending) >= 48:  # output buffers are reused: at most 48 queries outstanding
            done.append(coop.coop_server_wait(sv, pending.popleft()[1]))
        pending.append((i, coop.coop_server_submit(sv, gi, kind, src, outs[i % 64])))
    while pending:
        done.append(coop.coop_server_wait(sv, pending.popleft()[1]))
    wall = time.perf_counter() - t_start
    stop.set()
    th.join()
    coop.coop_server_destroy(sv)
    lat = sorted(r.latency_us / 1e3 for r in done)
    es = sum(r.stats.reached_edges for r in done)
    # results of the mix equal the oracle (the last 8 queries, whose outputs are intact)
    exact = 0
    for i in range(max(0, n_q - 8), n_q):
        gi, kind, src = qs[i]
        g, w = graphs[gi][0], graphs[gi][1]
        got = outs[i % 64][: g.num_vertices].cpu().numpy()
        exp = oracle.bfs(g, src) if kind == coop.COOP_JOB_BFS else oracle.dijkstra(g, w, src).view(np.int32)
        exact += int(np.array_equal(got, exp))

    def pct(v, q):
        v = sorted(v)
        return round(v[min(len(v) - 1, int(round(q * (len(v) - 1))))], 4)

    # saturation: all queries at once, `slots` slots vs one slot
    def saturate(k):
        sv2 = make_server(k)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ts = [coop.coop_server_submit(sv2, gi, kind, src, outs[i]) for i, (gi, kind, src) in enumerate(qs[:64])]
        rs = [coop.coop_server_wait(sv2, t) for t in ts]
        dt = time.perf_counter() - t0
        coop.coop_server_destroy(sv2)
        return sum(r.stats.reached_edges for r in rs) / dt / 1e9, dt * 1e3

    g_multi, ms_multi = saturate(slots)
    g_one, ms_one = saturate(1)
    return {"graphs": n_graphs, "scales": [int(x) for x in scales], "queries": len(done), "rate_per_s": rate,
            "slots": slots, "hbm_budget_gb": budget >> 30, "wall_s": round(wall, 3),
            "latency_ms_p50": pct(lat, 0.5), "latency_ms_p99": pct(lat, 0.99),
            "gteps_open_loop": round(es / wall / 1e9, 3),
            "saturation_gteps": round(g_multi, 3), "saturation_ms": round(ms_multi, 2),
            "saturation_gteps_one_at_a_time": round(g_one, 3), "saturation_ms_one_at_a_time": round(ms_one, 2),
            "served_vs_one_at_a_time": round(g_multi / g_one, 3),
            "corunner_jobs": len(lat_co), "corunner_ms_p50": pct(lat_co, 0.5) if lat_co else None,
            "corunner_ms_p99": pct(lat_co, 0.99) if lat_co else None,
            "last_queries_bit_exact": f"{exact}/8",
            "all_ok": all(r.status == 0 for r in done)}


EXTRAS = ("sssp_rmat20", "bfs_rmat22", "corunner", "grid_bfs", "preemption", "gather_by_kill_mode", "occupancy_trace",
          "topology_driven_sssp", "octree", "batched", "serving", "barrier_us")


def selected_extras(spec: str):
    """The secondary figures named by --extras, in their fixed order ("all" = every one)."""
    if spec.strip() == "all":  # the co-runner alone is part of bfs_rmat22 already
        return tuple(x for x in EXTRAS if x != "corunner")
    names = [x.strip() for x in spec.split(",") if x.strip()]
    bad = [x for x in names if x not in EXTRAS]
    if bad:
        raise SystemExit(f"unknown --extras {bad}; choose from {', '.join(EXTRAS)}")
    return tuple(x for x in EXTRAS if x in names)


def secondary(coop, ctx, dev, stream, flush, args, head):
    """SSSP on R-MAT 20 (with its own roofline, e2e and oracle baseline), the R-MAT 22
    BFS's non-cooperative baseline ratio, kill/fork schedules and co-runner, grid BFS, the
    co-runner with and without cooperation, batching, serving and barrier latency.  Each
    part runs on its own: one that fails records its error under its key and the others
    still run.  `head` is the headline measurement (its graph is reused)."""
    import traceback
    import numpy as np
    import torch
    import graphgen as gg
    out = {}

    def guarded(name, fn, label=None):
        try:
            res = fn()
            if isinstance(res, dict) and name is None:
                out.update(res)
            else:
                out[name] = res
        except Exception as exc:  # recorded, so that the JSON line is still printed
            out[name or label] = {"error": f"{type(exc).__name__}: {exc}",
                                    "where": traceback.format_exc(limit=3).splitlines()[-3:]}
            try:
                torch.cuda.synchronize(dev)
                coop.coop_set_schedule(ctx, 0, 0.0, 0.0)
                coop.coop_set_kill_mode(ctx, coop.COOP_KILL_CHUNK)
            except Exception:
                pass

    def timed(fn, reps):
        ts, ks = [], []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            ks.append(coop.coop_get_stats(ctx).kernel_us)
        return statistics.median(ts), statistics.median(ks)

    hbm, _ = peaks()

    def sssp_rmat20():
        # frontier SSSP on R-MAT scale 20: the full set of figures of the headline
        m = measure(coop, ctx, dev, stream, flush, "rmat20-sssp", max(3, args.steps), args.warmup, 1,
                    min(args.cpu_budget, 10.0))
        m.pop("_graph", None)
        m["parity_vs_oracle"] = m.pop("parity_last_step")
        return m

    def rmat22_graph():
        ref = None
        if args.workload == "rmat22-bfs":
            g, src, ro, col, csr, ref = head["_graph"]
        else:
            g = gg.rmat(22, 16, seed=22)
            src = gg.max_out_degree_vertex(g)
            ro = torch.from_numpy(np.array(g.row_off)).to(dev)
            col = torch.from_numpy(np.array(g.col)).to(dev)
            csr = coop.make_csr(ro, col)
        if ref is None:
            ref = oracle_run(g, None, src, "bfs")
        return g, src, csr, ref

    def corunner_only():
        # the co-runner beside back-to-back R-MAT 22 BFS traversals, alone
        g, src, csr, ref = rmat22_graph()
        lv = torch.empty(g.num_vertices, dtype=torch.int32, device=dev)
        coop.coop_bfs(ctx, csr, src, lv, stream=stream)
        stream.synchronize()
        vr, es = reached_work(g, ref >= 0)
        B = 4 * g.num_vertices + 20 * vr + 8 * es
        with ClockSampler(dev.index or 0, every_ms=200) as ck:
            res = corunner(coop, ctx, dev, csr, src, lv, stream, work=(es, B, hbm))
        res["clocks"] = ck.summary()
        res["bit_exact"] = bool(np.array_equal(lv.cpu().numpy(), ref))
        return res

    def rmat22():
        # BFS on R-MAT scale 22: the non-cooperative baseline, schedules and the co-runner
        g, src, csr, ref = rmat22_graph()
        lv = torch.empty(g.num_vertices, dtype=torch.int32, device=dev)
        f = lambda: coop.coop_bfs(ctx, csr, src, lv, stream=stream)
        for _ in range(3):
            f()
        ms, kus = timed(f, max(3, args.steps))
        lvh = lv.cpu().numpy()
        assert np.array_equal(lvh, ref), "R-MAT 22 BFS levels differ from the oracle"
        vr, es = reached_work(g, lvh >= 0)
        B = 4 * g.num_vertices + 20 * vr + 8 * es
        fb = lambda: coop.coop_bfs_baseline(ctx, csr, src, lv, stream=stream)
        for _ in range(2):
            fb()
        msb, kusb = timed(fb, max(3, args.steps))
        res = {"bfs_rmat22": {"V": g.num_vertices, "E": g.num_edges, "E_s": es, "V_reached": vr,
                              "ms": round(ms, 4), "kernel_us": round(kus, 2),
                              "gteps": round(es / (ms / 1e3) / 1e9, 3), "hbm_frac": round(B / (kus / 1e6) / 1e9 / hbm, 4),
                              "baseline_kernel_us": round(kusb, 2), "coop_overhead": round(kus / kusb, 4)}}
        res["bfs_rmat22_schedules"] = random_schedules(coop, ctx, csr, src, lv, lvh, stream, es)
        # each with the clocks seen while it ran: a throttling episode shows up beside it
        with ClockSampler(dev.index or 0, every_ms=200) as ck:
            res["corunner"] = corunner(coop, ctx, dev, csr, src, lv, stream, work=(es, B, hbm))
        res["corunner"]["clocks"] = ck.summary()
        with ClockSampler(dev.index or 0, every_ms=200) as ck:
            res["table3"] = table3(coop, ctx, dev, stream, csr, src, lv, lvh)
        res["table3"]["clocks"] = ck.summary()
        return res

    def grid():
        # grid 256x256 BFS: barrier-latency bound
        g = gg.grid(256, 256)
        ro = torch.from_numpy(np.array(g.row_off)).to(dev)
        col = torch.from_numpy(np.array(g.col)).to(dev)
        lv = torch.empty(g.num_vertices, dtype=torch.int32, device=dev)
        csr = coop.make_csr(ro, col)
        f = lambda: coop.coop_bfs(ctx, csr, 0, lv, stream=stream)
        for _ in range(3):
            f()
        ms, kus = timed(f, max(3, args.steps))
        ok = bool(np.array_equal(lv.cpu().numpy(), np.add(*np.divmod(np.arange(65536), 256))))
        return {"levels": 511, "ms": round(ms, 4), "kernel_us": round(kus, 2), "us_per_level": round(kus / 511, 3),
                "closed_form_ok": ok}

    def barriers():
        # empty resizing barriers: at M = N, at M = N/2 (half the CTAs lent), and at M = N
        # with a forced schedule that kills or forks at about one barrier in eight
        n = 20000
        N = coop.coop_query(ctx)["max_ctas"]
        f = lambda: coop.coop_barrier_bench(ctx, n, stream=stream, stats=False)

        def per_barrier():
            f()
            _, kus = timed(f, 3)
            return round(kus / n, 4)

        res = {"barrier_us": per_barrier()}
        got = coop.coop_request_resources(ctx, N // 2)
        res["barrier_us_half"] = per_barrier()
        coop.coop_release(ctx, got)
        coop.coop_set_schedule(ctx, 7, p_kill=1.0 / 16, p_fork=1.0 / 16)
        us = per_barrier()
        st = coop.coop_get_stats(ctx)
        coop.coop_set_schedule(ctx, 0, 0.0, 0.0)
        res["barrier_us_resizing"] = {"us": us, "kills": st.kills, "forks": st.forks, "barriers": st.barriers,
                                      "min_active": st.min_active}
        return res

    parts = {
        "sssp_rmat20": lambda: guarded("sssp_rmat20", sssp_rmat20),
        "bfs_rmat22": lambda: guarded(None, rmat22, "bfs_rmat22"),
        "corunner": lambda: guarded("corunner", corunner_only),
        "grid_bfs": lambda: guarded("grid_bfs", grid),
        "preemption": lambda: guarded("preemption", lambda: preemption(coop, ctx, dev, stream)),
        "gather_by_kill_mode": lambda: guarded("gather_by_kill_mode", lambda: gather_by_kill_mode(coop, ctx, dev, stream)),
        "occupancy_trace": lambda: guarded("occupancy_trace", lambda: occupancy_trace(coop, ctx, dev, stream)),
        "topology_driven_sssp": lambda: guarded("topology_driven_sssp",
                                                lambda: topology_driven(coop, ctx, dev, stream, flush)),
        "octree": lambda: guarded("octree", lambda: octree(coop, ctx, dev, stream, flush)),
        "batched": lambda: guarded("batched", lambda: batched(coop, ctx, dev, stream, flush)),
        "serving": lambda: guarded("serving", lambda: serving(coop, dev)),
        "barrier_us": lambda: guarded(None, barriers, "barrier_us"),
    }
    assert tuple(parts) == EXTRAS
    for name in selected_extras(args.extras):
        parts[name]()
    return out


if __name__ == "__main__":
    sys.exit(main())
