"""Benchmark of the PDR sweep (Alg. 1 with the exact edge solver of Alg. 2) on one GB300.

Headline workload (the largest single-GPU configuration): the 100 x 100
bidirectional grid, n = 10,000, m = 39,600 arcs, K = 10,000 random OD pairs
with lognormal(1, 0.5) demands, capacities 1.1x the load of a seeded random
hop-shortest-path routing (seed 0).  The FP32 flows alone are 1.58 GB, far
above L2, so every sweep streams its rows from HBM.

One step = one call of pdr_solve from f = 0 that runs exactly S sweeps (the
stop rules stay armed but do not fire before S) plus the FP64 residual and
certificate evaluation: every row of the hot path.  The metric is
edge-commodity updates per second, m * K * S / step time.

Timing: W warm-up steps, then K timed steps, each bracketed by CUDA events on
the solver's stream, with a 256 MiB buffer overwritten between steps so every
step starts with a cold L2.  ``value`` has the inputs resident in HBM; ``e2e``
times the same step through the C ABI from pinned host buffers (pdr_create,
which copies the instance in, pdr_solve, and pdr_flows, which writes the
flows into a pinned host buffer).  ``roofline`` takes the dominant kernel's
mean launch along the S sweeps of one step (CUDA events around each launch)
and reconciles it with the sweep time inside the graph loop.

Beside the headline the line carries (rank 0, one GPU): the error of one
FP32 sweep against the FP64 oracle on sampled edges, the L2-resident
knn2500_k500 instance (reported against L2 traffic, not HBM), time to
residual 1e-6 and the residuals reached within a fixed budget, the batched
form against the single-instance form (256 uneven instances, and 256 small
ones), the differentiated form against the forward alone, and the oracle on
this host's cores.

Multi-GPU: the sweep does not shard (replicas only): under torchrun every rank
solves its own replica and ``value`` is the sum of the ranks' updates over the
slowest rank's time.

``--impl reference`` times the FP64 CPU oracle (the paper's algorithms,
unoptimised) on this host's cores on a bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PDR edge·commodity updates/s, time-to-residual 1e-6, % of HBM peak"
UNIT = "edge·commodity updates/s"
WORKLOADS = {
    "knn2500_k500": "knn2500_k500: n=2500, m=15000 (3-NN both ways), K=500, d~U{1..20}, u=1.2x routing load, seed 0",
    "grid100_k10000": "grid100_k10000: 100x100 grid, n=10000, m=39600, K=10000, d~lognormal(1,0.5), u=1.1x routing "
                      "load, seed 0",
    "digraph20k_k2000": "digraph20k_k2000: random digraph n=20000, out-degree 5, m=100000, K=2000, d~U{1..10}, "
                        "u=1.05x routing load, seed 0",
    "batch256": "batch256: 256 random out-degree-4 digraphs, n~U[100,5000], K~U[10,1000], d~U{1..10}, u=1.2x "
                "routing load (20% at 0.7x), seed 0",
}
ALGOS = {"eso": 0, "agd": 1, "gdm": 2, "ck": 3}  # ck: Alg. 1 with the capacity kept (Program (6))
DEFAULT_WORKLOAD = "grid100_k10000"
WORKLOAD = WORKLOADS[DEFAULT_WORKLOAD]
L2_RESIDENT_BYTES = 96 << 20  # working sets up to this stay in GB300's L2 across sweeps (measured)
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--sweeps", type=int, default=0, help="sweeps per step (default 2000 on knn2500_k500, else 200)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--algo", choices=sorted(ALGOS), default="eso",
                    help="eso: Alg. 1 + Alg. 2; agd: Alg. 3; gdm: Alg. 4")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the differentiated form (T = 50 sweeps, checkpoints every 10) on the workload")
    ap.add_argument("--compare-algos", action="store_true",
                    help="time Alg. 1, Alg. 3 and Alg. 4 on the workload and print one comparison line")
    ap.add_argument("--edge-variant", type=int, default=-1,
                    help="edge-kernel variant (index of the library's variant table; -1 = the library's choice)")
    ap.add_argument("--to-residual", action="store_true",
                    help="solve to the verdict (residuals <= 1e-6 or a Farkas certificate, FP32 with the FP64 "
                         "tail; --sweeps caps the sweeps); batch256: as one batch and one after another")
    ap.add_argument("--instances", type=int, default=256, help="batch256: number of instances")
    ap.add_argument("--compare-engines", action="store_true",
                    help="time the sweep-loop engines (host loop, CUDA graph, persistent kernel) on instances "
                         "from m = 80 to the bench workload and print one JSON line")
    ap.add_argument("--excess-variant", type=int, default=-1,
                    help="excess kernel form: -1 library default, 0 per-thread gathers, 1..5 bulk copies")
    ap.add_argument("--compare-excess", action="store_true",
                    help="time the excess kernel forms (alone, warm and cold L2) and the sweep loop with each")
    ap.add_argument("--compare-variants", action="store_true",
                    help="time every edge-kernel variant that holds the rows (Alg. 1) and print one JSON line")
    ap.add_argument("--impl", choices=["pdr", "reference"], default="pdr")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the roofline, oracle error, CPU baseline and the extra blocks")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched and differentiated-form blocks of the default run")
    ap.add_argument("--profile-sweeps", type=int, default=0,
                    help="profiler driver: run this many host-launched sweeps from f = 0 on the workload and exit")
    ap.add_argument("--engine", choices=["graph", "persistent"], default="graph",
                    help="sweep-loop engine of the solve (CUDA graph with a while node, or the persistent kernel)")
    ap.add_argument("--host-loop", action="store_true",
                    help="launch the sweep kernels from a host loop instead of the device-side graph loop "
                         "(same kernels; used for profiler runs)")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms while active."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- helpers


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def source_digest():
    """Digest of the sweep kernels' sources (the files the ncu counters depend on)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2108_07549_gb300", "csrc")
    for name in ("sweep.cu", "sweep_common.cuh", "pdr_internal.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the
    current sources and on this workload."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_digest") != source_digest() or rec.get("workload") != WORKLOAD.split(":")[0]:
        return None
    k = rec.get("kernels", {}).get(kernel)
    return None if k is None else float(k["dram_bytes_per_launch"])


def cpu_baseline(inst, budget_s=12.0, single_s=4.0):
    """The FP64 oracle (Alg. 1 + Alg. 2, unoptimised) on all host cores, on a
    bounded sample, and beside it on one core."""
    import oracle

    P = oracle.Problem.from_instance(inst)

    def timed(threads, budget):
        used = oracle.set_threads(threads)
        t0 = time.perf_counter()
        P.solve_eso(max_sweeps=1, eps_obj=0.0)
        per = time.perf_counter() - t0
        n_sweeps = int(budget / max(per, 1e-6))
        if n_sweeps <= 1:  # one sweep already fills the budget: that run is the sample
            return used, 1, per
        t0 = time.perf_counter()
        _, rep = P.solve_eso(max_sweeps=n_sweeps, eps_obj=0.0)
        dt = time.perf_counter() - t0
        return used, rep["sweeps"], dt

    threads, sweeps, dt = timed(os.cpu_count() or 1, budget_s)
    _, sweeps1, dt1 = timed(1, single_s)
    oracle.set_threads(1)
    return {"value": inst.m * inst.K * sweeps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{sweeps} FP64 sweeps of Alg. 1 (sort-based Alg. 2) from f = 0 on the same instance, "
                      f"{dt:.1f} s",
            "single_core": {"value": inst.m * inst.K * sweeps1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"{sweeps1} FP64 sweeps from f = 0, {dt1:.1f} s"}}


# --------------------------------------------------------------------------- reference arm


def run_reference(args, inst):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle

    threads = oracle.set_threads(os.cpu_count() or 1)
    P = oracle.Problem.from_instance(inst)
    t0 = time.perf_counter()
    P.solve_eso(max_sweeps=1, eps_obj=0.0)
    per = time.perf_counter() - t0
    # each step: a bounded sample of the workload, about 20 s for the whole
    # run (at least one sweep per step)
    total_steps = args.steps + args.warmup
    sweeps = max(1, int(20.0 / max(per, 1e-6) / max(total_steps, 1)))
    for _ in range(args.warmup):
        P.solve_eso(max_sweeps=sweeps, eps_obj=0.0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        P.solve_eso(max_sweeps=sweeps, eps_obj=0.0)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = inst.m * inst.K * sweeps / (ms / 1e3)
    sample = f"each step {sweeps} FP64 sweeps of Alg. 1 (sort-based Alg. 2) from f = 0"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sweeps_per_step": sweeps, "threads": threads},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def update_bytes(algo: str, inst) -> int:
    """Algorithmic bytes of one launch of the flow-update kernel (FP32).

    All: read f, write f', read h once (4K(2m + n)), tail/head/capacity per
    edge (12m).  Alg. 3 / Alg. 4 add the rates read and written (8m); Alg. 4
    adds the velocities read and written (8Km)."""
    m, n, K = inst.m, inst.n, inst.K
    b = 4 * K * (2 * m + n) + 12 * m
    if algo in ("agd", "gdm"):
        b += 8 * m
    if algo == "gdm":
        b += 8 * K * m
    return b


def compare_algos(args, inst, pdr, torch, stream):
    """Alg. 1 (ESO), Alg. 3 (AGD) and Alg. 4 (GDM) on the same instance: time
    per sweep (CUDA events around a fixed number of sweeps from f = 0), the
    objective reached, and each update kernel alone with a cold L2."""
    peak, peak_src = load_peaks()
    out = {"kind": "algorithm comparison", "workload": WORKLOAD, "sweeps": args.sweeps, "dtype": "f32",
           "peak_gbs": peak, "peak_source": peak_src, "algos": {}}
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for name, code in ALGOS.items():
        with torch.cuda.stream(stream):
            with pdr.Solver.from_instance(inst, stream=stream.cuda_stream, precision=pdr.PREC_FP32, algo=code,
                                          eps_obj=0.0, resid_tol=0.0, max_sweeps=args.sweeps) as sv:
                sv.solve()  # warm-up (graph capture, first touch)
                times = []
                for q in range(3):
                    sv.reset()
                    flush.fill_(q & 0xFF)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    r = sv.solve()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = sorted(times)[1]
                t_up = sv.time_kernel("qp", 10, FLUSH_BYTES)
                t_ex = sv.time_kernel("excess", 10, FLUSH_BYTES)
        b_up = update_bytes(name, inst)
        b_ex = 4 * inst.K * (inst.m + inst.n) + 8 * inst.m + 8 * inst.n
        out["algos"][name] = {
            "ms_per_sweep": ms / args.sweeps, "updates_per_s": inst.m * inst.K * args.sweeps / (ms / 1e3),
            "z_after": r["z"], "cons_rel_after": r["cons_rel"],
            "update_kernel_us_cold": t_up * 1e3, "update_gbs": b_up / (t_up / 1e3) / 1e9,
            "update_frac": b_up / (t_up / 1e3) / 1e9 / peak,
            "excess_kernel_us_cold": t_ex * 1e3, "excess_gbs": b_ex / (t_ex / 1e3) / 1e9,
            "excess_frac": b_ex / (t_ex / 1e3) / 1e9 / peak,
        }
    # the FP64 oracle of each algorithm on a bounded sample: one sweep from f = 0
    import oracle

    threads = oracle.set_threads(os.cpu_count() or 1)
    P = oracle.Problem.from_instance(inst)
    for name in ALGOS:
        t0 = time.perf_counter()
        if name == "eso":
            P.solve_eso(max_sweeps=1, eps_obj=0.0)
        elif name == "ck":
            P.solve_ck(max_sweeps=1, eps_obj=0.0)
        else:
            P.solve_gd(oracle.gd_params(name == "gdm", inst.K), max_sweeps=1, eps_obj=0.0)
        dt = time.perf_counter() - t0
        out["algos"][name]["cpu_baseline"] = {"value": inst.m * inst.K / dt, "unit": UNIT, "cores": threads,
                                              "kind": "oracle", "sample": f"1 FP64 sweep from f = 0, {dt:.2f} s"}
    oracle.set_threads(1)
    print(json.dumps(out), flush=True)


def compare_variants(args, inst, pdr, torch, stream):
    """Alg. 1 with each edge-kernel variant that holds the rows: time per
    sweep inside the graph loop (CUDA events around a fixed number of sweeps
    from f = 0) and the edge kernel alone with a cold L2."""
    peak, peak_src = load_peaks()
    out = {"kind": "edge-kernel variant comparison", "workload": WORKLOAD, "algo": args.algo, "sweeps": args.sweeps,
           "dtype": "f32", "peak_gbs": peak, "peak_source": peak_src, "variants": {}}
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    b_up = update_bytes(args.algo, inst)
    for v, cap, pipe in pdr.edge_variants(pdr.PREC_FP32):
        if cap < inst.K or (pipe and args.algo != "eso"):
            continue
        with torch.cuda.stream(stream):
            with pdr.Solver.from_instance(inst, stream=stream.cuda_stream, precision=pdr.PREC_FP32, eps_obj=0.0,
                                          resid_tol=0.0, max_sweeps=args.sweeps, edge_variant=v,
                                          algo=ALGOS[args.algo]) as sv:
                sv.solve()
                times = []
                for q in range(3):
                    sv.reset()
                    flush.fill_(q & 0xFF)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    r = sv.solve()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = sorted(times)[1]
                t_up = sv.time_kernel("qp", 10, FLUSH_BYTES)
        out["variants"][str(v)] = {
            "capacity": cap, "pipelined": pipe, "us_per_sweep": ms / args.sweeps * 1e3,
            "updates_per_s": inst.m * inst.K * args.sweeps / (ms / 1e3), "z_after": r["z"],
            "qp_kernel_us_cold": t_up * 1e3, "qp_frac": b_up / (t_up / 1e3) / 1e9 / peak,
        }
    print(json.dumps(out), flush=True)


def compare_excess(args, inst, pdr, torch, stream):
    """Alg. 1 in FP32 with each excess-kernel form: time per sweep inside the
    graph loop (CUDA events around a fixed number of sweeps from f = 0, the
    median of three) and the excess kernel alone, in the L2 state of the loop
    (warm) and with L2 flushed before every launch (cold)."""
    peak, peak_src = load_peaks()
    S = args.sweeps
    b_ex = 4 * inst.K * (inst.m + inst.n) + 8 * inst.m + 8 * inst.n
    out = {"kind": "excess-kernel form comparison", "workload": WORKLOAD, "sweeps": S, "dtype": "f32",
           "algorithmic_bytes": b_ex, "peak_gbs": peak, "peak_source": peak_src, "forms": {}}
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for form in (0, 1, 2, 3, 4, 5):
        with torch.cuda.stream(stream):
            with pdr.Solver.from_instance(inst, stream=stream.cuda_stream, precision=pdr.PREC_FP32, eps_obj=0.0,
                                          resid_tol=0.0, max_sweeps=S, excess_variant=form) as sv:
                sv.solve()
                times = []
                for q in range(3):
                    sv.reset()
                    flush.fill_(q & 0xFF)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    r = sv.solve()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = sorted(times)[1]
                t_w = sv.time_kernel("excess", 20, 0)
                t_c = sv.time_kernel("excess", 10, FLUSH_BYTES)
        out["forms"][str(form)] = {
            "us_per_sweep": ms / S * 1e3, "updates_per_s": inst.m * inst.K * S / (ms / 1e3), "z_after": r["z"],
            "excess_us_warm": t_w * 1e3, "excess_us_cold": t_c * 1e3,
            "frac_warm": b_ex / (t_w / 1e3) / 1e9 / peak, "frac_cold": b_ex / (t_c / 1e3) / 1e9 / peak,
        }
    print(json.dumps(out), flush=True)


def compare_engines(args, inst, pdr, torch, stream):
    """Alg. 1 in FP32 with each sweep-loop engine on instances of growing size
    (the last one the bench workload): microseconds per sweep of a solve of a
    fixed number of sweeps (CUDA events; the FP64 residual pass is included
    and is below 1 % of these solves)."""
    import numpy as np

    from paper_2108_07549_gb300 import instances as I

    rng = np.random.default_rng(0)
    cases = [I.grid5_k10(1.2),
             I.make_instance("digraph200_k50", I.random_digraph(200, 3, rng), 50, ("uniform_int", 1, 9), 1.1, rng),
             I.make_instance("knn500_k100", I.knn_graph(500, 3, rng), 100, ("uniform_int", 1, 20), 1.2, rng),
             I.make_instance("knn1000_k250", I.knn_graph(1000, 3, rng), 250, ("uniform_int", 1, 20), 1.2, rng),
             inst]
    S = args.sweeps
    out = {"kind": "sweep-loop engine comparison", "sweeps": S, "dtype": "f32", "us_per_sweep": {}}
    for c in cases:
        row = {"m": c.m, "K": c.K}
        for name, eng in (("host_loop", 0), ("graph", 1), ("persistent", 2), ("cluster", 3)):
            with torch.cuda.stream(stream):
                with pdr.Solver.from_instance(c, stream=stream.cuda_stream, precision=pdr.PREC_FP32, eps_obj=0.0,
                                              resid_tol=0.0, max_sweeps=S, use_graph=eng) as sv:
                    sv.solve()
                    times = []
                    for q in range(3):
                        sv.reset()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        sv.solve()
                        e1.record(stream)
                        torch.cuda.synchronize()
                        times.append(e0.elapsed_time(e1))
            row[name] = sorted(times)[1] * 1e3 / S
        out["us_per_sweep"][c.name] = row
    print(json.dumps(out), flush=True)


def time_reverse_mode(pdr, torch, stream, inst, T, ckpt):
    """The differentiated form through T sweeps: the forward sweeps alone,
    then forward + gradient with checkpoints every ckpt sweeps and with every
    sweep kept (ckpt_every = 1, nothing recomputed).  FP32, median of three,
    CUDA events on the solver's stream; one untimed call of each first (it
    also sizes the workspace the context keeps between calls)."""
    import numpy as np

    out = {"T": T, "ckpt_every": ckpt, "dtype": "f32"}
    peak, peak_src = load_peaks()
    with torch.cuda.stream(stream):
        with pdr.Solver.from_instance(inst, stream=stream.cuda_stream, precision=pdr.PREC_FP32) as sv:
            def timed(c, grads):
                sv.backward(T, c, grads=grads)
                times = []
                for _ in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    res = sv.backward(T, c, grads=grads)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                return sorted(times)[1], res

            out["forward_only_ms"], _ = timed(ckpt, False)
            for c, key in ((ckpt, None), (1, "ckpt_every_1")):
                ms, (L, gu, gd) = timed(c, True)
                extra_bytes = T * gradient_sweep_bytes(inst, keep_all=(c == 1))
                extra_ms = ms - out["forward_only_ms"]
                rec = {"forward_and_gradient_ms": ms, "gradient_over_forward": ms / out["forward_only_ms"],
                       "gradient_roofline": {"bound": "hbm", "algorithmic_bytes": extra_bytes, "ms": extra_ms,
                                             "achieved": extra_bytes / (extra_ms / 1e3) / 1e9, "peak": peak,
                                             "unit": "GB/s", "peak_source": peak_src,
                                             "frac": extra_bytes / (extra_ms / 1e3) / 1e9 / peak}}
                if key is None:
                    out.update(rec)
                    out["L"] = L
                    out["grad_u_norm"] = float(np.linalg.norm(gu))
                    out["grad_d_norm"] = float(np.linalg.norm(gd))
                    out["euler_identity_rel"] = float(abs(np.dot(inst.u, gu) + np.dot(inst.d, gd) - 2 * L) / (2 * L))
                    g_ref = (L, gu, gd)
                else:
                    rec["same_gradients_bitwise"] = bool(L == g_ref[0] and np.array_equal(gu, g_ref[1]) and
                                                         np.array_equal(gd, g_ref[2]))
                    out[key] = rec
    out["forward_updates_per_s"] = inst.m * inst.K * T / (out["forward_only_ms"] / 1e3)
    return out


def bench_adjoint(args, inst, pdr, torch, stream, T=50, ckpt=10):
    """The differentiated form (time_reverse_mode) on the chosen workload."""
    out = {"kind": "differentiated form", "workload": WORKLOAD}
    out.update(time_reverse_mode(pdr, torch, stream, inst, T, ckpt))
    out["cpu_baseline"] = adjoint_cpu_baseline(inst)
    print(json.dumps(out), flush=True)


def gradient_sweep_bytes(inst, keep_all: bool = False) -> int:
    """Algorithmic bytes of the gradient's extra work per unrolled sweep (FP32),
    each array counted once: the segment's forward sweep again (excess: f in,
    h out, 4K(m+n); edge QP: f, h in, f' out, 4K(2m+n); the heights are kept
    per sweep), the Jacobian step (f, h, dL/dc' and dL/dDelta' in, dL/dc out,
    4K(3m+2n); it forms dL/df from them) and the vertex gather (dL/dc in,
    dL/dDelta out, 4K(m+n)): 4K(7m+5n).  With every sweep kept (keep_all) the
    recomputation drops out: 4K(4m+3n)."""
    if keep_all:
        return 4 * inst.K * (4 * inst.m + 3 * inst.n)
    return 4 * inst.K * (7 * inst.m + 5 * inst.n)


def adjoint_cpu_baseline(inst, T=1):
    """The FP64 oracle's reverse mode (unoptimised) on a bounded sample: T
    sweeps forward and back on the same instance."""
    import oracle

    threads = oracle.set_threads(os.cpu_count() or 1)
    P = oracle.Problem.from_instance(inst)
    t0 = time.perf_counter()
    P.adjoint_eso(T)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return {"value": inst.m * inst.K * T / dt, "unit": "edge·commodity updates/s (forward + gradient)",
            "cores": threads, "kind": "oracle",
            "sample": f"reverse mode through {T} FP64 sweep(s) of Alg. 1 on the same instance, {dt:.1f} s"}


def solve_to_residual(args, inst, pdr, torch, stream):
    """One instance solved to its verdict: FP32 sweeps until they stall, then
    FP64 sweeps, until cap_rel and cons_rel <= 1e-6 (or the Farkas
    certificate holds, or the sweep cap).  Reports the time, the sweeps of
    each phase and the residuals reached."""
    max_sweeps = args.sweeps if args.sweeps > 0 else 2000000
    out = {"kind": "time to residual 1e-6", "workload": WORKLOAD, "max_sweeps": max_sweeps,
           "precision": "FP32 sweeps, FP64 tail, FP64 residuals and certificate", "algos": {}}
    for name in (["eso", "ck"] if args.algo == "eso" else [args.algo]):
        opts = dict(precision=pdr.PREC_FP32_FP64TAIL, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13,
                    max_sweeps=max_sweeps, algo=ALGOS[name])
        with torch.cuda.stream(stream):
            with pdr.Solver.from_instance(inst, stream=stream.cuda_stream, **opts) as sv:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = sv.solve()
                dt = time.perf_counter() - t0
        out["algos"][name] = {"s": dt, "sweeps": r["sweeps"], "sweeps_fp64": r["sweeps_fp64"],
                              "cap_rel": r["cap_rel"], "cons_rel": r["cons_rel"], "z": r["z"],
                              "verdict": r["verdict_name"], "stop": r["stop_name"]}
    print(json.dumps(out), flush=True)


def bench_batch_to_residual(args, insts, pdr, torch, stream):
    """The batched form against the single-instance form at residual <= 1e-6:
    every instance solved to its verdict (FP32 sweeps, then FP64 sweeps once
    FP32 stalls; stop when cap_rel and cons_rel <= 1e-6 or, for infeasible
    instances, when the Farkas certificate holds), (a) as one batch and (b)
    one after another.  Wall-clock time of each from f = 0, verdicts and
    residuals compared."""
    max_sweeps = args.sweeps if args.sweeps > 0 else 200000
    opts = dict(precision=pdr.PREC_FP32_FP64TAIL, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13, max_sweeps=max_sweeps)
    with torch.cuda.stream(stream):
        B = pdr.Batch(insts, stream=stream.cuda_stream, **opts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rb = B.solve()
        tb = time.perf_counter() - t0
        B.close()
        rs, ts = [], 0.0
        for x in insts:
            with pdr.Solver.from_instance(x, stream=stream.cuda_stream, **opts) as sv:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rs.append(sv.solve())
                ts += time.perf_counter() - t0
    want = [x.feasible_by_construction for x in insts]

    def summary(res):
        v = [r["verdict_name"] for r in res]
        feas = [r for r in res if r["verdict_name"] == "feasible"]
        return {"verdicts": {k: v.count(k) for k in sorted(set(v))},
                "sweeps_max": max(r["sweeps"] for r in res), "sweeps_sum": sum(r["sweeps"] for r in res),
                "max_cap_rel_feasible": max((r["cap_rel"] for r in feas), default=None),
                "max_cons_rel_feasible": max((r["cons_rel"] for r in feas), default=None),
                "verdicts_as_constructed": sum(
                    1 for r, w in zip(res, want)
                    if w is not None and r["verdict_name"] == ("feasible" if w else "infeasible"))}

    print(json.dumps({
        "kind": "batched form to residual 1e-6", "workload": WORKLOAD, "instances": len(insts),
        "precision": "FP32 sweeps, FP64 tail, FP64 residuals and certificate", "max_sweeps": max_sweeps,
        "batch": {"s": tb, **summary(rb)}, "single_form_sequential": {"s": ts, **summary(rs)},
        "speedup": ts / tb,
        "same_verdicts": all(a["verdict"] == b["verdict"] for a, b in zip(rb, rs)),
    }), flush=True)


def bench_batch(args, insts, pdr, torch, stream):
    """The batched form against the single-instance form on the same GPU: the
    same instances, the same S sweeps each (Alg. 1 + Alg. 2, FP32), solved
    (a) by one batch (one graph launch per solve) and (b) one after another,
    each by its own context (one graph launch per instance).  Both include
    the per-instance reset and FP64 residual pass."""
    import numpy as np

    S = args.sweeps
    opts = dict(precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=S)
    total = sum(x.m * x.K for x in insts) * S
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        B = pdr.Batch(insts, stream=stream.cuda_stream, **opts)
        t_create = time.perf_counter() - t0
        cfg, us = B.tuning()
        B.solve()
        bt = []
        for q in range(max(1, args.steps)):
            B.reset()
            flush.fill_(q & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = B.solve()
            bt.append(time.perf_counter() - t0)
        verdicts = [r["verdict_name"] for r in res]
        assert all(r["sweeps"] == S for r in res)
        B.close()
        singles = [pdr.Solver.from_instance(x, stream=stream.cuda_stream, **opts) for x in insts]
        for sv in singles:
            sv.solve()
        st = []
        for q in range(max(1, args.steps)):
            for sv in singles:
                sv.reset()
            flush.fill_(q & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for sv in singles:
                sv.solve()
            st.append(time.perf_counter() - t0)
        for sv in singles:
            sv.close()
    tb, ts = sorted(bt)[len(bt) // 2], sorted(st)[len(st) // 2]
    vals, counts = np.unique(cfg, return_counts=True)
    # the oracle on a bounded sample: 5 FP64 sweeps of the first 8 instances
    import oracle

    threads = oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    upd = 0
    for x in insts[:8]:
        oracle.Problem.from_instance(x).solve_eso(max_sweeps=5, eps_obj=0.0)
        upd += x.m * x.K * 5
    cpu = {"value": upd / (time.perf_counter() - t0), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": "5 FP64 sweeps of Alg. 1 on each of the first 8 instances"}
    oracle.set_threads(1)
    print(json.dumps({
        "kind": "batched form", "workload": WORKLOAD, "instances": len(insts), "sweeps_per_instance": S,
        "updates_per_solve": total, "dtype": "f32",
        "batch": {"s_per_solve": tb, "updates_per_s": total / tb, "create_and_autotune_s": t_create},
        "single_form_sequential": {"s_per_solve": ts, "updates_per_s": total / ts},
        "speedup": ts / tb,
        "autotuner_variants": {str(int(v)): int(c) for v, c in zip(vals, counts)},
        "verdicts_after_S": {v: verdicts.count(v) for v in sorted(set(verdicts))},
        "cpu_baseline": cpu,
    }), flush=True)


# --------------------------------------------------------------------------- blocks of the default run


def timed_solves(pdr, torch, stream, sv, flush, reps):
    """Device time (ms) of reset + solve, CUDA events on the solver's stream, L2
    flushed before each; returns every repeat and the last result."""
    times, r = [], None
    for q in range(reps):
        flush.fill_(q & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sv.reset()
        r = sv.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times, r


def error_vs_oracle(pdr, inst, sv, samples=64, seed=123):
    """Error of the solver's next FP32 sweep against the FP64 oracle on sampled
    edges: the rows of the sampled edges and of every edge incident to their
    endpoints are read back, the oracle computes the endpoints' heights
    (eq. (3), (2)) from them and the edge update (Alg. 2), and the GPU runs the
    sweep.  Reports the largest error scaled by the row scale
    sigma_e = max_k(|f| + |h_i| + |h_j|), and the element-relative error over
    entries with |f'| > 1e-3 * mean(d)."""
    import numpy as np

    import oracle

    P = oracle.Problem.from_instance(inst)
    rng = np.random.default_rng(seed)
    edges = np.sort(rng.choice(inst.m, min(samples, inst.m), replace=False))
    src = inst.src
    verts = np.unique(np.concatenate([src[edges], inst.col[edges]]))
    need = set(edges.tolist())
    for i in verts:
        need |= set(P.in_eid[P.in_ptr[i]:P.in_ptr[i + 1]].tolist())
        need |= set(range(int(inst.row_ptr[i]), int(inst.row_ptr[i + 1])))
    need = np.array(sorted(need), dtype=np.int64)
    roe = np.full(inst.m, -1, dtype=np.int64)
    roe[need] = np.arange(need.shape[0])
    rows = sv.flow_rows(need)
    sv.sweeps(1)
    new = sv.flow_rows(edges)
    h = {int(i): P.excess_vertex(int(i), roe, rows)[1] for i in verts}
    floor = 1e-3 * float(np.mean(inst.d))
    row_scaled, rel = [], []
    for q, e in enumerate(edges):
        f = rows[roe[e]]
        hi, hj = h[int(src[e])], h[int(inst.col[e])]
        want = oracle.edge_qp(hi, hj, f, inst.u[e])[0]
        sigma = float(np.max(np.abs(f) + np.abs(hi) + np.abs(hj)))
        d = np.abs(new[q] - want)
        row_scaled.append(float(d.max()) / max(sigma, 1e-300))
        big = np.abs(want) > floor
        if big.any():
            rel.append(d[big] / np.abs(want[big]))
    rel = np.concatenate(rel) if rel else np.zeros(1)
    return {"edges": int(edges.shape[0]), "entries_compared": int(rel.shape[0]),
            "max_row_scaled_err": max(row_scaled), "max_elem_rel_err": float(rel.max()),
            "p999_elem_rel_err": float(np.quantile(rel, 0.999)), "tolerance_row_scaled": 1e-5,
            "within_tolerance": bool(max(row_scaled) <= 1e-5),
            "how": "one FP32 sweep from the solver's current flows vs the FP64 oracle's heights (eq. (3), (2)) "
                   "and Alg. 2 on %d sampled edges; element-relative over |f'| > 1e-3 mean(d)" % edges.shape[0]}


def l2_resident_block(pdr, torch, stream, inst, flush, steps=5, S=2000):
    """knn2500_k500: the whole working set (both flow buffers and the heights,
    65 MB) stays in L2 across sweeps, so its kernels are reported against the
    bytes they move through L2, not as a fraction of HBM."""
    m, n, K = inst.m, inst.n, inst.K
    opts = dict(precision=pdr.PREC_FP32, eps_obj=1e-6, resid_tol=1e-6, max_sweeps=S)
    out = {"workload": WORKLOADS["knn2500_k500"], "sweeps_per_step": S, "l2_resident": True}
    with torch.cuda.stream(stream):
        with pdr.Solver.from_instance(inst, stream=stream.cuda_stream, **opts) as sv:
            timed_solves(pdr, torch, stream, sv, flush, 2)
            times, r = timed_solves(pdr, torch, stream, sv, flush, steps)
            ms = statistics.median(times)
            sv.reset()
            t_ex, t_qp = sv.time_sweeps(S)
            out["error_vs_oracle"] = error_vs_oracle(pdr, inst, sv)
        with pdr.Solver.from_instance(inst, stream=stream.cuda_stream, precision=pdr.PREC_FP32, eps_obj=1e-6,
                                      resid_tol=1e-6, max_sweeps=1000000) as sv:
            rr = sv.solve()
    b_qp = update_bytes("eso", inst)
    b_ex = 4 * K * (m + n) + 8 * m + 8 * n
    out.update({
        "updates_per_s": m * K * S / (ms / 1e3), "ms_per_step": ms,
        "us_per_sweep": ms * 1e3 / S,
        "kernel_us": {"edge_qp": t_qp * 1e3, "excess_height": t_ex * 1e3},
        "l2_gbs": {"edge_qp": b_qp / (t_qp / 1e3) / 1e9, "excess_height": b_ex / (t_ex / 1e3) / 1e9},
        "algorithmic_bytes": {"edge_qp": b_qp, "excess_height": b_ex},
        "note": "bytes per launch / mean launch along one step: L2 traffic (the 65 MB working set never leaves "
                "L2), so no fraction of the HBM peak is claimed",
        "time_to_eps": {"rule": "|z^(t)-z^(t-1)| < 1e-6 (Alg. 1)", "sweeps": rr["sweeps"], "ms": rr["ms_total"],
                        "z": rr["z"], "cap_rel": rr["cap_rel"], "cons_rel": rr["cons_rel"],
                        "verdict": rr["verdict_name"]},
    })
    return out


def residual_block(pdr, torch, stream, big, budget_sweeps=2000):
    """Time to residual 1e-6 (cap_rel and cons_rel <= 1e-6, or a Farkas
    certificate) on the 5x5 grid and its infeasible twin (GPU FP64, GPU FP32
    with the FP64 tail on the CUDA-graph engine, the same with its FP32
    sweeps on the cluster engine -- one block holding the instance in shared
    memory -- and the FP64 oracle), and on the headline instance the
    residuals reached within a fixed budget of FP32 sweeps, with the oracle's
    residuals at the same early sweep beside the GPU's."""
    import oracle
    from paper_2108_07549_gb300 import instances as I

    out = {"target": "cap_rel <= 1e-6 and cons_rel <= 1e-6 (feasible) or Farkas margin > 0 (infeasible)"}
    g = I.grid5_k10(1.3, seed=0)
    for label, inst in (("grid5_k10_feasible_1.3x", g), ("grid5_k10_infeasible_0.6x", g.with_factor(0.6))):
        row = {}
        for prec, code, eng in (("gpu_fp64", pdr.PREC_FP64, 1), ("gpu_fp32_fp64tail", pdr.PREC_FP32_FP64TAIL, 1),
                                ("gpu_fp32_fp64tail_cluster_engine", pdr.PREC_FP32_FP64TAIL, 3)):
            with torch.cuda.stream(stream):
                with pdr.Solver.from_instance(inst, stream=stream.cuda_stream, precision=code, eps_obj=0.0,
                                              resid_tol=1e-6, eps_rel=1e-13, max_sweeps=600000,
                                              use_graph=eng) as sv:
                    sv.solve()  # warm-up (graph capture)
                    sv.reset()
                    r = sv.solve()
            row[prec] = {"ms": r["ms_total"], "sweeps": r["sweeps"], "sweeps_fp64": r["sweeps_fp64"],
                         "cap_rel": r["cap_rel"], "cons_rel": r["cons_rel"], "margin": r["margin"],
                         "verdict": r["verdict_name"], "stop": r["stop_name"],
                         "fp32_phase_stop": r["stop_name_fp32"]}
        P = oracle.Problem.from_instance(inst)
        t0 = time.perf_counter()
        f, rep = P.solve_eso(max_sweeps=300000, eps_obj=0.0, resid_tol=1e-6)
        if rep["stop_reason"] != 2:
            f, rep2 = P.solve_eso(max_sweeps=300000, eps_obj=1e-15, f0=f)
            rep = dict(rep2, sweeps=rep["sweeps"] + rep2["sweeps"])
        dt = time.perf_counter() - t0
        res = P.residuals(f)
        row["oracle_fp64"] = {"ms": dt * 1e3, "sweeps": rep["sweeps"], "cap_rel": res["cap_rel"],
                              "cons_rel": res["cons_rel"], "margin": res["margin"],
                              "verdict": {0: "unknown", 1: "feasible", 2: "infeasible"}[res["verdict"]]}
        row["same_verdict"] = len({v["verdict"] for v in row.values()}) == 1
        out[label] = row
    # the headline instance: residuals within a budget, and beside the oracle at sweep 3
    P = oracle.Problem.from_instance(big)
    chk = {}
    for S in (3, budget_sweeps):
        with torch.cuda.stream(stream):
            with pdr.Solver.from_instance(big, stream=stream.cuda_stream, precision=pdr.PREC_FP32, eps_obj=0.0,
                                          resid_tol=1e-6, max_sweeps=S) as sv:
                r = sv.solve()
        chk[str(S)] = {"gpu_fp32": {"ms": r["ms_total"], "cap_rel": r["cap_rel"], "cons_rel": r["cons_rel"],
                                    "z": r["z"], "verdict": r["verdict_name"]}}
    threads = oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    f3, _ = P.solve_eso(max_sweeps=3, eps_obj=0.0)
    res = P.residuals(f3)
    oracle.set_threads(1)
    chk["3"]["oracle_fp64"] = {"s": time.perf_counter() - t0, "cap_rel": res["cap_rel"], "cons_rel": res["cons_rel"],
                               "z": res["z"], "threads": threads}
    g3, o3 = chk["3"]["gpu_fp32"], chk["3"]["oracle_fp64"]
    chk["3"]["rel_diff"] = {k: abs(g3[k] - o3[k]) / max(abs(o3[k]), 1e-300) for k in ("z", "cap_rel", "cons_rel")}
    out[big.name.split("@")[0] + "_within_budget"] = {
        "checkpoints": chk,
        "note": "PDR is first order: on this instance the 1e-6 residuals lie far beyond a bench budget, so the "
                "residuals reached after %d FP32 sweeps are reported" % budget_sweeps}
    return out


def batch_forms_block(pdr, torch, stream, big_batch, small_batch, flush):
    """The batched form against the single-instance form on the same GPU, the
    same instances and the same S sweeps each (Alg. 1 + Alg. 2, FP32): one
    batch against one solve after another.  For the first 64 small instances
    also to residual 1e-6 (FP32 with the FP64 tail)."""
    out = {}
    for label, insts, S in (("batch256_uneven", big_batch, 50), ("batch256_small", small_batch, 200)):
        opts = dict(precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=S)
        total = sum(x.m * x.K for x in insts) * S
        with torch.cuda.stream(stream):
            t0 = time.perf_counter()
            B = pdr.Batch(insts, stream=stream.cuda_stream, **opts)
            t_create = time.perf_counter() - t0
            B.solve()
            bt = []
            for q in range(3):
                B.reset()
                flush.fill_(q & 0xFF)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = B.solve()
                bt.append(time.perf_counter() - t0)
            assert all(r["sweeps"] == S for r in res)
            B.close()
            singles = [pdr.Solver.from_instance(x, stream=stream.cuda_stream, **opts) for x in insts]
            for sv in singles:
                sv.solve()
            st = []
            for q in range(3):
                for sv in singles:
                    sv.reset()
                flush.fill_(q & 0xFF)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for sv in singles:
                    sv.solve()
                st.append(time.perf_counter() - t0)
            for sv in singles:
                sv.close()
        tb, ts = statistics.median(bt), statistics.median(st)
        out[label] = {"instances": len(insts), "sweeps_per_instance": S, "updates_per_solve": total,
                      "n_range": [min(x.n for x in insts), max(x.n for x in insts)],
                      "K_range": [min(x.K for x in insts), max(x.K for x in insts)],
                      "batch_s": tb, "batch_updates_per_s": total / tb, "create_and_autotune_s": t_create,
                      "sequential_s": ts, "sequential_updates_per_s": total / ts, "speedup": ts / tb}
    # the first 64 small instances solved to residual 1e-6
    small_batch = small_batch[:64]
    opts = dict(precision=pdr.PREC_FP32_FP64TAIL, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13, max_sweeps=20000)
    with torch.cuda.stream(stream):
        B = pdr.Batch(small_batch, stream=stream.cuda_stream, **opts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rb = B.solve()
        tb = time.perf_counter() - t0
        B.close()
        rs, ts = [], 0.0
        for x in small_batch:
            with pdr.Solver.from_instance(x, stream=stream.cuda_stream, **opts) as sv:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rs.append(sv.solve())
                ts += time.perf_counter() - t0
    want = [x.feasible_by_construction for x in small_batch]

    def summary(res):
        v = [r["verdict_name"] for r in res]
        feas = [r for r in res if r["verdict_name"] == "feasible"]
        tails = [r["stop_name_fp32"] for r in res if r["sweeps_fp64"] > 0]
        return {"verdicts": {k: v.count(k) for k in sorted(set(v))},
                "sweeps_max": max(r["sweeps"] for r in res),
                "fp64_tail_started_by": {k: tails.count(k) for k in sorted(set(tails))},
                "max_cap_rel_feasible": max((r["cap_rel"] for r in feas), default=None),
                "max_cons_rel_feasible": max((r["cons_rel"] for r in feas), default=None),
                "verdicts_as_constructed": sum(1 for r, w in zip(res, want)
                                               if w is not None and r["verdict_name"] ==
                                               ("feasible" if w else "infeasible"))}

    out["batch64_small_to_residual"] = {
        "instances": len(small_batch),
        "precision": "FP32 sweeps, FP64 tail, FP64 residuals and certificate", "max_sweeps": 20000,
        "batch": {"s": tb, **summary(rb)}, "sequential": {"s": ts, **summary(rs)}, "speedup": ts / tb,
        "same_verdicts": all(a["verdict"] == b["verdict"] for a, b in zip(rb, rs))}
    return out


def adjoint_block(pdr, torch, stream, inst, T=50, ckpt=10):
    """The differentiated form on digraph20k_k2000 (time_reverse_mode)."""
    out = {"workload": WORKLOADS["digraph20k_k2000"]}
    out.update(time_reverse_mode(pdr, torch, stream, inst, T, ckpt))
    return out


# --------------------------------------------------------------------------- GPU arm


def main():
    args = parse()
    rank, world, local = dist_info()
    from paper_2108_07549_gb300 import instances

    inst = {"knn2500_k500": lambda: instances.knn2500_k500(1.2, seed=0),
            "grid100_k10000": lambda: instances.grid100_k10000(1.1, seed=0),
            "digraph20k_k2000": lambda: instances.digraph20k_k2000(1.05, seed=0),
            # a spawn pool, before any CUDA work in this process
            "batch256": lambda: instances.batch256(seed=0, count=args.instances,
                                                   processes=os.cpu_count() or 1)}[args.workload]()
    if args.sweeps <= 0 and not args.to_residual:
        args.sweeps = 2000 if args.workload == "knn2500_k500" else 200
    global WORKLOAD
    WORKLOAD = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, inst)
        return
    plain = not (args.profile_sweeps or args.compare_algos or args.compare_variants or args.compare_excess or
                 args.compare_engines or args.adjoint or args.to_residual or args.workload == "batch256")
    extras = plain and not args.no_extras and rank == 0 and world == 1
    side = {}
    if extras:
        # the extra blocks' inputs, generated before any CUDA work (spawn pools)
        side["knn"] = instances.knn2500_k500(1.2, seed=0)
        if not args.no_forms:
            side["batch"] = instances.batch256(seed=0, count=256, processes=os.cpu_count() or 1)
            side["small"] = instances.batch256(seed=1, count=256, n_range=(100, 500), k_range=(10, 100),
                                               processes=os.cpu_count() or 1)
            side["c5"] = instances.digraph20k_k2000(1.05, seed=0)

    import numpy as np
    import torch

    from paper_2108_07549_gb300 import build, pdr, replicas

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    pdr.load()
    stream = torch.cuda.Stream()
    if args.profile_sweeps > 0:
        with torch.cuda.stream(stream):
            with pdr.Solver.from_instance(inst, stream=stream.cuda_stream, precision=pdr.PREC_FP32,
                                          algo=ALGOS[args.algo], edge_variant=args.edge_variant,
                                          excess_variant=args.excess_variant) as sv:
                sv.sweeps(args.profile_sweeps)
        torch.cuda.synchronize()
        return
    if args.compare_algos:
        compare_algos(args, inst, pdr, torch, stream)
        return
    if args.compare_variants:
        compare_variants(args, inst, pdr, torch, stream)
        return
    if args.compare_excess:
        compare_excess(args, inst, pdr, torch, stream)
        return
    if args.compare_engines:
        compare_engines(args, inst, pdr, torch, stream)
        return
    if args.workload == "batch256":
        if args.to_residual:
            bench_batch_to_residual(args, inst, pdr, torch, stream)
        else:
            bench_batch(args, inst, pdr, torch, stream)
        return
    if args.adjoint:
        bench_adjoint(args, inst, pdr, torch, stream)
        return
    if args.to_residual:
        solve_to_residual(args, inst, pdr, torch, stream)
        return
    S = args.sweeps
    opts = dict(precision=pdr.PREC_FP32, eps_obj=1e-6, resid_tol=1e-6, max_sweeps=S,
                use_graph=0 if args.host_loop else (2 if args.engine == "persistent" else 1), algo=ALGOS[args.algo],
                edge_variant=args.edge_variant, excess_variant=args.excess_variant)
    m, K = inst.m, inst.K
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- device-resident steps
    with torch.cuda.stream(stream):
        solver = pdr.Solver.from_instance(inst, stream=stream.cuda_stream, **opts)
        for _ in range(args.warmup):
            solver.reset()
            r = solver.solve()
        assert r["sweeps"] == S, r
        barrier()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        with ClockSampler(local) as clocks:
            for q in range(args.steps):
                flush.fill_(q & 0xFF)
                ev0[q].record(stream)
                solver.reset()
                r = solver.solve()
                ev1[q].record(stream)
            torch.cuda.synchronize()
        times = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        barrier()
    ms_step = replicas.slowest(sum(times) / len(times), world, device="cuda")
    value = replicas.job_throughput(m * K * S, ms_step / 1e3, world)
    # S + 1 objective evaluations (the last one stops); the graph body holds 32
    # sweeps (two kernels each), the host loop launches chunks of 256 sweeps;
    # plus residuals (3), solve state init (1), reset (psi refresh + state init)
    if args.engine == "persistent" and not args.host_loop:
        # one cooperative launch per 1024 sweeps (+ barrier reset each), the
        # congestion refresh at the end, residuals, state init, reset
        launches_per_step = 2 * (-(-(S + 1) // 1024)) + 1 + 3 + 1 + 2
    else:
        chunk = 256 if args.host_loop else 32
        launches_per_step = 2 * chunk * (-(-(S + 1) // chunk)) + 3 + 1 + 2

    # ---------------------------------------------------------------- end to end through the C ABI
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    host = [pin(x) for x in (inst.row_ptr, inst.col, inst.u, inst.s, inst.t, inst.d)]
    out = torch.empty((m, K), dtype=torch.float64).pin_memory().numpy()
    h2d = sum(x.nbytes for x in host)
    d2h = m * K * 8  # the flows, widened to double on the device and written into pinned host memory
    e2e_times = []
    with torch.cuda.stream(stream):
        for q in range(max(1, args.warmup) + args.steps):
            flush.fill_(q & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with pdr.Solver(inst.n, *host, stream=stream.cuda_stream, **opts) as sv:
                sv.solve()
                sv._check(sv._lib.pdr_flows(sv._h, out.ctypes.data_as(__import__("ctypes").c_void_p)))
            t1 = time.perf_counter()
            if q >= max(1, args.warmup):
                e2e_times.append(t1 - t0)
    e2e_s = replicas.slowest(sum(e2e_times) / len(e2e_times), world, device="cuda")
    e2e_value = replicas.job_throughput(m * K * S, e2e_s, world)
    working_set = 4 * K * (2 * m + inst.n)  # both flow buffers and the heights, FP32

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sweeps_per_step": S, "precision": "FP32 flows and edge QP, FP64 stop "
                   "test and certificate",
                   "l2": "256 MiB buffer overwritten between timed steps; the working set (%.2f GB) exceeds L2"
                         % (working_set / 1e9) if working_set > L2_RESIDENT_BYTES else
                         "256 MiB buffer overwritten between timed steps",
                   "parallelism": "replicas" if world > 1 else "single",
                   "engine": "host loop" if args.host_loop else args.engine},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks.summary(),
        "step_result": {k: r[k] for k in ("sweeps", "z", "cap_rel", "cons_rel", "verdict_name")},
    }

    if not args.no_extras and rank == 0:
        # each kernel's mean launch along the S sweeps of one step from f = 0,
        # host-launched with CUDA events on the solver's stream around every
        # launch, reconciled with the sweep time inside the graph loop (two
        # solves of S and 2S sweeps)
        with torch.cuda.stream(stream):
            solver.reset()
            t_ex, t_qp = solver.time_sweeps(S)
            t_qp_c = solver.time_kernel("qp", 10, FLUSH_BYTES)
            t_ex_c = solver.time_kernel("excess", 10, FLUSH_BYTES)
            t1, _ = timed_solves(pdr, torch, stream, solver, flush, 3)
            solver.set_options(max_sweeps=2 * S)
            t2, _ = timed_solves(pdr, torch, stream, solver, flush, 3)
            solver.set_options(max_sweeps=S)
            solver.reset()
            solver.solve()
            line["error_vs_oracle"] = error_vs_oracle(pdr, inst, solver)
        graph_us = (statistics.median(t2) - statistics.median(t1)) * 1e3 / S
        n = inst.n
        bytes_qp = update_bytes(args.algo, inst)
        bytes_ex = 4 * K * (m + n) + 4 * 2 * m + 8 * n  # f once, h out; incidence lists
        upd = {"eso": "edge_qp", "agd": "agd_step", "gdm": "gdm_step", "ck": "edge_qp_ck"}[args.algo]
        dom, t_dom, b_dom = (upd, t_qp, bytes_qp) if t_qp >= t_ex else ("excess_height", t_ex, bytes_ex)
        t_dom_c = t_qp_c if dom == upd else t_ex_c
        peak, peak_src = load_peaks()
        achieved = b_dom / (t_dom / 1e3) / 1e9
        resident = working_set <= L2_RESIDENT_BYTES
        line["roofline"] = {"bound": "l2" if resident else "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": ncu_traffic(dom), "kernel": dom,
                            "peak_source": f"{peak_src} hbm_gbs (burst copy)",
                            "timing": "mean launch over the %d sweeps of one step from f = 0, CUDA events around "
                                      "each launch on the solver's stream" % S,
                            "kernel_us": {upd: t_qp * 1e3, "excess_height": t_ex * 1e3},
                            "kernel_us_sum_per_sweep": (t_qp + t_ex) * 1e3,
                            "graph_loop_us_per_sweep": graph_us,
                            "step_us_per_sweep": ms_step * 1e3 / S,
                            "algorithmic_bytes": {upd: bytes_qp, "excess_height": bytes_ex},
                            "sweep_algorithmic_bytes": bytes_qp + bytes_ex,
                            "sweep_achieved_gbs": (bytes_qp + bytes_ex) / (graph_us / 1e6) / 1e9,
                            "share_update": t_qp / (t_qp + t_ex),
                            "l2_state": ("warm: the working set (%.0f MB) stays in L2" % (working_set / 1e6))
                                        if resident else
                                        ("the working set (%.2f GB) exceeds L2: the rows stream from HBM "
                                         "every sweep" % (working_set / 1e9)),
                            "cold_l2": {"kernel_us": {upd: t_qp_c * 1e3, "excess_height": t_ex_c * 1e3},
                                        "frac": b_dom / (t_dom_c / 1e3) / 1e9 / peak}}
        if world == 1:  # the host cores are shared by the ranks of a multi-GPU run
            line["cpu_baseline"] = cpu_baseline(inst)
    solver.close()
    if extras:
        del out, host
        line["l2_resident_knn2500_k500"] = l2_resident_block(pdr, torch, stream, side["knn"], flush)
        line["time_to_residual"] = residual_block(pdr, torch, stream, inst)
        if not args.no_forms:
            line["batched_form"] = batch_forms_block(pdr, torch, stream, side["batch"], side["small"], flush)
            line["differentiated_form"] = adjoint_block(pdr, torch, stream, side["c5"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
