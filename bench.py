#!/usr/bin/env python
"""Time-to-solution of the GB300 barycentric Lagrange treecode on its headline workload.

Workload: 1e6 particles uniform in [-1,1]^3 with charges uniform in [-1,1] (Sec. IV test
systems), Coulomb kernel, theta = 0.7, degree n = 8, N_L = N_B = 2000, mixed precision.
A step is one pass of the whole path for new positions on resident device inputs: source
tree (= target batches), MAC lists, modified charges, far- and near-field sweep, finalize,
run as one CUDA graph sized on the device (bltc_graph_create_positions); the steps alternate
two seeded draws of the workload.  The host-driven bltc_solve of the first draw is timed
beside it and gives the per-phase times and the sweep's roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own independent system
on its own GPU (replicas: the treecode of one system needs no exchange); the value is the
whole job's targets per second over the slowest rank.  ``--impl reference`` times the FP64
CPU oracle (Algorithm 1 as written, on the host cores) on a bounded sample of the same
workload in every step: the evaluation of eight batches per core.

The default run adds sub-records for the 1e4 cube (errors over all targets), the 8e6 Plummer
(Yukawa) and the 2.56e8 uniform (n = 10) configurations under "configs", and the oracle's measured time for the whole 1e6 system under
"cpu_baseline".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("targets/sec and effective interactions/sec at rel. err ≤1e-6 vs FP64 GPU BLTC; "
          "p50/p99")
WORKLOAD = dict(kind="cube", n=1_000_000, theta=0.7, degree=8, leaf=2000, batch=2000,
                kernel=0, kappa=0.0, seed=20031838)
WORKLOAD_NAME = ("uniform cube N=1e6 (q in [-1,1]), Coulomb, theta=0.7, n=8, N_L=N_B=2000, "
                 "mixed FP32 evaluation / FP64 accumulation")


def workload_name(w):
    """The workload's description, with any size or theta override spelled out."""
    if w["n"] == WORKLOAD["n"] and w["theta"] == WORKLOAD["theta"]:
        return WORKLOAD_NAME
    return (f"uniform cube N={w['n']} (q in [-1,1]), Coulomb, theta={w['theta']}, n={w['degree']}, "
            f"N_L=N_B={w['leaf']}, mixed FP32 evaluation / FP64 accumulation (override of the "
            f"1e6 workload)")
# Roofline of the sweep: one interaction of the Coulomb kernel costs one MUFU.RSQ; the SFU
# (XU) pipe issues 16 per clock per SM, so the peak interaction rate is SMs * 16 * f_max.
XU_PER_CLK_PER_SM = 16
# A Yukawa evaluation adds one MUFU.EX2 on the same pipe, measured at 26 per clock per SM
# (microbenchmark): 1/16 + 1/26 clocks of the pipe per evaluation.
XU_EX2_PER_CLK_PER_SM = 26
SM_MAX_MHZ = 2070.0
L2_FLUSH_BYTES = 256 << 20
# the sweep kernel's source: its device code and the file that plans, instantiates and launches
# it, less the finalize kernel defined there (it runs after the sweep and does not change it)
SWEEP_SOURCES = [os.path.join(ROOT, "paper_2003_01836_gb300", "csrc", f)
                 for f in ("sweep_device.cuh", "sweep.cu")]
FINALIZE_START = "__global__ void k_finalize("


def sweep_source_sha256():
    h = hashlib.sha256()
    for path in SWEEP_SOURCES:
        with open(path) as f:
            text = f.read()
        if FINALIZE_START in text:
            a = text.index(FINALIZE_START)
            text = text[:a] + text[text.index("\n}\n", a) + 3:]
        h.update(text.encode())
    return h.hexdigest()
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_sweep_mixed_traffic.txt")


# ---- distributed helpers (one process per GPU, replicas) --------------------------------

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local_rank)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(per_rank_ms: float, n_per_rank: int, dist: Dist) -> dict:
    """Whole-job throughput over the slowest rank (weak scaling: fixed work per GPU)."""
    slowest = dist.max(per_rank_ms)
    total_targets = dist.sum(n_per_rank)
    return {"ms_per_step": slowest, "targets_per_s": total_targets / (slowest / 1e3),
            "total_targets": total_targets}


# ---- clocks sampled during the timed region ----------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=self.out,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ---- the CPU oracle on a bounded sample ----------------------------------------------------

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_measured(x, y, z, q, w, sample_batches=None, threads=None):
    """Algorithm 1 on the host cores, measured: the setup (trees, modified charges), then the
    evaluation of every batch; with ``sample_batches`` also the evaluation of that many batches
    spread over the system (one per core), extrapolated by target count, and the error of that
    estimate against the measured whole."""
    import oracle
    cores = threads or os.cpu_count() or 1
    prep = oracle.Prepared(x, y, z, q, w["theta"], w["degree"], w["leaf"], w["batch"],
                           w["kernel"], w["kappa"], threads=cores)
    setup = prep.timings["setup"] + prep.timings["precompute"]
    n = len(x)
    out = {"cores": cores, "cpu_model": cpu_model(), "setup_s": setup, "n_batches": prep.n_batches}
    if sample_batches:
        st = oracle.Tree(x, y, z, w["batch"])
        nl = len(st.leaves)
        pick = np.unique(np.linspace(0, nl - 1, min(nl, sample_batches)).astype(np.int64))
        targets = int(st.count[st.leaves[pick]].sum())
        _, _, sec = prep.evaluate(pick, threads=cores)
        out["estimate_s"] = setup + sec * (n / targets)
        out["estimate_sample"] = (f"ComputePotential on {len(pick)} of {nl} batches ({targets} "
                                  f"targets), extrapolated by target count")
    _, _, sec = prep.evaluate(None, threads=cores)
    out["measured_full_s"] = setup + sec
    if sample_batches:
        out["estimate_error"] = out["estimate_s"] / out["measured_full_s"] - 1.0
    prep.close()
    return out


def oracle_sample(x, y, z, q, w, budget_batches=None, threads=None):
    """Algorithm 1 on the host cores: full trees and modified charges, ComputePotential on a
    sample of batches; time-to-solution extrapolated by target count (an estimate)."""
    import oracle
    cores = threads or os.cpu_count() or 1
    st = oracle.Tree(x, y, z, w["leaf"])
    nl = len(st.leaves)
    k = budget_batches or max(2, min(nl, cores))
    pick = (np.array([nl // 2], dtype=np.int64) if k == 1
            else np.unique(np.linspace(0, nl - 1, k).astype(np.int64)))
    targets = int(st.count[st.leaves[pick]].sum())
    t0 = time.perf_counter()
    _, _, tm = oracle.bltc(x, y, z, q, w["theta"], w["degree"], w["leaf"], w["batch"],
                           w["kernel"], w["kappa"], threads=cores, batches=pick)
    wall = time.perf_counter() - t0
    n = len(x)
    t_est = tm["setup"] + tm["precompute"] + tm["compute"] * (n / targets)
    # the sampled batches run one per thread: threads beyond the sample idle in the compute phase
    return {"targets_per_s": n / t_est, "t_est_s": t_est, "wall_s": wall, "cores": min(cores, len(pick)),
            "cpu_model": cpu_model(),
            "sample": (f"full source/batch trees and modified charges of the {n}-particle "
                       f"system, ComputePotential on {len(pick)} of {nl} batches "
                       f"({targets} targets); time extrapolated by target count"),
            "phases_s": tm}


# ---- our arm -----------------------------------------------------------------------------

def traffic_for_current_kernel():
    """DRAM bytes per sweep launch from the committed ncu summary, if it was taken on the
    current sweep source (matching SHA-256), else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            kv = dict(line.strip().split(": ", 1) for line in f if ": " in line)
        sha = sweep_source_sha256()
        if kv.get("sweep_source_sha256") != sha:
            return None
        return float(kv["dram_bytes_per_launch_full_size"])
    except (OSError, KeyError, ValueError):
        return None


def run_ours(args, dist: Dist):
    import torch

    import paper_2003_01836_gb300 as b
    from paper_2003_01836_gb300 import build, inputs
    build.build()
    dev = dist.local_rank
    torch.cuda.set_device(dev)
    w = dict(WORKLOAD)
    if args.n:
        w["n"] = args.n
    if args.theta >= 0:
        w["theta"] = args.theta
    x, y, z, q = inputs.system(w["kind"], w["n"], w["seed"] + dist.rank)
    X = [torch.from_numpy(a).to(f"cuda:{dev}") for a in (x, y, z, q)]
    # a second seeded draw of the workload: the graph's steps alternate the two systems, so
    # that every step solves positions other than the previous step's
    X2 = [torch.from_numpy(a).to(f"cuda:{dev}")
          for a in inputs.system(w["kind"], w["n"], w["seed"] + dist.rank + 1000)]
    systems = (X, X2)
    phi = torch.empty_like(X[0])
    ctx = b.Context(dev)
    p = b.params(w["degree"], w["theta"], w["leaf"], w["batch"], w["kernel"], w["kappa"],
                 b.BLTC_PRECISION_MIXED)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{dev}")

    # The step: the whole solve for new positions as one CUDA graph (bltc_graph_create_positions:
    # tree, lists, upward pass, plan, sweep and finalize sized on the device).  A step copies
    # the step's positions and charges into the graph's bound tensors and launches it.
    B = [t.clone() for t in X]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = b.Graph(ctx, *B[:3], B[3], p, positions=True)
    torch.cuda.synchronize()
    graph_setup_ms = 1e3 * (time.perf_counter() - t0)

    def load(k):
        for t, src in zip(B, systems[k]):
            t.copy_(src)

    for i in range(args.warmup):
        load(i % 2)
        g.launch()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    step_ms = []
    launches0 = b.bltc_context_launch_count(ctx.h)
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for i in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        load(i % 2)
        g.launch()
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    dist.barrier()
    launches = b.bltc_context_launch_count(ctx.h) - launches0
    mean_ms = sum(step_ms) / len(step_ms)
    agg = aggregate(mean_ms, w["n"], dist)
    graph_info = g.info

    # The host-driven solve (bltc_solve) of the first system, with phase events: the sweep's
    # time for the roofline (the same kernel the graph runs) and the per-phase split.
    b.bltc_context_set_timing(ctx.h, True)
    for _ in range(args.warmup):
        ctx.solve(*X, p, phi)
    torch.cuda.synchronize()
    host_ms, phases = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.solve(*X, p, phi)
        e1.record()
        e1.synchronize()
        host_ms.append(e0.elapsed_time(e1))
        phases.append(b.bltc_last_timings(ctx.h))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    b.bltc_context_set_timing(ctx.h, False)
    load(0)
    g.launch()
    graph_bits_equal = bool(torch.equal(g.phi, phi))

    # evaluated interactions of one step (same lists every step)
    st = b.bltc_tree_build(ctx.h, X[0], X[1], X[2], X[3], w["leaf"])
    L = b.bltc_lists_build(ctx.h, st, st, p)
    counts = b.bltc_stats(ctx.h, L)
    # kernel evaluations the sweep performs (a mutual leaf pair once for both batches)
    kernel_evals = b.bltc_evaluations(ctx.h, L, p)
    n_batches = b.bltc_lists_info(L)["n_batches"]
    b.bltc_lists_destroy(L)
    b.bltc_tree_destroy(st)
    evaluated = counts["direct"] + counts["approx"]

    ph = {k: statistics.mean(d[k] for d in phases) for k in phases[0]}
    sweep_s = ph["sweep"] / 1e3
    achieved = kernel_evals / sweep_s / 1e9
    peak = ctx.sm_count * XU_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e9
    roofline = {"bound": "alu", "pipe": "XU (MUFU rsqrt), 1 per Coulomb interaction",
                "kernel": "k_sweep_mixed<Coulomb>", "achieved": achieved, "peak": peak,
                "unit": "G interactions/s", "frac": achieved / peak,
                "traffic": traffic_for_current_kernel(),
                "peak_basis": f"{ctx.sm_count} SMs x {XU_PER_CLK_PER_SM}/clk x "
                              f"{SM_MAX_MHZ:.0f} MHz (recipe max SM clock)",
                "units_per_launch": kernel_evals,
                "unit_definition": "kernel evaluations G(x_i, y_j) performed by the sweep: "
                                   "approximation terms plus direct terms, a mutual leaf pair "
                                   "evaluated once for both batches"}

    out = {"metric": METRIC, "value": agg["targets_per_s"], "unit": "targets/s",
           "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": agg["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (f64 accumulation)", "data": "synthetic",
           "config": {"workload": workload_name(w), "n_particles": w["n"], "theta": w["theta"],
                      "degree": w["degree"], "leaf_size": w["leaf"], "batch_size": w["batch"],
                      "kernel": "coulomb", "precision": "mixed", "batches": n_batches,
                      "parallelism": f"replicas x{dist.world}",
                      "l2": "flushed before every timed step (256 MiB device write)"},
           "effective_interactions_per_s": w["n"] * w["n"] * dist.world / (agg["ms_per_step"] / 1e3),
           "evaluated_interactions_per_step": evaluated,
           "kernel_evaluations_per_step": kernel_evals,
           "evaluated_interactions_per_s": evaluated * dist.world / (agg["ms_per_step"] / 1e3),
           "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                          "p99": float(np.percentile(step_ms, 99)),
                          "min": min(step_ms), "max": max(step_ms)},
           "phases_ms": ph, "clocks": clocks, "gpu_launches": int(launches),
           "roofline": roofline,
           "step": {"api": "bltc_graph_create_positions + bltc_graph_launch (whole solve, one CUDA graph)",
                    "systems": "two seeded draws of the workload, alternating",
                    "kernels_per_launch": graph_info["kernels"], "redone": graph_info["redone"],
                    "graph_setup_ms": graph_setup_ms, "bits_equal_to_bltc_solve": graph_bits_equal},
           "host_driven": {"api": "bltc_solve (host reads each count back)",
                           "ms_per_step": statistics.mean(host_ms),
                           "p50": float(np.percentile(host_ms, 50)),
                           "p99": float(np.percentile(host_ms, 99)),
                           "note": "phases_ms and the roofline come from these solves"}}

    if not args.no_check:
        out["error"] = check_errors(ctx, b, X, p, w, g.phi)
    if not args.no_e2e:
        out["e2e"] = run_e2e(ctx, b, x, y, z, q, g, B, args, dist, w)
    g.close()
    # the sub-records run on one GPU only: under torchrun every rank is a replica of the main
    # workload, and N copies of the 2.56e8 system or the request stream would crowd the host
    if dist.world == 1 and not args.no_serving:
        sv = serve_measure(args.serve_record_requests, (0.5,), args.serve_workers, dist,
                           args.serve_slice_us, args.serve_setup_blocks, args.serve_slices_in_flight)
        out["serving"] = {"requests": sv["config"]["requests"], "total_targets": sv["config"]["total_targets"],
                          "mix": sv["config"]["mix"], "slice_us": sv["config"]["slice_us"],
                          "setup_blocks": sv["config"]["setup_blocks"],
                          "slices_in_flight": sv["config"]["slices_in_flight"], "levels": sv["levels"], "solo": sv["solo"],
                          "served_vs_solo": sv["served_vs_solo"]}
    if dist.world == 1 and not args.no_configs:
        out["configs"] = {}
        for key in args.configs.split(","):
            if key == "1":
                out["configs"][key] = run_config1(ctx, b, dist)
            elif key:
                out["configs"][key] = run_config(ctx, b, key, args, dist)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cb = oracle_measured(x, y, z, q, w, sample_batches=os.cpu_count() or 1)
        one = oracle_sample(x, y, z, q, w, budget_batches=1, threads=1)
        out["cpu_baseline"] = {"value": w["n"] / cb["measured_full_s"], "unit": "targets/s",
                               "cores": cb["cores"], "kind": "oracle",
                               "sample": (f"the whole {w['n']}-particle system, measured: trees and "
                                          f"modified charges, then ComputePotential on all "
                                          f"{cb['n_batches']} batches"),
                               "cpu_model": cb["cpu_model"], "measured_full_s": cb["measured_full_s"],
                               "setup_s": cb["setup_s"],
                               "sampled_estimate": {"t_est_s": cb["estimate_s"], "sample": cb["estimate_sample"],
                                                    "error_vs_measured": cb["estimate_error"]},
                               "single_thread": {"value": one["targets_per_s"], "cores": 1,
                                                 "kind": "estimate", "sample": one["sample"],
                                                 "t_est_s": one["t_est_s"], "wall_s": one["wall_s"]}}
    ctx.close()
    return out


# ---- the large configurations: sub-records of the default run ------------------------------

CONFIGS = {
    "3": dict(kind="plummer", n=8_000_000, theta=0.8, degree=8, kernel=1, kappa=0.5, seed=20031839,
              fp32_storage=False, steps=3, warmup=1, error_targets=10_000, tiles=True,
              name=("truncated Plummer sphere N=8e6 (a=1, r<=10), q in [-1,1], Yukawa kappa=0.5, "
                    "theta=0.8, n=8, leaf=batch autotuned over {500,1000,2000,3000,4000}, then the "
                    "sweep's tile shape autotuned, mixed")),
    "5": dict(kind="cube", n=256_000_000, theta=0.8, degree=10, kernel=0, kappa=0.0, seed=20031841,
              fp32_storage=True, steps=2, warmup=1, error_targets=2048,
              name=("uniform cube N=2.56e8, xyzq stored in FP32 (read as FP64), Coulomb, theta=0.8, "
                    "n=10, leaf=batch autotuned over {500,1000,2000,3000,4000}, mixed")),
}
CANDIDATES = (500, 1000, 2000, 3000, 4000)
# tile shapes tried after the sizes (bltc_params.tile): the default, caps of 4 and 2 source
# groups per batch, and 8 or 32 work items per resident block
TILE_CANDIDATES = (0, 4, 2, 8 << 4, 32 << 4)


def tile_name(t):
    g, ipb = t & 15, (t >> 4) & 255
    return f"groups<={g or 8},items/block={ipb or 16}"


def xu_peak(sm_count, kernel):
    """Kernel evaluations per second the XU pipe allows at the recipe's maximum SM clock:
    one MUFU.RSQ per evaluation (16 per clock per SM), plus one MUFU.EX2 for Yukawa (26)."""
    per_clk = XU_PER_CLK_PER_SM if kernel == 0 else 1.0 / (1.0 / XU_PER_CLK_PER_SM +
                                                            1.0 / XU_EX2_PER_CLK_PER_SM)
    return sm_count * per_clk * SM_MAX_MHZ * 1e6, per_clk


def sample_batches(leaf_counts, goal, seed):
    """Seeded random batches, in increasing order, until they hold `goal` targets (a cluster
    sample of targets: the error of Eq. 16 on a subset of targets, Sec. IV)."""
    order = np.random.default_rng(seed).permutation(len(leaf_counts))
    total, pick = 0, []
    for i in order:
        pick.append(int(i))
        total += int(leaf_counts[i])
        if total >= goal:
            break
    return np.sort(np.array(pick, dtype=np.int32))


def run_config(ctx, b, key, args, dist):
    """One large configuration: autotuned leaf/batch size, a few timed solves (inputs larger
    than L2), kernel evaluations and the sweep's roofline, and Eq. 16 errors on sampled
    batches: mixed and FP64 treecode against the FP64 direct sum, and mixed against FP64."""
    import torch
    from paper_2003_01836_gb300 import inputs
    c = dict(CONFIGS[key])
    if key == "5" and args.error_targets5:
        c["error_targets"] = args.error_targets5
    t0 = time.perf_counter()
    host = inputs.system(c["kind"], c["n"], c["seed"] + dist.rank)
    if c["fp32_storage"]:
        host = [a.astype(np.float32).astype(np.float64) for a in host]
    X = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in host]
    del host
    gen_s = time.perf_counter() - t0
    p = b.params(c["degree"], c["theta"], 2000, 2000, c["kernel"], c["kappa"], b.BLTC_PRECISION_MIXED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, tune_ms = b.bltc_autotune(ctx.h, *X, p, leaf=CANDIDATES, repeats=1, use_cache=False)
    tune_s = time.perf_counter() - t0
    tile_rec = {"searched": False, "reason": "one solve of this configuration takes seconds; "
                                             "the default tile is kept"}
    if c.get("tiles"):
        t0 = time.perf_counter()
        best, tile_ms = b.bltc_autotune_tile(ctx.h, *X, best, TILE_CANDIDATES, repeats=1, use_cache=False)
        tile_rec = {"searched": True, "seconds": time.perf_counter() - t0,
                    "candidates": {tile_name(t): v for t, v in tile_ms.items()},
                    "chosen": tile_name(best.tile)}
    phi = torch.empty_like(X[0])
    b.bltc_context_set_timing(ctx.h, True)          # phase events for the sweep's roofline
    for _ in range(c["warmup"]):
        ctx.solve(*X, best, phi)
    torch.cuda.synchronize()
    sampler = ClockSampler(dist.local_rank)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    step_ms, phases = [], []
    sampler.start()
    for _ in range(c["steps"]):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.solve(*X, best, phi)
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        phases.append(b.bltc_last_timings(ctx.h))
    clocks = sampler.stop()
    b.bltc_context_set_timing(ctx.h, False)
    del flush
    ph = {k: statistics.mean(d[k] for d in phases) for k in phases[0]}
    mean_ms = statistics.mean(step_ms)

    # work counts, the sweep's roofline, and the FP64 treecode on sampled batches
    st = b.bltc_tree_build(ctx.h, *X, best.leaf_size)
    L = b.bltc_lists_build(ctx.h, st, st, best)
    counts = b.bltc_stats(ctx.h, L)
    evals = b.bltc_evaluations(ctx.h, L, best)
    n_batches = b.bltc_lists_info(L)["n_batches"]
    tree = b.bltc_tree_export(ctx.h, st, want=("perm", "begin", "count", "n_children"))
    leaves = np.flatnonzero(tree["n_children"] == 0)
    pick = sample_batches(tree["count"][leaves], c["error_targets"], c["seed"] + 1000)
    idx = np.concatenate([tree["perm"][tree["begin"][leaves[i]]:tree["begin"][leaves[i]] +
                                       tree["count"][leaves[i]]] for i in pick])
    p64 = b.params(c["degree"], c["theta"], best.leaf_size, best.batch_size, c["kernel"], c["kappa"],
                   b.BLTC_PRECISION_FP64)
    t0 = time.perf_counter()
    S = b.bltc_lists_select(ctx.h, L, pick)
    b.bltc_modified_charges(ctx.h, st, S, p64)
    phi64 = torch.empty_like(phi)
    b.bltc_evaluate(ctx.h, S, st, st, p64, phi64)
    torch.cuda.synchronize()
    fp64_s = time.perf_counter() - t0
    b.bltc_lists_destroy(S)
    b.bltc_lists_destroy(L)
    b.bltc_tree_destroy(st)
    tidx = torch.from_numpy(idx).cuda()
    T = [a.index_select(0, tidx).contiguous() for a in X[:3]]
    ref = torch.empty_like(T[0])
    t0 = time.perf_counter()
    b.bltc_direct_sum(ctx.h, *T, *X[:3], X[3], p64, ref)
    torch.cuda.synchronize()
    direct_s = time.perf_counter() - t0
    h = lambda t: t.detach().cpu().numpy()
    ref_h, mx_h, d64_h = h(ref), h(phi.index_select(0, tidx)), h(phi64.index_select(0, tidx))
    peak, per_clk = xu_peak(ctx.sm_count, c["kernel"])
    achieved = evals / (ph["sweep"] / 1e3)
    out = {"workload": c["name"], "n_particles": c["n"], "leaf_size": best.leaf_size,
           "batch_size": best.batch_size, "batches": n_batches,
           "autotune": {"seconds": tune_s, "candidates": list(CANDIDATES),
                        "timed_ms": {str(k[0]): v for k, v in tune_ms.items() if v == v},
                        "tile": tile_rec},
           "input_generation_s": gen_s, "steps": c["steps"], "warmup": c["warmup"],
           "ms_per_step": mean_ms, "targets_per_s": c["n"] / (mean_ms / 1e3),
           "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "max": max(step_ms)},
           "phases_ms": ph, "clocks": clocks,
           "evaluated_interactions_per_step": counts["direct"] + counts["approx"],
           "kernel_evaluations_per_step": evals,
           "roofline": {"bound": "alu", "kernel": f"k_sweep_mixed<{'Coulomb' if c['kernel'] == 0 else 'Yukawa'}>",
                        "pipe": ("XU: MUFU.RSQ at 16/clk/SM" if c["kernel"] == 0 else
                                 "XU: MUFU.RSQ (16/clk/SM) + MUFU.EX2 (26/clk/SM) per evaluation"),
                        "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "G evaluations/s",
                        "frac": achieved / peak, "evaluations_per_clk_per_sm_peak": per_clk,
                        "traffic": None,
                        "peak_basis": f"{ctx.sm_count} SMs x {per_clk:.2f}/clk x {SM_MAX_MHZ:.0f} MHz"},
           "error": {"sample": (f"targets of {len(pick)} seeded random batches ({len(idx)} targets)"),
                     "mixed_vs_fp64_gpu_bltc": rel_err(d64_h, mx_h),
                     "meets_1e-6": bool(rel_err(d64_h, mx_h) <= 1e-6),
                     "mixed_bltc_vs_fp64_direct": rel_err(ref_h, mx_h),
                     "fp64_bltc_vs_fp64_direct": rel_err(ref_h, d64_h),
                     "fp64_bltc_sampled_seconds": fp64_s, "fp64_direct_sampled_seconds": direct_s}}
    del X, phi, phi64, T, ref
    torch.cuda.empty_cache()
    return out


CONFIG1 = dict(kind="cube", n=10_000, theta=0.7, degree=4, leaf=500, kernel=0, kappa=0.0,
               seed=20031837, steps=20, warmup=3,
               name=("uniform cube N=1e4 (q in [-1,1]), Coulomb, theta=0.7, n=4, N_L=N_B=500: "
                     "FP64 and mixed GPU treecode against the FP64 GPU direct sum on all targets"))


def run_config1(ctx, b, dist):
    """The small configuration: every target's potential by the FP64 and the mixed treecode,
    each against the FP64 direct sum of Eq. 1 over all targets (Eq. 16 on the whole system),
    beside the time of each solve."""
    import torch
    from paper_2003_01836_gb300 import inputs
    c = CONFIG1
    X = [torch.from_numpy(a).cuda() for a in inputs.system(c["kind"], c["n"], c["seed"] + dist.rank)]
    out = {"workload": c["name"], "n_particles": c["n"], "steps": c["steps"], "warmup": c["warmup"]}
    phis = {}
    for name, prec in (("fp64", b.BLTC_PRECISION_FP64), ("mixed", b.BLTC_PRECISION_MIXED)):
        p = b.params(c["degree"], c["theta"], c["leaf"], c["leaf"], c["kernel"], c["kappa"], prec)
        phi = torch.empty_like(X[0])
        for _ in range(c["warmup"]):
            ctx.solve(*X, p, phi)
        torch.cuda.synchronize()
        ms = []
        for _ in range(c["steps"]):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.solve(*X, p, phi)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        phis[name] = phi.cpu().numpy()
        out[f"{name}_ms_per_solve"] = statistics.median(ms)
    p64 = b.params(c["degree"], c["theta"], c["leaf"], c["leaf"], c["kernel"], c["kappa"],
                   b.BLTC_PRECISION_FP64)
    ref = torch.empty_like(X[0])
    b.bltc_direct_sum(ctx.h, *X[:3], *X[:3], X[3], p64, ref)
    ref_h = ref.cpu().numpy()
    out["error"] = {"sample": "all targets",
                    "fp64_bltc_vs_fp64_direct": rel_err(ref_h, phis["fp64"]),
                    "mixed_bltc_vs_fp64_direct": rel_err(ref_h, phis["mixed"]),
                    "mixed_vs_fp64_gpu_bltc": rel_err(phis["fp64"], phis["mixed"]),
                    "meets_1e-6": bool(rel_err(phis["fp64"], phis["mixed"]) <= 1e-6)}
    return out


def rel_err(reference, approx):
    """Eq. 16: relative 2-norm error of approx against reference."""
    reference = np.asarray(reference, dtype=np.float64)
    approx = np.asarray(approx, dtype=np.float64)
    return float(np.sqrt(np.sum((reference - approx) ** 2) / np.sum(reference ** 2)))


def check_errors(ctx, b, X, p, w, phi_mixed):
    """Relative 2-norm errors (Eq. 16): mixed vs FP64 GPU treecode (the metric's condition),
    and both vs the FP64 GPU direct sum on a seeded sample of targets."""
    import torch
    phi_mx = phi_mixed.clone()
    p64 = b.params(w["degree"], w["theta"], w["leaf"], w["batch"], w["kernel"], w["kappa"],
                   b.BLTC_PRECISION_FP64)
    phi64 = torch.empty_like(phi_mx)
    t0 = time.perf_counter()
    ctx.solve(*X, p64, phi64)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    rng = np.random.default_rng(20031836)
    idx = torch.from_numpy(np.sort(rng.choice(w["n"], size=min(w["n"], 4096), replace=False))).cuda()
    T = [a.index_select(0, idx).contiguous() for a in X[:3]]
    ref = torch.empty_like(T[0])
    b.bltc_direct_sum(ctx.h, *T, *X[:3], X[3], p64, ref)
    torch.cuda.synchronize()
    # the GPU direct sum (Eq. 1) over all targets, FP32 evaluation with FP64 accumulation: the
    # time-to-solution the treecode is compared with (the FP64 direct sum over all 1e6 targets
    # would take tens of seconds on this GPU's FP64 rate, so only its sample is run)
    pmx = b.params(w["degree"], w["theta"], w["leaf"], w["batch"], w["kernel"], w["kappa"],
                   b.BLTC_PRECISION_MIXED)
    dmx = torch.empty_like(phi_mx)
    b.bltc_direct_sum(ctx.h, *T, *X[:3], X[3], pmx, ref.clone())       # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.bltc_direct_sum(ctx.h, *X[:3], *X[:3], X[3], pmx, dmx)
    e1.record()
    e1.synchronize()
    h = lambda t: t.cpu().numpy()
    e_mx_64 = rel_err(h(phi64), h(phi_mx))
    return {"mixed_vs_fp64_gpu_bltc": e_mx_64, "meets_1e-6": bool(e_mx_64 <= 1e-6),
            "fp64_bltc_vs_direct_sampled": rel_err(h(ref), h(phi64.index_select(0, idx))),
            "mixed_bltc_vs_direct_sampled": rel_err(h(ref), h(phi_mx.index_select(0, idx))),
            "fp64_gpu_bltc_seconds": t64, "direct_sample_targets": int(idx.numel()),
            "gpu_direct_sum_mixed_seconds": e0.elapsed_time(e1) * 1e-3,
            # the mixed direct sum is bound by the FMA pipe: 13 FP32 operations per evaluation
            # (three per coordinate difference from FP32 pairs, three for r^2, one accumulation)
            # against 128 per clock per SM
            "gpu_direct_sum_mixed_roofline": direct_roofline(ctx, w["n"], e0.elapsed_time(e1) * 1e-3),
            "gpu_direct_sum_mixed_vs_fp64_sampled": rel_err(h(ref), h(dmx.index_select(0, idx)))}


def direct_roofline(ctx, n, seconds):
    """The mixed direct sum's evaluations per second against its FMA-pipe bound."""
    evals = n * (n - 1)
    peak = ctx.sm_count * 128.0 / 13.0 * SM_MAX_MHZ * 1e6
    return {"bound": "alu", "pipe": "FMA (13 FP32 operations per evaluation)",
            "achieved": evals / seconds / 1e9, "peak": peak / 1e9, "unit": "G evaluations/s",
            "frac": evals / seconds / peak}


def run_e2e(ctx, b, x, y, z, q, g, B, args, dist, w):
    """The same metric end to end through the graph's public API: every timed step copies the
    step's positions and charges from pinned host memory into the graph's bound tensors,
    launches the graph (which synchronizes) and copies phi back to pinned host memory."""
    import torch
    H = [torch.from_numpy(a).pin_memory() for a in (x, y, z, q)]
    out = torch.empty(w["n"], dtype=torch.float64).pin_memory()

    def step():
        for t, h in zip(B, H):
            t.copy_(h, non_blocking=True)
        g.launch()
        out.copy_(g.phi, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    k = max(1, min(args.steps, 5))
    dist.barrier()
    times = []
    for _ in range(k):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    dist.barrier()
    t = dist.max(sum(times) / len(times))
    total = dist.sum(w["n"])
    return {"value": total / t, "unit": "targets/s", "h2d_bytes_per_step": 4 * 8 * w["n"],
            "d2h_bytes_per_step": 8 * w["n"], "steps": k, "ms_per_step": t * 1e3,
            "api": "pinned host -> bound device tensors, bltc_graph_launch, phi -> pinned host"}


# ---- serving: continuous batching of a request stream --------------------------------------

SERVE_METRIC = "served requests: targets/s at saturation; p50/p99 latency (ms) at Poisson load"


def serve_requests(count, seed=20031836 + 4):
    """The request mix: N log-uniform in [1e3, 1e6], cube or Plummer, Coulomb or Yukawa
    (kappa uniform [0.1, 1]), theta uniform [0.5, 0.8], n in {4, 6, 8, 10}, mixed precision."""
    import paper_2003_01836_gb300 as b
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(10 ** rng.uniform(3.0, 6.0)))
        kind = "cube" if rng.random() < 0.5 else "plummer"
        ker = int(rng.random() < 0.5)
        kappa = float(rng.uniform(0.1, 1.0)) if ker else 0.0
        theta = float(rng.uniform(0.5, 0.8))
        deg = int(rng.choice([4, 6, 8, 10]))
        out.append((kind, n, seed * 10000 + i,
                    b.params(deg, theta, 2000, 2000, ker, kappa, b.BLTC_PRECISION_MIXED)))
    return out


def serve_solo_time(reqs, data, dist):
    """Seconds each request takes solved alone (bltc_solve, inputs already on the device),
    one after another: the work the server batches, without the batching."""
    import torch

    import paper_2003_01836_gb300 as b
    ctx = b.Context(dist.local_rank)
    times = []
    phi = None
    seen = set()
    for (kind, n, sd, p), arrs in zip(reqs, data):
        X = [torch.from_numpy(a).cuda() for a in arrs]
        phi = torch.empty_like(X[0])
        if (p.degree, p.kernel) not in seen:       # first of its kind: kernel attributes, pool
            ctx.solve(*X, p, phi)
            seen.add((p.degree, p.kernel))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.solve(*X, p, phi)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    ctx.close()
    return np.array(times)


def run_serving(args, dist: Dist):
    from paper_2003_01836_gb300 import build
    build.build()
    return serve_measure(args.serve_requests, (0.5, 0.8, 1.0), args.serve_workers, dist,
                         args.serve_slice_us, args.serve_setup_blocks, args.serve_slices_in_flight)


def serve_measure(count, fractions, workers, dist, slice_us=15000, setup_blocks=0, slices_in_flight=0):
    """The serving runtime on the first `count` requests of the stream: all at once
    (saturated), then Poisson arrivals at each fraction of that rate; every request is also
    solved alone for the comparison."""
    import concurrent.futures as cf
    import threading

    import paper_2003_01836_gb300 as b
    from paper_2003_01836_gb300 import inputs
    reqs = serve_requests(count)

    def make(r):
        kind, n, sd, _ = r
        return [np.ascontiguousarray(a) for a in inputs.system(kind, n, sd)]

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        data = list(ex.map(make, reqs))
    total_targets = sum(r[1] for r in reqs)
    srv = b.Server(dist.local_rank, setup_workers=workers, max_batch=64, slice_us=slice_us,
                   setup_blocks=setup_blocks, slices_in_flight=slices_in_flight)
    try:
        # warm-up: a few requests
        for i in range(min(8, len(reqs))):
            srv.wait(srv.submit(*data[i], reqs[i][3]))

        def run_load(rate):
            """Submits every request (Poisson arrivals at `rate` per second, or all at once
            for rate None) and returns the wall time and per-request latencies."""
            rng = np.random.default_rng(7)
            gaps = rng.exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
            tickets = [None] * len(reqs)
            t0 = time.perf_counter()

            def submitter():
                t = t0
                for i, g in enumerate(gaps):
                    t += g
                    d = t - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    tickets[i] = srv.submit(*data[i], reqs[i][3])
            th = threading.Thread(target=submitter)
            th.start()
            lat, parts = [], []
            for i in range(len(reqs)):
                while tickets[i] is None:
                    time.sleep(0.0002)
                st, _, info = srv.wait(tickets[i])
                if st != b.BLTC_OK:
                    raise RuntimeError(f"request {i} failed with status {st}: {srv.last_error()}")
                lat.append((info["t_done"] - info["t_submit"]) * 1e3)
                parts.append(((info["t_admit"] - info["t_submit"]) * 1e3, (info["t_ready"] - info["t_admit"]) * 1e3,
                              (info["t_done"] - info["t_ready"]) * 1e3, (info["t_swept"] - info["t_ready"]) * 1e3,
                              (info["t_copy"] - info["t_swept"]) * 1e3, (info["t_done"] - info["t_copy"]) * 1e3))
            th.join()
            return time.perf_counter() - t0, np.array(lat), np.array(parts)

        wall, lat, parts = run_load(None)
        x_req = len(reqs) / wall
        runs = [("saturated (all submitted at t=0)", None, wall, lat, parts)]
        for frac in fractions:
            wall_f, lat_f, parts_f = run_load(frac * x_req)
            runs.append((f"Poisson at {frac:.1f} x saturated rate", frac * x_req, wall_f, lat_f, parts_f))
        stats = srv.stats()
    finally:
        srv.close()
    solo_each = serve_solo_time(reqs, data, dist)
    solo = float(solo_each.sum())
    levels = []
    for name, offered, wall_f, lat_f, parts_f in runs:
        slow = lat_f / (1e3 * solo_each)          # latency over the request's solo solve time
        tail = slow >= np.percentile(slow, 99)
        lv = {"load": name, "requests_per_s": len(reqs) / wall_f, "targets_per_s": total_targets / wall_f,
              "p50_ms": float(np.percentile(lat_f, 50)), "p99_ms": float(np.percentile(lat_f, 99)),
              "slowdown_p50": float(np.percentile(slow, 50)), "slowdown_p99": float(np.percentile(slow, 99)),
              # where the slowest 1% (by slowdown) spent their time: waiting for admission, in
              # setup (copy-in, tree, lists, charges, plan), and from ready to copied out
              "tail_ms": {"requests": int(tail.sum()), "n_mean": float(np.mean([reqs[i][1] for i in np.flatnonzero(tail)])),
                          "queued": float(parts_f[tail, 0].mean()), "setup": float(parts_f[tail, 1].mean()),
                          "sweep_and_copy_out": float(parts_f[tail, 2].mean()),
                          "ready_to_enqueued": float(parts_f[tail, 3].mean()),
                          "enqueued_to_complete": float(parts_f[tail, 4].mean()),
                          "copy_out": float(parts_f[tail, 5].mean()),
                          "solo": float(1e3 * solo_each[tail].mean())}}
        if offered is not None:
            lv["offered_requests_per_s"] = offered
        levels.append(lv)
    return {"metric": SERVE_METRIC, "value": levels[0]["targets_per_s"], "unit": "targets/s",
            "n_gpus": dist.world, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (f64 accumulation)", "data": "synthetic",
            "config": {"workload": "serving stream", "requests": len(reqs),
                       "total_targets": total_targets,
                       "mix": "N log-uniform [1e3,1e6]; cube|Plummer; Coulomb|Yukawa kappa U[0.1,1]; "
                              "theta U[0.5,0.8]; n in {4,6,8,10}; N_L=N_B=2000; mixed",
                       "setup_workers": workers, "max_batch": 64, "slice_us": slice_us,
                       "setup_blocks": setup_blocks, "slices_in_flight": slices_in_flight or 1},
            "levels": levels,
            "solo": {"seconds": solo, "targets_per_s": total_targets / solo,
                     "p50_ms": float(np.percentile(solo_each, 50) * 1e3),
                     "p99_ms": float(np.percentile(solo_each, 99) * 1e3),
                     "note": "every request solved alone with bltc_solve, back to back on one stream "
                             "(device inputs, CUDA events around each solve); slowdown = a request's "
                             "served latency over its solo solve time"},
            "served_vs_solo": solo / wall,
            "server": {k: stats[k] for k in ("sweep_launches", "max_batch", "peak_reserved_bytes",
                                             "peak_live_bytes", "budget_bytes")}}


# ---- cluster-particle and cluster-cluster variants -----------------------------------------------------------------

VARIANT_NAMES = {"cp": "cluster-particle", "cc": "cluster-cluster (dual tree traversal)",
                 "hermite": "barycentric Hermite"}
HERMITE_DEGREE = 4          # Hermite interpolation on n+1 = 5 points reproduces degree 2n+1 = 9


def run_variant(args, dist: Dist):
    """A variant on the same workload: cp (targets interpolated, sources exact) or cc (dual
    tree traversal, both sides interpolated); time-to-solution with inputs resident, and its
    errors next to the treecode's."""
    import torch

    import paper_2003_01836_gb300 as b
    from paper_2003_01836_gb300 import build, inputs
    build.build()
    dev = dist.local_rank
    torch.cuda.set_device(dev)
    w = dict(WORKLOAD)
    if args.n:
        w["n"] = args.n
    if args.theta >= 0:
        w["theta"] = args.theta
    x, y, z, q = inputs.system(w["kind"], w["n"], w["seed"] + dist.rank)
    X = [torch.from_numpy(a).to(f"cuda:{dev}") for a in (x, y, z, q)]
    phi = torch.empty_like(X[0])
    ctx = b.Context(dev)
    herm = args.variant == "hermite"
    if herm:
        w["degree"] = HERMITE_DEGREE
    p = b.params(w["degree"], w["theta"], w["leaf"], w["batch"], w["kernel"], w["kappa"],
                 b.BLTC_PRECISION_MIXED)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{dev}")
    if herm:
        solve = lambda pp, out: b.bltc_solve_hermite(ctx.h, *X, pp, out)
    else:
        fn = b.bltc_solve_cp if args.variant == "cp" else b.bltc_solve_cc
        solve = lambda pp, out: fn(ctx.h, *X[:3], *X, pp, out)
    name = VARIANT_NAMES[args.variant]
    for _ in range(args.warmup):
        solve(p, phi)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    step_ms = []
    launches0 = b.bltc_context_launch_count(ctx.h)
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        solve(p, phi)
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    launches = b.bltc_context_launch_count(ctx.h) - launches0
    agg = aggregate(sum(step_ms) / len(step_ms), w["n"], dist)
    out = {"metric": f"{name} variant: targets/s (time-to-solution, inputs resident)",
           "value": agg["targets_per_s"], "unit": "targets/s", "n_gpus": dist.world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": agg["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 (f64 accumulation and interpolation)", "data": "synthetic",
           "config": {"workload": f"{name} variant on " + workload_name(w), "n_particles": w["n"],
                      "theta": w["theta"], "degree": w["degree"], "leaf_size": w["leaf"],
                      "batch_size": w["batch"], "kernel": "coulomb", "precision": "mixed",
                      "l2": "flushed before every timed step (256 MiB device write)"},
           "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
           "clocks": clocks, "gpu_launches": int(launches)}
    if not args.no_check:
        p64 = b.params(w["degree"], w["theta"], w["leaf"], w["batch"], w["kernel"], w["kappa"],
                       b.BLTC_PRECISION_FP64)
        phi64 = torch.empty_like(phi)
        solve(p64, phi64)
        tree = torch.empty_like(phi)
        ctx.solve(*X, b.params(WORKLOAD["degree"], w["theta"], w["leaf"], w["batch"], w["kernel"], w["kappa"],
                               b.BLTC_PRECISION_MIXED), tree)
        rng = np.random.default_rng(20031836)
        idx = torch.from_numpy(np.sort(rng.choice(w["n"], size=min(w["n"], 4096), replace=False))).cuda()
        T = [a.index_select(0, idx).contiguous() for a in X[:3]]
        ref = torch.empty_like(T[0])
        b.bltc_direct_sum(ctx.h, *T, *X[:3], X[3], p64, ref)
        torch.cuda.synchronize()
        h = lambda t: t.cpu().numpy()
        v = args.variant
        out["error"] = {f"fp64_{v}_vs_direct_sampled": rel_err(h(ref), h(phi64.index_select(0, idx))),
                        "mixed_treecode_vs_direct_sampled": rel_err(h(ref), h(tree.index_select(0, idx))),
                        "direct_sample_targets": int(idx.numel()),
                        f"mixed_vs_fp64_gpu_{v}": rel_err(h(phi64), h(phi)),
                        f"mixed_{v}_vs_direct_sampled": rel_err(h(ref), h(phi.index_select(0, idx)))}
    ctx.close()
    return out


# ---- fixed positions, new charges: the solve replayed as one CUDA graph ---------------------

def run_graph(args, dist: Dist):
    """Iterative use: the positions stay, every step brings new charges.  The setup (trees,
    lists, plans) is built once and captured with the charge-dependent launches in one CUDA
    graph; a step writes the step's charges into the bound tensor and launches the graph."""
    import torch

    import paper_2003_01836_gb300 as b
    from paper_2003_01836_gb300 import build, inputs
    build.build()
    dev = dist.local_rank
    torch.cuda.set_device(dev)
    w = dict(WORKLOAD)
    if args.n:
        w["n"] = args.n
    if args.theta >= 0:
        w["theta"] = args.theta
    x, y, z, q = inputs.system(w["kind"], w["n"], w["seed"] + dist.rank)
    X = [torch.from_numpy(a).to(f"cuda:{dev}") for a in (x, y, z, q)]
    charges = [X[3].clone(), torch.from_numpy(np.random.default_rng(20031836 + dist.rank)
                                              .uniform(-1.0, 1.0, w["n"])).to(f"cuda:{dev}")]
    qd = X[3].clone()
    ctx = b.Context(dev)
    p = b.params(w["degree"], w["theta"], w["leaf"], w["batch"], w["kernel"], w["kappa"],
                 b.BLTC_PRECISION_MIXED)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{dev}")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = b.Graph(ctx, *X[:3], qd, p)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    for i in range(args.warmup):
        qd.copy_(charges[i % 2])
        g.launch()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    step_ms = []
    launches0 = b.bltc_context_launch_count(ctx.h)
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for i in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        qd.copy_(charges[i % 2])
        g.launch()
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    launches = b.bltc_context_launch_count(ctx.h) - launches0
    agg = aggregate(sum(step_ms) / len(step_ms), w["n"], dist)
    out = {"metric": "graph variant: re-evaluation with fixed positions and new charges, targets/s",
           "value": agg["targets_per_s"], "unit": "targets/s", "n_gpus": dist.world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": agg["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 (f64 accumulation)", "data": "synthetic",
           "config": {"workload": "solve replayed as one CUDA graph on " + workload_name(w), "n_particles": w["n"],
                      "theta": w["theta"], "degree": w["degree"], "leaf_size": w["leaf"],
                      "batch_size": w["batch"], "kernel": "coulomb", "precision": "mixed",
                      "l2": "flushed before every timed step (256 MiB device write)"},
           "setup_ms": setup_ms, "kernels_per_launch": g.kernels,
           "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
           "clocks": clocks, "gpu_launches": int(launches)}
    if not args.no_check:
        phi_g = g.phi.clone()
        ref = torch.empty_like(phi_g)
        ctx.solve(*X[:3], qd, p, ref)
        torch.cuda.synchronize()
        out["bits_equal_to_solve"] = bool(torch.equal(phi_g, ref))
    g.close()
    ctx.close()
    return out


def run_graph_positions(args, dist: Dist):
    """New positions at every step: the whole solve (tree, lists, upward pass, plan, sweep,
    finalize) sized on the device and captured as one CUDA graph.  A step copies the step's
    positions and charges into the bound tensors (two seeded systems of the workload,
    alternating) and launches the graph (one cudaGraphLaunch, one read of the overflow flag)."""
    import torch

    import paper_2003_01836_gb300 as b
    from paper_2003_01836_gb300 import build, inputs
    build.build()
    dev = dist.local_rank
    torch.cuda.set_device(dev)
    w = dict(WORKLOAD)
    if args.n:
        w["n"] = args.n
    if args.theta >= 0:
        w["theta"] = args.theta
    systems = [[torch.from_numpy(a).to(f"cuda:{dev}") for a in inputs.system(w["kind"], w["n"], w["seed"] + dist.rank + 1000 * k)]
               for k in range(2)]
    X = [t.clone() for t in systems[0]]
    ctx = b.Context(dev)
    p = b.params(w["degree"], w["theta"], w["leaf"], w["batch"], w["kernel"], w["kappa"],
                 b.BLTC_PRECISION_MIXED)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{dev}")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = b.Graph(ctx, *X[:3], X[3], p, positions=True)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)

    def load(k):
        for t, src in zip(X, systems[k]):
            t.copy_(src)

    for i in range(args.warmup):
        load(i % 2)
        g.launch()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    step_ms = []
    launches0 = b.bltc_context_launch_count(ctx.h)
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for i in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        load(i % 2)
        g.launch()
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    launches = b.bltc_context_launch_count(ctx.h) - launches0
    agg = aggregate(sum(step_ms) / len(step_ms), w["n"], dist)
    # the host-driven solve of the same systems, for comparison
    solve_ms = []
    ref = torch.empty_like(X[0])
    for i in range(args.warmup + args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.solve(*systems[i % 2], p, ref)
        e1.record()
        e1.synchronize()
        if i >= args.warmup:
            solve_ms.append(e0.elapsed_time(e1))
    info = g.info
    out = {"metric": "graph_positions variant: new positions every step, whole solve as one CUDA graph, targets/s",
           "value": agg["targets_per_s"], "unit": "targets/s", "n_gpus": dist.world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": agg["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 (f64 accumulation)", "data": "synthetic",
           "config": {"workload": "whole solve sized on the device, one CUDA graph, on " + workload_name(w),
                      "n_particles": w["n"], "theta": w["theta"], "degree": w["degree"],
                      "leaf_size": w["leaf"], "batch_size": w["batch"], "kernel": "coulomb",
                      "precision": "mixed", "systems": "two seeded draws, alternating",
                      "l2": "flushed before every timed step (256 MiB device write)"},
           "setup_ms": setup_ms, "kernels_per_launch": info["kernels"], "redone": info["redone"],
           "captures": info["captures"],
           "host_driven_solve_ms": float(np.median(solve_ms)), "step_ms": [round(t, 3) for t in step_ms],
           "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
           "clocks": clocks, "gpu_launches": int(launches)}
    if not args.no_check:
        load(1)
        g.launch()
        ctx.solve(*systems[1], p, ref)
        torch.cuda.synchronize()
        out["bits_equal_to_solve"] = bool(torch.equal(g.phi, ref))
    g.close()
    ctx.close()
    return out


# ---- reference arm: the oracle --------------------------------------------------------------

def run_reference(args, dist: Dist):
    """The oracle on the host cores, every step a bounded, measured sample of the workload:
    Algorithm 1's evaluation (ComputePotential) of eight batches per core, the batches drawn in
    turn from a seeded permutation of all of them.  The trees and modified charges are built
    once before the warm-up (their time is reported, not in the steps)."""
    if dist.rank != 0:
        return None
    from paper_2003_01836_gb300 import inputs
    import oracle
    oracle.build()
    w = dict(WORKLOAD)
    if args.n:
        w["n"] = args.n
    if args.theta >= 0:
        w["theta"] = args.theta
    x, y, z, q = inputs.system(w["kind"], w["n"], w["seed"])
    cores = os.cpu_count() or 1
    prep = oracle.Prepared(x, y, z, q, w["theta"], w["degree"], w["leaf"], w["batch"],
                           w["kernel"], w["kappa"], threads=cores)
    setup_s = prep.timings["setup"] + prep.timings["precompute"]
    st = oracle.Tree(x, y, z, w["batch"])
    counts = st.count[st.leaves]
    nl = len(counts)
    order = np.random.default_rng(20031836).permutation(nl)
    # eight batches per core: the batches' costs differ by up to 8x (leaves of ~1953 and ~250
    # targets), and with two per core the slowest core paced each step at 61% of the whole
    # solve's rate; the oracle schedules batches dynamically over its threads
    per_step = min(8 * cores, nl)

    def batches(i):
        return np.sort(np.take(order, np.arange(i * per_step, (i + 1) * per_step), mode="wrap"))

    for i in range(args.warmup):
        prep.evaluate(batches(i), threads=cores)
    times, targets = [], 0
    for i in range(args.warmup, args.warmup + args.steps):
        pick = batches(i)
        t0 = time.perf_counter()
        prep.evaluate(pick, threads=cores)
        times.append(time.perf_counter() - t0)
        targets += int(counts[pick].sum())
    prep.close()
    v = targets / sum(times)
    sample = (f"Algorithm 1's evaluation (ComputePotential) of {per_step} of the {nl} batches per step "
              f"(eight per core), drawn in turn from a seeded permutation; {targets} targets over the "
              f"timed steps; the trees and modified charges ({setup_s:.2f} s) are built once before "
              f"the warm-up and are not in the steps")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "targets/s",
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(w).replace("mixed FP32 evaluation / FP64 accumulation",
                                                         "FP64 CPU oracle"),
                       "n_particles": w["n"], "theta": w["theta"], "degree": w["degree"],
                       "leaf_size": w["leaf"], "batch_size": w["batch"]},
            "setup_s": setup_s,
            "cpu_baseline": {"value": v, "unit": "targets/s", "cores": cores,
                             "cpu_model": cpu_model(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "targets/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=0, help="override the particle count (smoke runs)")
    ap.add_argument("--theta", type=float, default=-1.0,
                    help="override theta of the main workload (profiling: 0 makes the sweep all near field)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the sub-records of the 8e6 Plummer and 2.56e8 cube configurations")
    ap.add_argument("--configs", default="1,3,5", help="which other configurations to add (1, 3, 5)")
    ap.add_argument("--error-targets5", type=int, default=0,
                    help="targets of the 2.56e8 configuration's error sample (default 2048)")
    ap.add_argument("--serving", action="store_true",
                    help="time the serving runtime on the request stream instead")
    ap.add_argument("--variant", choices=("treecode", "cp", "cc", "hermite", "graph", "graph_positions"), default="treecode",
                    help="cp / cc / hermite: time the cluster-particle, cluster-cluster or "
                         "barycentric Hermite (n = 4) variant on the same workload instead; "
                         "graph: replays with fixed positions and new charges")
    ap.add_argument("--serve-requests", type=int, default=4096)
    ap.add_argument("--serve-slice-us", type=int, default=15000,
                    help="serving engine slice length in microseconds (0: all ready work at once)")
    ap.add_argument("--serve-setup-blocks", type=int, default=0,
                    help="block slots the serving sweeps leave to requests in preparation (0: none)")
    ap.add_argument("--serve-slices-in-flight", type=int, default=0, choices=(0, 1, 2),
                    help="slices the serving engine keeps enqueued (0: the library's default)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving sub-record of the default run")
    ap.add_argument("--serve-record-requests", type=int, default=1024,
                    help="requests of the default run's serving sub-record")
    ap.add_argument("--serve-workers", type=int, default=3)
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    dist = Dist()
    try:
        if args.impl == "reference":
            out = run_reference(args, dist)
        elif args.serving:
            out = run_serving(args, dist)
        elif args.variant == "graph":
            out = run_graph(args, dist)
        elif args.variant == "graph_positions":
            out = run_graph_positions(args, dist)
        elif args.variant in ("cp", "cc", "hermite"):
            out = run_variant(args, dist)
        else:
            out = run_ours(args, dist)
        if out is not None and dist.rank == 0:
            print(json.dumps(out), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
