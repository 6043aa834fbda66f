"""Benchmark: interface-node Monte Carlo of PDD on GB300.

Workload: the 3-D elliptic problem (1/2) Lap u + b.grad u - u = F on the unit
cube, 4096 interface nodes on the 9 internal planes of a 4x4x4 split, 1e5
paths per node, dt = 1e-4, FP32 paths with FP64 reductions, Brownian-bridge
exit test.  One step = one pdd_interface_solve over the whole node set (path
kernel + per-node reduction + finalize).  Metric: path-steps per second (plus
nodes per second at the achieved standard error).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pdd|reference]

--impl reference times the FP64 CPU oracle (the slow, obviously correct
restatement of the method) on the host cores, on a bounded node/path sample of
the same workload.  Under torchrun (N ranks) the run's node list is N copies
of the 4096 nodes, copy r keyed by stream indices [r 4096, (r + 1) 4096):
rank r solves its copy (node_offset) and every step ends with the method's
one exchange, an all-gather of the per-node (count, mean, M2) triples over
NCCL; per-GPU work is fixed, so the scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1705_03666_gb300 import workloads as W  # noqa: E402

METRIC = "path-steps/sec and interface nodes/sec at fixed std error; % of FP32/INT issue peak"
UNIT = "path-steps/s"
WORKLOAD = W.workload(2)

# Algorithmic issue slots per path-step of the FP32 3-D path (three quarters
# of a Philox block -- three words per step --, 1.5 Box-Muller pairs, one
# bridge uniform from the words' spare low bits, the drift/source of the
# manufactured problem, the Euler-Maruyama update and the exit tests), each
# elementary operation or minimal transcendental sequence counted once;
# derivation in the design notes.
ALG_SLOTS_PER_PATH_STEP = 105
# Algorithmic issue slots per particle segment of the branching estimator
# (one Philox block 40, the lifetime's logarithm 2, a Box-Muller pair 10, the
# move 4, psi 3, the tree product 1).
ALG_SLOTS_PER_SEGMENT = 60
# Algorithmic issue slots per path-step of the 2-D Poisson-Fourier path
# (three quarters of a Philox block 30, word-to-uniform maps 6, a Box-Muller
# pair 10, the drift -- sine and cosine of x and y, two eight-term Chebyshev
# recurrences and two eight-term sums -- 38, the Euler update 5, the exit
# tests 14, loop control 3); the gradient adds the 16 likelihood-ratio FMAs.
ALG_SLOTS_PER_STEP_POISSON = 106
ALG_SLOTS_PER_STEP_POISSON_GRAD = 122


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def _oracle_sample(prob, nodes, node_ids, n_paths, threads):
    import oracle
    t0 = time.perf_counter()
    r = oracle.interface_solve(prob, nodes, node_ids=node_ids, seed=WORKLOAD["seed"],
                               dt=WORKLOAD["dt"], n_paths=n_paths, n_threads=threads)
    return time.perf_counter() - t0, r["total_steps"]


def cpu_baseline(api=None, dev=None, target_s: float = 12.0) -> dict:
    """The FP64 oracle on the host cores, every 64th node, paths sized so the
    run takes about target_s seconds.  With the library (api, dev) the same
    sample also gives the parity record of the timed workload: the GPU paths
    of those nodes (node_offset = their index in the full list, so the
    full run's streams) against the oracle's, path by path."""
    import oracle
    threads = os.cpu_count() or 1
    ids = np.arange(0, 4096, 64)
    nodes = WORKLOAD["nodes"][ids]
    dt_cal, steps_cal = _oracle_sample(WORKLOAD["prob"], nodes, ids, 200, threads)
    n_paths = int(max(200, min(20000, 200 * target_s / max(dt_cal, 1e-3))))
    t0 = time.perf_counter()
    o = oracle.interface_solve(WORKLOAD["prob"], nodes, node_ids=ids, seed=WORKLOAD["seed"],
                               dt=WORKLOAD["dt"], n_paths=n_paths, n_threads=threads,
                               dump_paths=api is not None)
    el, steps = time.perf_counter() - t0, o["total_steps"]
    out = {"value": steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{len(ids)} nodes (every 64th) x {n_paths} paths, dt=1e-4, FP64, "
                     f"{steps:.3e} path-steps in {el:.2f} s"}
    if api is not None:
        out["parity"] = _parity_record(api, dev, ids, n_paths, o)
    return out


def _parity_record(api, dev, ids, n_paths, o) -> dict:
    """Exit flips and per-node agreement of the benchmark's FP32 paths with
    the FP64 oracle on the sampled nodes (tests/parity.py classification)."""
    import torch
    from tests import parity
    w = WORKLOAD
    kw = dict(seed=w["seed"], dt=w["dt"], n_paths=n_paths, precision="fp32", bridge=True)
    sc, st, ex = [], [], []
    with api.Context(w["prob"], dev) as ctx:
        for i in ids:
            r = ctx.interface_solve(torch.from_numpy(w["nodes"][i:i + 1]), node_offset=int(i),
                                    dump_paths=True, **kw)
            sc.append(r["score"].cpu().numpy())
            st.append(r["steps"].cpu().numpy())
            ex.append(r["exit"].cpu().numpy())
    g = {"score": np.concatenate(sc), "steps": np.concatenate(st), "exit": np.concatenate(ex)}
    c = parity.compare_paths(g, o, prob=w["prob"], geometry="unit_cube")
    return {"sample": f"{len(ids)} nodes (every 64th) x {n_paths} paths on the timed run's "
                      "streams (node_offset = node index)",
            "exit_flip_frac": c["flip_frac"], "step_flips": c["step_flips"],
            "face_flips": c["face_flips"], "same_exit_score_mismatches": c["mismatch"],
            "max_path_rel_same_exit": c["max_path_rel"],
            "max_ratio_to_path_bound": c["max_bound_ratio"],
            "max_node_rel_same_exit": c["node_rel_max"],
            "max_node_rel_all_paths": float(np.max(np.abs(g["score"].mean(1) - o["score"].mean(1))
                                                   / np.abs(o["score"].mean(1)))),
            "node_tolerance": 1e-5,
            "path_bound": "2^-22 ((n + 8) |grad g(x_exit)| + 16 (1 + |s|)), n = exit step"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    ids = np.arange(0, 4096, 64)
    nodes = WORKLOAD["nodes"][ids]
    dt_cal, _ = _oracle_sample(WORKLOAD["prob"], nodes, ids, 100, threads)
    n_paths = int(max(100, min(20000, 100 * 6.0 / max(dt_cal, 1e-3))))  # ~6 s per step
    for _ in range(args.warmup):
        _oracle_sample(WORKLOAD["prob"], nodes, ids, n_paths, threads)
    tot_t, tot_steps = 0.0, 0
    for _ in range(args.steps):
        el, st = _oracle_sample(WORKLOAD["prob"], nodes, ids, n_paths, threads)
        tot_t += el
        tot_steps += st
    value = tot_steps / tot_t
    sample = f"{len(ids)} nodes (every 64th) x {n_paths} paths per step, dt=1e-4, FP64"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD["name"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_pdd(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_03666_gb300 import api

    from paper_1705_03666_gb300 import shard

    w = WORKLOAD
    seed = w["seed"]
    nodes_h = torch.from_numpy(w["nodes"]).pin_memory()
    nodes = nodes_h.to(dev)
    n = nodes.shape[0]
    node_offset, n_total = shard.copy_block(n, world, rank)
    n_paths = args.paths or w["n_paths"]
    kw = dict(seed=seed, dt=w["dt"], n_paths=n_paths, precision="fp32", bridge=True,
              node_offset=node_offset)

    def exchange(res):
        """The method's one exchange step (N > 1): all-gather of the per-node
        (count, mean, M2) triples of every rank's node block."""
        if world == 1:
            return None
        return shard.allgather_nodes(shard.triples(res["mean"], res["se"], res["n"]), n_total)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    ctx = api.Context(w["prob"], dev)
    out = (torch.empty(n, dtype=torch.float64, device=dev),
           torch.empty(n, dtype=torch.float64, device=dev),
           torch.empty(n, dtype=torch.int64, device=dev))
    # path-steps per step (deterministic for a given seed): one diagnostic call
    r = ctx.interface_solve(nodes, diag=True, out=out, **kw)
    steps_per_call = r["path_steps"]
    se_median = float(out[1].median())
    for _ in range(max(0, args.warmup - 1)):
        exchange(ctx.interface_solve(nodes, out=out, **kw))
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(dev.index)
    ctx.profile(True)
    ctx.profile_read()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.4)
    for i in range(args.steps):
        flush.zero_()                       # L2 flush between steps (outside the events)
        evs[i][0].record(stream)
        exchange(ctx.interface_solve(nodes, out=out, **kw))
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    kern_ms, kern_launches = ctx.profile_read()
    ctx.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_total = sum(step_ms) / 1e3
    t_max = torch.tensor([t_total], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    t_total = float(t_max.item())
    # path-steps of one step over all ranks (each rank's node copy has its own
    # streams, so its own count)
    steps_all = torch.tensor([float(steps_per_call)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(steps_all, op=dist.ReduceOp.SUM)
    steps_all = float(steps_all.item())

    # end to end through the public API with host buffers: pinned H2D of the
    # nodes and D2H of (mean, se, n) inside the timed region
    e2e_steps = max(1, min(args.steps, 2))
    host_out = [torch.empty(n, dtype=torch.float64).pin_memory(),
                torch.empty(n, dtype=torch.float64).pin_memory(),
                torch.empty(n, dtype=torch.int64).pin_memory()]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        d_nodes = nodes_h.to(dev, non_blocking=True)
        res = ctx.interface_solve(d_nodes, out=out, **kw)
        exchange(res)
        host_out[0].copy_(res["mean"], non_blocking=True)
        host_out[1].copy_(res["se"], non_blocking=True)
        host_out[2].copy_(res["n"], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    if world > 1:
        e_max = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(e_max, op=dist.ReduceOp.MAX)
        e2e_s = float(e_max.item())

    # the plain one-node-per-launch form at the same paths per node (equal SE)
    naive = None
    if not args.no_naive and world == 1:
        torch.cuda.synchronize()
        n0, n1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0.record(stream)
        rn = ctx.interface_solve_naive(nodes, seed=seed, dt=w["dt"], n_paths=n_paths)
        n1.record(stream)
        torch.cuda.synchronize()
        naive_ms = n0.elapsed_time(n1)
        naive = {"ms_per_step": naive_ms, "speedup": naive_ms / (1e3 * t_total / args.steps),
                 "median_se": float(rn["se"].median()),
                 "form": "one launch per node, one thread per path, block sums + FP64 atomics"}
    ctx.close()

    batch = None
    if not args.no_batch and world == 1:
        batch = run_batch_once(api, dev, scale=args.batch_scale)
    others = None
    if not args.no_others and world == 1:
        others = run_other_workloads(api, dev, pf_paths=args.pf_paths)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    value = args.steps * steps_all / t_total
    nodes_per_s = world * args.steps * n / t_total
    avg_kernel_s = kern_ms / 1e3 / max(1, kern_launches)
    launches_per_step = kern_launches / max(1, args.steps)
    alg_per_launch = ALG_SLOTS_PER_PATH_STEP * steps_per_call / max(1.0, launches_per_step)
    achieved = alg_per_launch / avg_kernel_s / 1e9          # G issue slots / s
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    f_mhz = clk.get("sm_mhz") or 2070.0
    peak = n_sm * 4 * 32 * f_mhz * 1e6 / 1e9                # G thread-issue slots / s
    traffic = _ncu_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w["name"] if n_paths == w["n_paths"] else
                   f"{w['name']} (profiling case: {n_paths} paths/node)",
                   "nodes": n, "paths_per_node": n_paths,
                   "dt": w["dt"], "path_precision": "fp32 paths, fp64 reductions",
                   "bridge": True, "path_steps_per_step": steps_all,
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": ("one GPU" if world == 1 else
                                   f"node blocks: {world} copies of the node list "
                                   f"({world * n} nodes, one copy per GPU by node_offset), "
                                   "all-gather of per-node (n, mean, M2) over NCCL each step")},
        "nodes_per_s": nodes_per_s, "median_se": se_median,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "G issue-slots/s", "frac": achieved / peak, "traffic": traffic,
                     "kernel": "path_kernel<EllipticManufactured, Box<3>, float>",
                     "alg_slots_per_path_step": ALG_SLOTS_PER_PATH_STEP,
                     "kernel_ms_avg": avg_kernel_s * 1e3,
                     "peak_basis": f"{n_sm} SMs x 4 warp-issue/clk x 32 lanes x {f_mhz:.0f} MHz "
                                   "(median SM clock sampled during the timed region)"},
        "clocks": clk,
        "gpu_launches": int(args.steps * (launches_per_step + 1)),
        "e2e": {"value": e2e_steps * steps_all / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(nodes_h.numel() * 8),
                "d2h_bytes_per_step": int(n * 24)},
    }
    if naive is not None:
        line["vs_naive_equal_se"] = naive
    if batch is not None:
        line["batch_adaptive"] = batch
    if others is not None:
        line["other_workloads"] = others
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(api, dev)
        line["parity"] = cb.pop("parity")
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _timed(stream, fn):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def run_other_workloads(api, dev, pf_paths=None) -> dict:
    """One timed call (after one warm-up) of each other workload at full size:
    KPP branching (1024 space-time nodes x 1e5 trees), the Poisson-Fourier
    forward solve and its gradient (2048 nodes x 1e5 paths, dt = 1e-3),
    stage two of the 2-D Laplace workload (two 129 x 129 CG solves), Walk
    on Spheres against Euler-Maruyama on that workload's 16 nodes, the KPP
    nodes with one tree per sample for all 16 times (Algorithm 3.1), the
    bounded-domain KPP problem (Eq. 3.2) on the unit square, and the 2-D
    Laplace nodes with Neumann and Robin faces (Eq. 2.4)."""
    import torch
    out = {}
    stream = torch.cuda.current_stream(dev)
    w = W.workload(4)
    with api.Context(w["prob"], dev) as ctx:
        nodes = torch.from_numpy(w["nodes"]).to(dev)
        kw = dict(seed=w["seed"], n_trees=w["n_trees"], max_particles=w["max_particles"],
                  max_depth=w["max_depth"])
        r = ctx.branching_solve(nodes, diag=True, **kw)
        ms, _ = _timed(stream, lambda: ctx.branching_solve(nodes, **kw))
        seg_s = r["segments"] / (ms / 1e3)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        out["kpp_branching"] = {"workload": w["name"], "ms": ms,
                                "trees_per_s": len(w["nodes"]) * w["n_trees"] / (ms / 1e3),
                                "segments_per_s": seg_s,
                                "nodes_per_s": len(w["nodes"]) / (ms / 1e3),
                                "median_se": float(r["se"].median()),
                                "precision": "fp32 positions, float-float tree products, "
                                             "fp64 node sums",
                                "issue_roofline_frac_at_2070mhz": ALG_SLOTS_PER_SEGMENT * seg_s
                                / (n_sm * 4 * 32 * 2070e6),
                                "alg_slots_per_segment": ALG_SLOTS_PER_SEGMENT}
        # Algorithm 3.1's time-point sharing on the same 1024 space-time
        # nodes: 64 positions x 16 times, one tree per sample for all times
        pos = torch.from_numpy(np.ascontiguousarray(w["nodes"][::16, :2])).to(dev)
        times = w["nodes"][:16, 2]
        kw_g = dict(seed=w["seed"] + 1, n_trees=w["n_trees"], max_particles=w["max_particles"],
                    max_depth=w["max_depth"])
        rg = ctx.branching_grid_solve(pos, times, diag=True, **kw_g)
        ms_g, _ = _timed(stream, lambda: ctx.branching_grid_solve(pos, times, **kw_g))
        out["kpp_time_shared"] = {
            "workload": w["name"] + " as 64 positions x 16 times", "ms": ms_g,
            "estimates_per_s": 1024 * w["n_trees"] / (ms_g / 1e3),
            "trees_per_s": 64 * w["n_trees"] / (ms_g / 1e3),
            "speedup_vs_per_node_trees": ms / ms_g,
            "median_se": float(rg["se"].median())}
    wb = W.kpp_bounded_square()
    with api.Context(wb["prob"], dev) as ctx:
        nodes = torch.from_numpy(wb["nodes"]).to(dev)
        kw_b = dict(seed=wb["seed"], n_trees=wb["n_trees"], dt=wb["dt"])
        rb = ctx.branching_grid_solve(nodes, wb["times"], diag=True, **kw_b)
        ms_b, _ = _timed(stream, lambda: ctx.branching_grid_solve(nodes, wb["times"], **kw_b))
        a = float(np.sqrt(4.0 / 3.0))
        exact = 1 - (1 + np.exp(a * wb["nodes"][:, :1] - 5 * 4.0 * wb["times"][None, :] / 6)) ** -2
        err = np.abs(rb["mean"].cpu().numpy() - exact)
        out["kpp_bounded_square"] = {
            "workload": wb["name"], "ms": ms_b,
            "trees_per_s": len(wb["nodes"]) * wb["n_trees"] / (ms_b / 1e3),
            "steps_per_s": rb["steps"] / (ms_b / 1e3),
            "steps_per_tree": rb["steps"] / (len(wb["nodes"]) * wb["n_trees"]),
            "max_abs_err_vs_travelling_wave": float(err.max()),
            "max_err_over_se": float((err / rb["se"].cpu().numpy()).max())}
    w = W.workload(5)
    with api.Context(w["prob"], dev) as ctx:
        nodes = torch.from_numpy(w["nodes"]).to(dev)
        kw = dict(seed=w["seed"], dt=w["dt"], n_paths=pf_paths or w["n_paths"])
        r = ctx.interface_solve(nodes, diag=True, precision="fp32", **kw)
        ms_f, _ = _timed(stream, lambda: ctx.interface_solve(nodes, precision="fp32", **kw))
        gout = torch.ones(len(w["nodes"]), dtype=torch.float64, device=dev)
        ctx.interface_grad(nodes, grad_out=gout, jacobian=False, **kw)
        ms_g, _ = _timed(stream, lambda: ctx.interface_grad(nodes, grad_out=gout, **kw))
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = n_sm * 4 * 32 * 2070e6
        out["poisson_fourier_gradient"] = {
            "workload": w["name"], "n_paths": kw["n_paths"], "forward_ms": ms_f,
            "gradient_ms": ms_g,
            "path_steps_per_s_forward": r["path_steps"] / (ms_f / 1e3),
            "path_steps_per_s_gradient": r["path_steps"] / (ms_g / 1e3),
            "issue_roofline_frac_forward_at_2070mhz":
                ALG_SLOTS_PER_STEP_POISSON * r["path_steps"] / (ms_f / 1e3) / peak,
            "issue_roofline_frac_gradient_at_2070mhz":
                ALG_SLOTS_PER_STEP_POISSON_GRAD * r["path_steps"] / (ms_g / 1e3) / peak,
            "alg_slots_per_path_step": {"forward": ALG_SLOTS_PER_STEP_POISSON,
                                        "gradient": ALG_SLOTS_PER_STEP_POISSON_GRAD},
            "outputs": "jacobian [2048, 80] + vjp (dtheta[64], dphi[16])"}
    w = W.workload(1)
    with api.Context(w["prob"], dev) as ctx:
        r = ctx.interface_solve(torch.from_numpy(w["nodes"]).to(dev), seed=w["seed"], dt=w["dt"],
                                n_paths=w["n_paths"], precision="fp64")
        s = torch.from_numpy(w["nodes"][:, 1]).to(dev)
        args_l = ((0.0, 0.0), (0.5, 1.0), (129, 129), 0, 1, s, r["mean"])
        args_r = ((0.5, 0.0), (1.0, 1.0), (129, 129), 0, 0, s, r["mean"])
        ctx.subdomain_solve(*args_l)
        ms, (a, bb) = _timed(stream, lambda: (ctx.subdomain_solve(*args_l),
                                              ctx.subdomain_solve(*args_r)))
        iters = a["iters"] + bb["iters"]
        alg_bytes = iters * 129 * 129 * 13 * 8
        ctx.subdomain_solve(*args_l, method="cg_mixed")
        ms_m, (am, bm) = _timed(stream, lambda: (ctx.subdomain_solve(*args_l, method="cg_mixed"),
                                                 ctx.subdomain_solve(*args_r, method="cg_mixed")))
        ctx.subdomain_solve(*args_l, method="dst")
        ms_d, (ad, bd) = _timed(stream, lambda: (ctx.subdomain_solve(*args_l, method="dst"),
                                                 ctx.subdomain_solve(*args_r, method="dst")))
        out["stage_two_cg"] = {"grids": "2 x 129 x 129", "tol": 1e-12,
                               "fp64_cg": {"ms": ms, "iterations": iters,
                                           "achieved_gbs": alg_bytes / (ms / 1e3) / 1e9},
                               "mixed_cg": {"ms": ms_m, "fp32_iterations": am["iters"] + bm["iters"],
                                            "final_resid": max(am["resid"], bm["resid"]),
                                            "max_abs_diff_vs_fp64_cg": float(max(
                                                (am["u"] - a["u"]).abs().max(),
                                                (bm["u"] - bb["u"]).abs().max()))},
                               "dst": {"ms": ms_d, "final_resid": max(ad["resid"], bd["resid"]),
                                       "max_abs_diff_vs_fp64_cg": float(max(
                                           (ad["u"] - a["u"]).abs().max(),
                                           (bd["u"] - bb["u"]).abs().max())),
                                       "method": "direct: four FP64 products of the 127 x 127 "
                                                 "sine matrices per subdomain",
                                       # 2 subdomains x 4 products x 2 P^3 flops, P = 127
                                       "gflops_fp64": 2 * 4 * 2 * 127 ** 3 / (ms_d / 1e3) / 1e9},
                               "bytes_model": "13 vector accesses per point per CG iteration",
                               "residence": "L2/shared-resident (0.27 MB per vector)"}
        # the whole two-stage method on this workload: stage one at its 16
        # nodes (1e4 FP64 paths, dt = 1e-3), spline, both 129 x 129 halves
        kw2 = dict(n_nodes=16, n_paths=w["n_paths"], dt=w["dt"], seed=w["seed"], precision="fp64")
        api.laplace_pdd_solve(ctx, **kw2)
        ms_pdd, rp = _timed(stream, lambda: api.laplace_pdd_solve(ctx, **kw2))
        ys = torch.linspace(0.0, 1.0, 129, dtype=torch.float64, device=dev)
        errs = []
        for u, x0 in ((rp["left"], 0.0), (rp["right"], 0.5)):
            xs = torch.linspace(x0, x0 + 0.5, 129, dtype=torch.float64, device=dev)
            errs.append(float((u - torch.exp(xs)[None, :] * torch.cos(ys)[:, None]).abs().max()))
        out["pdd_laplace2d_two_stage"] = {
            "workload": w["name"] + " + two 129 x 129 subdomains", "ms": ms_pdd,
            "max_abs_err_vs_exact": max(errs), "median_node_se": float(rp["se"].median())}
        # Walk on Spheres against Euler-Maruyama + bridge on the same 16 nodes,
        # 1e6 walks / paths per node in FP32: time, jumps or steps per walk, and
        # the largest error against the harmonic solution e^x cos y.
        nodes = torch.from_numpy(w["nodes"]).to(dev)
        exact = torch.exp(nodes[:, 0]) * torch.cos(nodes[:, 1])
        N = 1_000_000
        kw_w = dict(seed=w["seed"], n_paths=N, eps=1e-4, precision="fp32")
        kw_e = dict(seed=w["seed"], n_paths=N, dt=w["dt"], precision="fp32")
        rw = ctx.wos_solve(nodes, diag=True, **kw_w)
        re = ctx.interface_solve(nodes, diag=True, **kw_e)
        ms_w, _ = _timed(stream, lambda: ctx.wos_solve(nodes, **kw_w))
        ms_e, _ = _timed(stream, lambda: ctx.interface_solve(nodes, **kw_e))
        out["wos_vs_em_laplace2d"] = {
            "nodes": len(w["nodes"]), "walks_per_node": N,
            "wos": {"eps": 1e-4, "ms": ms_w, "jumps_per_walk": rw["path_steps"] / (16 * N),
                    "walks_per_s": 16 * N / (ms_w / 1e3),
                    "max_abs_err": float((rw["mean"] - exact).abs().max()),
                    "median_se": float(rw["se"].median())},
            "em_bridge": {"dt": w["dt"], "ms": ms_e, "steps_per_path": re["path_steps"] / (16 * N),
                          "paths_per_s": 16 * N / (ms_e / 1e3),
                          "max_abs_err": float((re["mean"] - exact).abs().max()),
                          "median_se": float(re["se"].median())}}
    # The whole PDD method on the 3-D problem: stage one at the benchmark's
    # 4096 nodes (1e5 FP32 paths, dt = 1e-4), then stage two -- the cubic RBF
    # interpolant on each of the 9 internal planes and 64 independent 33^3
    # subdomain solves (sine-transform defect correction to 1e-12), batched.
    w3 = W.workload(2)
    with api.Context(w3["prob"], dev) as ctx:
        nodes3 = torch.from_numpy(w3["nodes"]).to(dev)
        ms1, r1 = _timed(stream, lambda: ctx.interface_solve(
            nodes3, seed=w3["seed"], dt=w3["dt"], n_paths=w3["n_paths"], precision="fp32"))
        axis3 = np.arange(len(w3["nodes"])) % 3
        api.elliptic3d_pdd_solve(ctx, nodes3, r1["mean"], axis3)          # warm-up
        t0 = time.perf_counter()
        ms2, r2 = _timed(stream, lambda: api.elliptic3d_pdd_solve(ctx, nodes3, r1["mean"], axis3))
        wall2 = time.perf_counter() - t0
        g3 = torch.linspace(0, 1, 129, dtype=torch.float64, device=dev)
        Z, Y, X = torch.meshgrid(g3, g3, g3, indexing="ij")
        ex3 = torch.sin(np.pi * X) * torch.sin(np.pi * Y) * torch.exp(Z)
        err3 = float((r2["u"] - ex3).abs().max())
        # one subdomain's solve alone, for the kernel rates
        ctx.profile(True)
        ctx.profile_read()
        faces = {fc: torch.zeros((33, 33), dtype=torch.float64, device=dev) for fc in range(6)}
        rs = ctx.subdomain_solve3d((0.25, 0.25, 0.25), (0.5, 0.5, 0.5), (33, 33, 33), faces)
        k_ms, _ = ctx.profile_read()
        # the 64 subdomains of the split as one batched solve
        boxes64 = [((kx / 4, ky / 4, kz / 4), ((kx + 1) / 4, (ky + 1) / 4, (kz + 1) / 4), faces)
                   for kz in range(4) for ky in range(4) for kx in range(4)]
        rb64 = ctx.subdomain_solve3d_batch(boxes64, (33, 33, 33))
        kb_ms, _ = ctx.profile_read()
        ctx.profile(False)
        P = 31
        flops = rs["iters"] * (6 * 2 * P ** 4 + 40 * P ** 3)
        flops64 = sum(rb64["iters_each"]) * (6 * 2 * P ** 4 + 40 * P ** 3)
        out["pdd_elliptic3d_two_stage"] = {
            "workload": w3["name"] + " + 9 plane interpolants + 64 subdomains of 33^3 "
                        "(h = 1/128)",
            "stage_one_ms": ms1, "stage_two_ms": ms2, "stage_two_wall_s": wall2,
            "max_abs_err_vs_exact": err3, "median_node_se": float(r1["se"].median()),
            "max_corrections": r2["iters"], "max_rel_residual": r2["resid"],
            "one_subdomain": {"ms": k_ms, "corrections": rs["iters"],
                              "gflops_fp32_transforms": flops / (k_ms / 1e3) / 1e9,
                              "flop_model": "per correction 6 dense sine passes (2 P^4) + "
                                            "residual/eigenvalues/update (~40 P^3), P = 31"},
            "batch_of_64_subdomains": {"ms": kb_ms, "corrections": rb64["iters"],
                                       "gflops_fp32_transforms": flops64 / (kb_ms / 1e3) / 1e9}}
    # Multilevel estimate on the 2-D Laplace nodes (4 levels, dt 4e-3 .. 5e-4)
    # against the plain scheme at the finest dt with enough paths for the
    # same standard error.
    with api.Context(W.laplace_expcos(), dev) as ctx:
        nodes = torch.from_numpy(W.nodes_cfg1(16)).to(dev)
        exact = torch.exp(nodes[:, 0]) * torch.cos(nodes[:, 1])
        kw_m = dict(seed=W.SEED_BASE + 8, dt0=4e-3, n_per_level=[400_000, 200_000, 100_000, 50_000])
        ctx.mlmc_solve(nodes, **kw_m)
        ms_m, rm = _timed(stream, lambda: ctx.mlmc_solve(nodes, **kw_m))
        v0 = float(rm["levels"][0]["var"].mean())
        se_m = float(rm["se"].median())
        n_em = int(min(8_000_000, max(1, v0 / se_m ** 2)))
        kw_p = dict(seed=W.SEED_BASE + 9, dt=5e-4, n_paths=n_em, precision="fp32")
        ctx.interface_solve(nodes, **kw_p)
        ms_p, rpl = _timed(stream, lambda: ctx.interface_solve(nodes, **kw_p))
        out["mlmc_laplace2d"] = {
            "nodes": 16, "levels": "dt 4e-3, 2e-3, 1e-3, 5e-4; 4e5, 2e5, 1e5, 5e4 pairs",
            "mlmc": {"ms": ms_m, "median_se": se_m,
                     "max_abs_err": float((rm["mean"] - exact).abs().max()),
                     "level_var": [float(L["var"].mean()) for L in rm["levels"]]},
            "plain_em_dt5e-4": {"ms": ms_p, "paths": n_em, "median_se": float(rpl["se"].median()),
                                "max_abs_err": float((rpl["mean"] - exact).abs().max())},
            "speedup_equal_se": ms_p / ms_m}
    # Mixed boundary conditions (Eq. 2.4): face y = 0 Neumann and face
    # x = 1 Robin (phi = -2), e^x cos y exact, on the same 16 nodes.
    wr = W.laplace_expcos(reflect=[1, 2], phi=-2.0)
    with api.Context(wr, dev) as ctx:
        nodes = torch.from_numpy(W.nodes_cfg1(16)).to(dev)
        exact = torch.exp(nodes[:, 0]) * torch.cos(nodes[:, 1])
        kw_r = dict(seed=W.SEED_BASE + 7, n_paths=1_000_000, dt=1e-3, precision="fp32")
        rr = ctx.interface_solve(nodes, diag=True, **kw_r)
        ms_r, _ = _timed(stream, lambda: ctx.interface_solve(nodes, **kw_r))
        out["laplace2d_robin_faces"] = {
            "faces": "y = 0 Neumann, x = 1 Robin phi = -2, others Dirichlet",
            "nodes": 16, "paths_per_node": 1_000_000, "dt": 1e-3, "ms": ms_r,
            "path_steps_per_s": rr["path_steps"] / (ms_r / 1e3),
            "steps_per_path": rr["path_steps"] / 16e6,
            "max_abs_err": float((rr["mean"] - exact).abs().max()),
            "median_se": float(rr["se"].median())}
    return out


def run_batch_once(api, dev, scale: float = 1.0) -> dict:
    """The heterogeneous adaptive batch (unit square / L-shape / unit cube,
    per-node dt in {1e-3, 1e-4}), at full scale by default (target SE 1e-4,
    n_max = 1e6), or reduced: target SE 1e-4/sqrt(scale), n_max = 1e6 * scale;
    one warm-up call builds and replays the graph, one timed replay.  Reports
    nodes/s over all nodes and over the nodes that reached the target SE."""
    import torch
    w = W.workload(3)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        ctx = api.Context(w["problems"][0], dev)
        kw = dict(seed=w["seed"], n_pilot=w["n_pilot"], n_min=w["n_min"],
                  n_max=int(w["n_max"] * scale), target_se=w["target_se"] / scale ** 0.5,
                  use_graph=True)
        args = (w["problems"], torch.from_numpy(w["nodes"]).to(dev),
                torch.from_numpy(w["problem_index"]).to(dev), torch.from_numpy(w["dt"]).to(dev))
        r = ctx.batch_solve(*args, diag=True, **kw)   # capture + replay, counts steps
        steps = r["path_steps"]
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        r = ctx.batch_solve(*args, **kw)               # graph replay
        b1.record(stream)
        stream.synchronize()
        ms = b0.elapsed_time(b1)
        npaths = r["n"].double()
        se = r["se"]
        at_target = int((se <= kw["target_se"]).sum())
        out = {"workload": w["name"] + (f" at scale {scale}" if scale != 1.0 else " (full scale)"),
               "ms": ms,
               "path_steps": steps, "path_steps_per_s": steps / (ms / 1e3),
               "nodes": int(r["n"].numel()), "nodes_per_s": r["n"].numel() / (ms / 1e3),
               "nodes_at_target_se": at_target,
               "nodes_per_s_at_target_se": at_target / (ms / 1e3),
               "nodes_at_n_max": int((r["n"] >= kw["n_max"]).sum()),
               "paths": float(npaths.sum()), "median_se": float(se.median()),
               "target_se": kw["target_se"], "n_max": kw["n_max"],
               "launch": "pilot + main persistent launches in one captured CUDA graph"}
        ctx.close()
    return out


KERNEL_SOURCES = ("paper_1705_03666_gb300/csrc/path_kernel.cuh",
                  "paper_1705_03666_gb300/csrc/models.cuh",
                  "paper_1705_03666_gb300/csrc/common.cuh",
                  "paper_1705_03666_gb300/csrc/nodefix.cuh")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic():
    """DRAM bytes per launch of the path kernel from the committed ncu
    summary, while the kernel sources are the ones it was measured on (None
    otherwise)."""
    p = os.path.join(ROOT, "profiles", "path_kernel_elliptic3d_4096x1e5_dram.md")
    try:
        fields = {}
        with open(p) as f:
            for line in f:
                if ":" in line and not line.startswith(("#", "|", " ")):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("kernel_source_sha1") != kernel_source_hash():
            return None
        return int(fields["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pdd", "reference"], default="pdd")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-naive", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-others", action="store_true")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="scale of the adaptive batch (1.0: SE* = 1e-4, n_max = 1e6)")
    ap.add_argument("--paths", type=int, default=None,
                    help="paths per node (profiling runs only; the benchmark uses 1e5)")
    ap.add_argument("--pf-paths", type=int, default=None,
                    help="paths per node of the Poisson-Fourier forward/gradient workload "
                         "(profiling runs only; the benchmark uses 1e5)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_pdd(args)


if __name__ == "__main__":
    main()
