#!/usr/bin/env python
"""Benchmark of the neural-preconditioned solve on one GB300 (or N replicas).

Metric: solves/sec (and s/solve) to true relative residual 1e-8 for the mixed
batched workload: 256 instances on grids of 32^3, 48^3 and 64^3 Q1 elements
(mixed uniformly), seeded random binary trees of 7-255 segments with 8 P1
elements each, radius U(0.01, 0.03), coupling beta log-uniform in [1, 100],
f ~ N(0,1), g = 1, solved together by FGMRES(30) with the block
preconditioner and the BF16 network; Jacobi-CG (FP64) on the same batch and
GPU is reported beside it, with per-instance p50/p99 times.  The 100-instance
binary-tree workload at 32^3 (15 segments, beta = 1) is measured as well and
reported under "other_workloads".

A step is one batched solve of the whole workload from x0 = 0.  Inputs are
resident in HBM for `value`; `e2e` copies b from pinned host memory and x
back every step.  The working set (Krylov bases of all instances, > 1 GB)
exceeds L2, and L2 is also flushed between steps.

Block order: both orders of the preconditioner are built; each workload runs
the one that solves it faster on the GPU (stated in config.prec_order): the
paper's upper-triangular order on the beta = 1 tree workload, the lower one
on the beta-mixed and transfer workloads.

--impl reference times the FP64 CPU oracle (the plain restatement of the
method, test infrastructure) on the host cores instead, one instance per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import mdgen  # noqa: E402

WORKLOAD = "batch256_mixed"
TOL = 1e-8
RESTART = 30
HIDDEN_FLOP_PER_NODE = 4 * 2 * 27 * 32 * 32     # the four 32->32 layers
METRIC = "solves/sec and s/solve to rel. residual 1e-8, CNN-FGMRES vs Jacobi-CG, 1 GB300"
# DRAM bytes (read + write) per grid node of one hidden-layer launch, from an
# ncu capture of the hidden convolution on 64 grids of 33^3 (traffic grows with
# the grid nodes a launch processes)
HIDDEN_TRAFFIC_BYTES_PER_NODE = 153.0
NET_FLOP_PER_NODE = 2 * 27 * (3 * 32 + 4 * 32 * 32 + 32)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d["bf16_tflops_sustained"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


WORKLOAD_TEXT = {
    "tree15_32": "seeded binary trees (15 segments, 8 el/seg), N=32, beta=1, f~N(0,1), g=1",
    "batch256_mixed": "seeded binary trees (7-255 segments), N in {32,48,64}, beta log-uniform [1,100], "
                      "R~U(.01,.03), f~N(0,1), g=1",
    "transfer_64": "seeded binary trees (31-127 segments, 16 el/seg), N=64, beta in {1,10,100}, R~U(.005,.02), "
                   "f~N(0,1), g=1; network trained at N<=32",
    "transfer_128": "seeded binary trees (31-127 segments, 16 el/seg), N=128, beta in {1,10,100}, R~U(.005,.02), "
                    "f~N(0,1), g=1; network trained at N<=32",
    "paper_21": "the paper's setting: seeded binary trees (1-127 segments, 8 el/seg), N=20 (21^3 nodes), natural "
                "conditions on the cube, k=sigma=1e-3, R=eps=1e-3, coupling 2 pi eps, u=1 at the root, no source; "
                "FGMRES(20), tol 1e-12",
}
DEFAULT_COUNT = {"tree15_32": 100, "batch256_mixed": 256, "transfer_64": 30, "transfer_128": 12, "paper_21": 30}
# the faster block order per workload (measured on the GPU)
DEFAULT_ORDER = {"tree15_32": "upper", "batch256_mixed": "lower", "transfer_64": "lower", "transfer_128": "lower",
                 "paper_21": "upper"}
# relative residual the solves stop at: 1e-8 (the metric), but 1e-12 for the
# paper's setting, whose tolerance of 1e-15 lies at the FP64 rounding floor
# of the true residual of those systems
WORKLOAD_TOL = {"paper_21": 1e-12}
# the paper's setting: its network and its 3D block solve (three inner
# P-FGMRES steps, Section 6)
PAPER_SETTING = {"paper_21"}
DEFAULT_INNER = {"paper_21": 3}


def tol_of(workload: str) -> float:
    return WORKLOAD_TOL.get(workload, TOL)


def network_params(workload: str, order: str):
    """The shipped network for the workload's setting and block order."""
    from paper_2505_08491_gb300.weights import default_network_params, paper_network_params
    return paper_network_params() if workload in PAPER_SETTING else default_network_params(order)


def make_operators(insts):
    """The library operators of workload instances (their physics, if any),
    assembled side by side on the host cores."""
    from paper_2505_08491_gb300 import assemble
    return assemble([(w["N"], w["graph"], w["beta"], w.get("physics", {})) for w in insts])


def restart_of(workload: str) -> int:
    return int(mdgen.WORKLOADS[workload].get("restart", RESTART))


def instances(workload: str, rank: int, count: int):
    """The instances rank `rank` solves: a disjoint block of `count` seeded
    instances per rank (weak scaling: every rank holds the same amount)."""
    return [mdgen.workload_instance(workload, rank * count + i) for i in range(count)]


def job_throughput(local_ms: float, local_solves: int, world: int, device, dist=None):
    """Whole-job solves/s from every rank's timed milliseconds and solve count:
    the slowest rank's time (MAX) and the solves of all ranks (SUM).
    Returns (max_ms, total_solves, solves_per_s)."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    n = torch.tensor([float(local_solves)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    max_ms, total = float(t.item()), int(round(n.item()))
    return max_ms, total, total / (max_ms / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


_ORACLE_CACHE = {}


def _oracle_problem(inst):
    """The oracle's assembled problem and right-hand side of an instance
    (cached: the reference arm returns to the same few instances)."""
    from oracle import fem
    key = (inst["N"], inst["f_seed"], float(inst["beta"]), len(inst["graph"]["edges"]))
    if key not in _ORACLE_CACHE:
        p = fem.Problem(inst["N"], inst["graph"], inst["beta"], **inst.get("physics", {}))
        _ORACLE_CACHE[key] = (p, p.rhs(p.source(inst["f_seed"]), inst["g"]))
    return _ORACLE_CACHE[key]


def oracle_solve_seconds(inst, params_flat, max_seconds=None, order="upper", smooth=(0, 1.0), inner=0,
                         restart=RESTART, tol=TOL):
    """Oracle FGMRES(restart) + network (FP64 CPU) on one instance.  Returns
    (seconds, iterations, relres, completed).  With max_seconds, one iteration
    is timed first and then as many as fit the budget, from x0 = 0 again."""
    from oracle import solvers
    from paper_2505_08491_gb300.weights import flat_to_layers
    layers = [(W, b) for W, b in flat_to_layers(params_flat)]
    p, b = _oracle_problem(inst)
    Q = solvers.BlockPreconditioner(p, mode="cnn", params=layers, bf16=True, order=order, smooth=smooth, inner=inner)
    t0 = time.perf_counter()
    if max_seconds is None:
        x, it, rel = solvers.fgmres(p.A, b, Q, tol, restart=restart, maxit=5000)
        return time.perf_counter() - t0, it, rel, True
    x, it, rel = solvers.fgmres(p.A, b, Q, tol, restart=restart, maxit=1)
    t1 = time.perf_counter() - t0
    n_more = max(1, min(200, int((max_seconds - t1) / max(t1, 1e-3))))
    t0 = time.perf_counter()
    x, it, rel = solvers.fgmres(p.A, b, Q, tol, restart=restart, maxit=n_more)
    return time.perf_counter() - t0, it, rel, rel <= tol


def oracle_threads() -> int:
    """Threads the oracle runs on: its network and Krylov arithmetic are numpy
    and scipy calls, whose BLAS uses its thread pool (the core count unless an
    environment variable caps it)."""
    try:
        from threadpoolctl import threadpool_info
        n = [int(i.get("num_threads", 0)) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and max(n) > 0:
            return max(n)
    except ImportError:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(var, "")
        if v.isdigit() and int(v) > 0:
            return int(v)
    return os.cpu_count() or 1


def oracle_other_solvers(inst, direct: bool, tol: float = TOL):
    """The oracle's other solvers on one instance, for context beside the
    network-preconditioned one: FP64 Jacobi-CG to the same tolerance and,
    when asked, the sparse direct solve (seconds per solve)."""
    from oracle import solvers
    p, b = _oracle_problem(inst)
    t0 = time.perf_counter()
    _, it, rel = solvers.jacobi_cg(p.A, b, tol)
    out = {"jacobi_cg": {"s_per_solve": time.perf_counter() - t0, "iterations": it, "relres": rel}}
    if direct:
        t0 = time.perf_counter()
        solvers.direct_solve(p.A, b)
        out["sparse_direct"] = {"s_per_solve": time.perf_counter() - t0}
    return out


def by_group(keys, its):
    """Mean iterations per distinct key (beta or N), keys rounded for beta log-uniform draws."""
    groups = {}
    for k, it in zip(keys, its):
        kk = k if isinstance(k, int) or len(set(keys)) <= 4 else (1 if k < 3 else (10 if k < 30 else 100))
        groups.setdefault(str(kk), []).append(it)
    return {k: float(np.mean(v)) for k, v in sorted(groups.items(), key=lambda kv: float(kv[0]))}


def bench_config(args, grid_nodes):
    return {"workload": f"{args.workload}: {args.count} {WORKLOAD_TEXT[args.workload]}; one batched "
                        f"FGMRES({restart_of(args.workload)}) solve per step, BF16 network, "
                        f"tol {tol_of(args.workload):g} (true FP64 residual)",
            "instances_per_gpu": args.count, "grid_nodes_per_gpu": grid_nodes,
            "prec_order": getattr(args, "prec_order", "upper"),
            "jacobi_smoothing": {"sweeps_before_and_after": args.smooth, "omega": args.omega},
            "inner_fgmres_steps": args.inner,
            "l2": "working set > L2, 256 MB flush between steps", "precision":
            "network bf16/fp32-acc, Krylov fp32, restart residual + Hessenberg fp64"}


REFERENCE_ITERATIONS_PER_STEP = 2
REFERENCE_PER_GRID = 3


def _reference_sample(workload: str, count: int):
    """Instances the reference arm cycles through: the first three of each
    grid size among the workload's instances (all of them for one size)."""
    picked, seen = [], {}
    for i in range(count):
        w = mdgen.workload_instance(workload, i)
        if seen.get(w["N"], 0) < REFERENCE_PER_GRID:
            seen[w["N"]] = seen.get(w["N"], 0) + 1
            picked.append((i, w))
        if len(picked) >= 3 * REFERENCE_PER_GRID:
            break
    return picked


def reference_arm(args):
    """The oracle (FP64 numpy/scipy, as it stands) on the host cores, on this
    workload.  Each step is a bounded sample: the next of a few instances of
    the workload (three per grid size), the oracle's FGMRES with the network
    for 2 iterations from x0 = 0, its time per iteration times the iterations
    the instance needs to tol 1e-8, extrapolated from the residual reduction
    those iterations reached (it * log(tol) / log(relres)); the first
    iterations of GMRES reduce the residual fastest, so the extrapolation
    errs in the oracle's favour."""
    import math
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    params = network_params(args.workload, args.prec_order)
    sample = _reference_sample(args.workload, args.count)
    rs = restart_of(args.workload)
    tol = tol_of(args.workload)
    kw = dict(order=args.prec_order, smooth=(args.smooth, args.omega), inner=args.inner, restart=rs)

    def run(inst, iters):
        from oracle import solvers
        from paper_2505_08491_gb300.weights import flat_to_layers
        p, b = _oracle_problem(inst)
        Q = solvers.BlockPreconditioner(p, mode="cnn", params=flat_to_layers(params), bf16=True, order=kw["order"],
                                        smooth=kw["smooth"], inner=kw["inner"])
        t0 = time.perf_counter()
        _, it, rel = solvers.fgmres(p.A, b, Q, tol, restart=rs, maxit=iters)
        return time.perf_counter() - t0, it, rel

    for w in range(args.warmup):
        run(sample[w % len(sample)][1], 1)
    ts, rows = [], []
    for k in range(args.steps):
        idx, inst = sample[k % len(sample)]
        t, it, rel = run(inst, REFERENCE_ITERATIONS_PER_STEP)
        need = it if rel <= tol else (it * math.log(tol) / math.log(rel) if 0.0 < rel < 1.0 else float("inf"))
        ts.append(t / max(it, 1) * need)
        rows.append((idx, inst["N"], it, float(rel), round(need, 1)))
    total = sum(ts)
    value = args.steps / total
    cores = oracle_threads()
    inst0 = sample[0][1]
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, sum((w["N"] + 1) ** 3 for w in instances(args.workload, 0, args.count))),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step, the next of {len(sample)} instances of the workload (three per "
                                       f"grid size): FP64 oracle FGMRES({rs}) + network for "
                                       f"{REFERENCE_ITERATIONS_PER_STEP} iterations, time per iteration x the "
                                       "iterations to tol 1e-8 extrapolated from their residual reduction "
                                       "(favours the oracle); (instance, N, iterations run, relres, iterations "
                                       f"needed): {rows}; BLAS threads: {cores}",
                             "other_oracle_solvers": oracle_other_solvers(inst0, direct=inst0["N"] <= 32, tol=tol)},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def network_only(args):
    """The network alone on `--net-batch` grids of `--net-n`^3 nodes, `--passes`
    forward passes (random weights and inputs): the convolution kernels in
    isolation, for profiling them.  Prints one JSON line."""
    import torch

    from paper_2505_08491_gb300 import Network
    from paper_2505_08491_gb300.weights import random_params
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    net = Network(random_params(1))
    n = args.net_n
    X = torch.from_numpy(np.random.default_rng(0).standard_normal((args.net_batch, 3, n, n, n)).astype(np.float32)).cuda()
    times = []
    for _ in range(args.passes):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Y = net.forward(X)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    nodes = args.net_batch * n ** 3
    best = min(times[1:]) if len(times) > 1 else times[0]
    print(json.dumps({"network_only": {"grids": args.net_batch, "nodes_per_edge": n, "passes": args.passes,
                                       "ms_per_pass_incl_workspace": times,
                                       "network_tflops_best": nodes * NET_FLOP_PER_NODE / best / 1e9,
                                       "output_mean_abs": float(Y.abs().mean())}}), flush=True)


# the paper's batched U-net forward on its V100 (2 x 21^3 inputs; its Table 11)
PAPER_UNET_FORWARD_MS = {1: 1.5, 100: 25.5}


def unet_flops(n: int) -> float:
    """Multiply-adds x 2 of one U3 forward on an n^3 grid (the md_unet layers)."""
    m1, m2 = n // 2, n // 2 // 2
    v0, v1, v2 = n ** 3, m1 ** 3, m2 ** 3
    conv = 27 * (2 * 32 * v0 + 32 * 64 * v1 + 64 * 128 * v2 + 128 * 128 * v2 + 128 * 64 * v1 + 64 * 32 * v0 + 32 * v0)
    up = 128 * 64 * (2 * m2) ** 3 + 64 * 32 * (2 * m1) ** 3
    return 2.0 * (conv + up)


def unet_forward(args):
    """The U-net U3 forward alone, batched (random weights, N(0,1) inputs of
    2 x n^3), timed with CUDA events after warm-up: batches of 1 and 100 at
    the paper's 21^3 (its Table 11 measures the same on a V100).  Prints one
    JSON line."""
    import torch

    from paper_2505_08491_gb300 import UNet
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2505_08491_gb300.weights import unet_random_params
    rng = np.random.default_rng(0)
    n = args.net_n if args.net_n != 33 else 21
    net = UNet(unet_random_params(0))
    out = {"nodes_per_edge": n, "flop_per_sample": unet_flops(n), "batches": {}}
    for batch in (1, 100):
        X = torch.from_numpy(rng.standard_normal((batch, 2, n, n, n)).astype(np.float32)).cuda()
        for _ in range(3):
            net.forward(X)
        reps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            Y = net.forward(X)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out["batches"][str(batch)] = {"ms_per_forward": ms, "ms_per_sample": ms / batch,
                                      "tflops": batch * unet_flops(n) / ms / 1e9,
                                      "paper_v100_ms": PAPER_UNET_FORWARD_MS.get(batch) if n == 21 else None,
                                      "output_mean_abs": float(Y.abs().mean())}
    net.close()
    print(json.dumps({"unet_forward": out}), flush=True)


def extra_workload(name: str, steps: int, flush, unet_params=None):
    """Solves/s of another workload on this GPU, measured like the headline
    (inputs resident, L2 flushed, CUDA events around each batched solve), with
    Jacobi-CG on the same batch beside it.  unet_params: the U-net (one
    application per iteration) as the 3D block solve instead of the CNN.
    Rank 0 of a one-GPU run only."""
    import torch

    from paper_2505_08491_gb300 import Batch, Network, Operator, UNet
    order = DEFAULT_ORDER[name]
    inner = DEFAULT_INNER.get(name, 0) if unet_params is None else 0
    tol = tol_of(name)
    insts = instances(name, 0, DEFAULT_COUNT[name])
    ops = make_operators(insts)
    b_all = torch.cat([op.rhs(torch.from_numpy(f).cuda() if f is not None else None, w["g"])
                       for w, op, f in ((w, op, mdgen.interior_source(w["N"], w["f_seed"]))
                                        for w, op in zip(insts, ops))]).contiguous()
    x_all = torch.zeros_like(b_all)
    stream = torch.cuda.current_stream()
    out = {"workload": f"{name}: {len(insts)} {WORKLOAD_TEXT[name]}", "prec_order": order, "tol": tol,
           "inner_fgmres_steps": inner, "network": "unet" if unet_params is not None else "cnn"}
    un = None
    # a U-net that leaves an instance stalled would otherwise run 1e5 iterations per step
    maxit = 100000 if unet_params is None else 20000
    for solver in ("fgmres_cnn", "cg_jacobi"):
        if solver == "fgmres_cnn":
            net = Network(network_params(name, order))
            B = Batch(ops, solver, net, restart=restart_of(name))
            B.set_prec_order(order)
            if inner:
                B.set_inner_iters(inner)
            if unet_params is not None:
                un = UNet(unet_params)
                B.set_unet(un)
        else:
            B = Batch(ops, solver)
        for _ in range(3):
            x_all.zero_()
            B.solve(b_all, x_all, tol=tol, maxit=maxit)
        ms = 0.0
        for _ in range(steps):
            flush.zero_()
            x_all.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            its, rels, ok = B.solve(b_all, x_all, tol=tol, maxit=maxit)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        out[solver] = {"solves_per_s": len(insts) * steps / (ms / 1e3), "mean_iterations": float(np.mean(its)),
                       "max_iterations": int(np.max(its)), "max_relres": float(max(rels)),
                       "converged": int(sum(1 for r in rels if r <= tol)), "instances": len(insts)}
        B.close()
        if un is not None:
            un.close()
            un = None
    out["speedup_fgmres_cnn_over_cg"] = out["fgmres_cnn"]["solves_per_s"] / out["cg_jacobi"]["solves_per_s"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--count", type=int, default=None, help="instances per GPU (default: the workload's)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--prec-order", default=None, choices=["upper", "lower"],
                    help="block order of the preconditioner (default: the faster one for the workload)")
    ap.add_argument("--smooth", type=int, default=0,
                    help="damped Jacobi sweeps before and after the network in the 3D solve (0: none)")
    ap.add_argument("--omega", type=float, default=None, help="damping of those sweeps (default: the package's SMOOTH_OMEGA, 2/3)")
    ap.add_argument("--inner", type=int, default=None,
                    help="the 3D block solve as this many inner FGMRES steps with the network (0: one application; "
                         "default: 3 for the paper's setting, as in its Section 6, else 0)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workload measurements")
    ap.add_argument("--weights", default=None, help="network file to use instead of the shipped one for the order")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-driven restart cycles instead of one graph launch per solve (for kernel profilers, "
                         "which cannot profile kernels inside conditional graph nodes)")
    ap.add_argument("--network-only", action="store_true",
                    help="run only the network's forward pass (profiling the convolutions)")
    ap.add_argument("--net-batch", type=int, default=16, help="--network-only: grids per pass")
    ap.add_argument("--net-n", type=int, default=33, help="--network-only: grid nodes per edge")
    ap.add_argument("--passes", type=int, default=4, help="--network-only: forward passes")
    ap.add_argument("--unet-forward", action="store_true",
                    help="time the U-net U3 forward alone, batches of 1 and 100 at 21^3 (or --net-n)")
    args = ap.parse_args()
    if args.network_only:
        return network_only(args)
    if args.unet_forward:
        return unet_forward(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.count is None:
        args.count = DEFAULT_COUNT[args.workload]
    if args.prec_order is None:
        args.prec_order = DEFAULT_ORDER[args.workload]
    if args.inner is None:
        args.inner = DEFAULT_INNER.get(args.workload, 0)
    if args.omega is None:
        from paper_2505_08491_gb300 import SMOOTH_OMEGA
        args.omega = SMOOTH_OMEGA
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import torch.distributed as dist

    from paper_2505_08491_gb300 import Batch, Network
    from paper_2505_08491_gb300.weights import read_network_file

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    insts = instances(args.workload, rank, args.count)
    torch.cuda.synchronize()
    t_asm = time.perf_counter()
    ops = make_operators(insts)
    torch.cuda.synchronize()
    assembly_s = (time.perf_counter() - t_asm) / len(ops)
    params = network_params(args.workload, args.prec_order) if not args.weights else read_network_file(args.weights)
    net = Network(params)
    bs = []
    for w, op in zip(insts, ops):
        f = mdgen.interior_source(w["N"], w["f_seed"])
        bs.append(op.rhs(torch.from_numpy(f).cuda() if f is not None else None, w["g"]))
    b_all = torch.cat(bs).contiguous()
    x_all = torch.zeros_like(b_all)
    B = Batch(ops, "fgmres_cnn", net, restart=restart_of(args.workload))
    B.set_prec_order(args.prec_order)
    B.set_smoothing(args.smooth, args.omega)
    B.set_inner_iters(args.inner)
    B.set_host_loop(args.host_loop)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    tol = tol_of(args.workload)
    # the timed solves record device timestamps (the time breakdown); the graph
    # with them is captured by the warm-up solves, outside the timed region
    B.set_profiling(True)
    for _ in range(args.warmup):
        x_all.zero_()
        B.solve(b_all, x_all, tol=tol)
    B.reset_stats()
    clocks = ClockSampler(local)
    clocks.start()
    total_ms = 0.0
    its_all, rel_all = [], []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        x_all.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its, rels, ok = B.solve(b_all, x_all, tol=tol)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        its_all.append(its)
        rel_all.append(max(rels))
        lat = B.times()
        if not ok:
            raise SystemExit(f"solve did not converge: max relres {max(rels):.3e}")
    barrier()
    clk = clocks.stop()
    stats = B.stats()
    B.set_profiling(False)
    total_ms, _, value = job_throughput(total_ms, args.count * args.steps, world, "cuda", dist)
    ms_per_step = total_ms / args.steps

    # end to end through the public API: pinned host b in, x out, every step
    b_host = b_all.cpu().pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    b_dev = torch.empty_like(b_all)
    # the solve graph without the device timestamps is captured once, untimed
    b_dev.copy_(b_host, non_blocking=True)
    x_all.zero_()
    B.solve(b_dev, x_all, tol=tol)
    barrier()
    e2e_ms = 0.0
    e2e_parts = [0.0, 0.0, 0.0]  # b in, solve (with its result read), x out
    for _ in range(args.steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        b_dev.copy_(b_host, non_blocking=True)
        ev[1].record(stream)
        x_all.zero_()
        B.solve(b_dev, x_all, tol=tol)
        ev[2].record(stream)
        x_host.copy_(x_all, non_blocking=True)
        ev[3].record(stream)
        ev[3].synchronize()
        e2e_ms += ev[0].elapsed_time(ev[3])
        for k in range(3):
            e2e_parts[k] += ev[k].elapsed_time(ev[k + 1])
    _, _, e2e_value = job_throughput(e2e_ms, args.count * args.steps, world, "cuda", dist)

    # Jacobi-CG on the same batch and GPU
    cg = None
    if not args.no_cg:
        Bc = Batch(ops, "cg_jacobi")
        x_all.zero_()
        Bc.solve(b_all, x_all, tol=tol, maxit=100000)
        barrier()
        cg_ms = 0.0
        cg_its = None
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            x_all.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cg_its, cg_rel, cg_ok = Bc.solve(b_all, x_all, tol=tol, maxit=100000)
            e1.record(stream)
            e1.synchronize()
            cg_ms += e0.elapsed_time(e1)
        reps = max(1, min(args.steps, 3))
        cg_value = args.count / (cg_ms / reps / 1e3)
        cg = {"solves_per_s": cg_value, "s_per_solve_batched": cg_ms / reps / 1e3 / args.count,
              "mean_iterations": float(np.mean(cg_its)), "converged": bool(cg_ok),
              "iterations_by_beta": by_group([w["beta"] for w in insts], cg_its),
              "speedup_fgmres_cnn_over_cg": value / world / cg_value}
        Bc.close()

    other = None
    if rank == 0 and world == 1 and not args.no_extra:
        other = {name: extra_workload(name, max(1, min(args.steps, 5)), flush)
                 for name in ("tree15_32", "paper_21") if name != args.workload}
        from paper_2505_08491_gb300.weights import paper_unet_params
        up = paper_unet_params()
        if up is not None:
            other["paper_21_unet"] = extra_workload("paper_21", max(1, min(args.steps, 5)), flush, unet_params=up)

    pk = peaks()
    launches = stats["conv_hidden_launches"]
    nodes_total = sum(op.n3 for op in ops)
    flops = stats["precond_nodes"] * HIDDEN_FLOP_PER_NODE
    conv_s = stats["conv_hidden_ms"] / 1e3
    achieved = flops / conv_s / 1e12 if conv_s > 0 else 0.0
    traffic = HIDDEN_TRAFFIC_BYTES_PER_NODE * stats["precond_nodes"] * 4 / max(launches, 1)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                "frac": achieved / pk["bf16_tflops_sustained"], "traffic": traffic,
                "kernel": "hidden 3x3x3 32->32 convolutions (4 per network application)",
                "launches": launches, "avg_launch_ms": stats["conv_hidden_ms"] / max(launches, 1),
                "traffic_note": "bytes per launch (average over the timed launches, like achieved): "
                                "153 B/node measured by ncu on 64 grids of 33^3, scaled by the nodes processed",
                "peak_source": pk["source"] + " bf16 dense, sustained"}
    breakdown = {k: stats[k] for k in ("prec_ms", "conv_hidden_ms", "apply_ms", "arnoldi_ms", "restart_ms")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        its0 = its_all[-1][0]
        t, it, rel, done = oracle_solve_seconds(insts[0], params, max_seconds=20.0, order=args.prec_order,
                                                smooth=(args.smooth, args.omega), inner=args.inner,
                                                restart=restart_of(args.workload), tol=tol)
        per_it = t / max(it, 1)
        cpu = {"value": 1.0 / (per_it * its0), "unit": "solves/s", "cores": oracle_threads(), "kind": "oracle",
               "sample": f"instance 0 (N={insts[0]['N']}), FP64 oracle FGMRES({restart_of(args.workload)})+network: "
                         f"{it} iterations timed ({t:.1f} s), "
                         f"scaled to the {its0} iterations its solve takes",
               "other_oracle_solvers": oracle_other_solvers(insts[0], direct=False)}

    line = {"metric": METRIC, "value": value,
            "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "s_per_solve": ms_per_step / 1e3 / args.count,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": bench_config(args, nodes_total),
            "iterations": {"mean": float(np.mean(its_all[-1])), "max": int(np.max(its_all[-1])),
                           "by_beta": by_group([w["beta"] for w in insts], its_all[-1]),
                           "by_N": by_group([w["N"] for w in insts], its_all[-1])},
            "instance_latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                   "note": "device globaltimer from solve start to each instance's convergence"},
            "max_relres": float(max(rel_all)),
            "assembly_s_per_instance": assembly_s,
            "assembly_threads": min(len(insts), len(os.sched_getaffinity(0)) or 1),
            "s_per_solve_with_assembly": ms_per_step / 1e3 / args.count + assembly_s,
            "jacobi_fallback_instances": int(stats["fallback_instances"]) // args.steps,
            "jacobi_cg": cg,
            "other_workloads": other,
            "roofline": roofline, "time_breakdown_ms": breakdown,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(b_all.numel() * 8),
                    "d2h_bytes_per_step": int(x_all.numel() * 8),
                    "ms_per_step": {"h2d": e2e_parts[0] / args.steps, "solve": e2e_parts[1] / args.steps,
                                    "d2h": e2e_parts[2] / args.steps}},
            "gpu_launches": int(stats["kernel_launches"]),
            "launches_per_solve": {"host_graph_launches": stats["graph_launches"] / args.steps,
                                   "kernels_run": stats["kernel_launches"] / args.steps, "slot_gating": stats["slot_gating"],
                                   "note": "slot_gating 2: each batched solve is one CUDA graph launch, its "
                                           "restart cycles a conditional WHILE node decided on the device; "
                                           "3: host-driven cycles (--host-loop)"},
            "autotuning": B.tuning(),
            "clocks": clk, "cpu_baseline": cpu}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
