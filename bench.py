#!/usr/bin/env python
"""Benchmark of the spectral-element Poisson CG solve on GB300.

One step = one complete mixed-precision solve (FP32 Jacobi-PCG inside FP64
iterative refinement, every kernel of the hot path) of the 16x16x16 deformed
box, N = 9 (4,096,000 local / 3,048,625 unique nodes), right-hand side
U[-1,1) per unique node, to a true FP64 relative residual of 1e-10.

value = unique degrees of freedom solved to 1e-10 per second, summed over
ranks (each rank solves its own replica: weak scaling).  The same line
reports the plain FP64 PCG time on the same GPU (the paper's Gain), the
operator throughput with its HBM roofline, an end-to-end number through the
host-buffer entry point, and the FP64 CPU oracle as a baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "CG time-to-solution & ax GDOF/s: mixed vs FP64 on 1 GB300 at equal residual"
UNIT = "GDOF/s (unique DOFs solved to FP64 rel. residual 1e-10 per second)"
BOX = W.MIXED_16CUBE_N9
WORKLOAD = ("mixed-precision Jacobi-PCG (FP32 operator and vectors, FP64 dots, FP64 iterative "
            "refinement) on the 16x16x16 deformed box, N=9, to FP64 relative residual 1e-10")
RTOL = 1e-10


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave the compact summary of the other workloads out of the line")
    ap.add_argument("--cpu-iters", type=int, default=40,
                    help="oracle iterations timed for the CPU baseline sample")
    ap.add_argument("--mode", choices=["full", "solve", "ax", "sweep", "batched", "learned", "vprec",
                                       "learned-step", "batched-step", "schwarz-step",
                                       "schwarz2-step", "extras"],
                    default="full",
                    help="solve: only the timed solves (for a kernel launch list); "
                         "ax: only a few launches of the operators (for a profiler capture); "
                         "sweep / batched / learned: the other workloads, one JSON line each")
    ap.add_argument("--prec", default="fp32", help="precision of --mode ax")
    ap.add_argument("--variant", type=int, default=-1,
                    help="operator variant of --mode ax (-1: the default)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default operator variants (profiler runs: timing under a "
                         "profiler would steer the autotuner)")
    ap.add_argument("--edge", type=int, default=0,
                    help="--mode solve / ax only: an edge^3 deformed box of order --order instead "
                         "of the 16^3, N=9 workload (profiling other mesh sizes)")
    ap.add_argument("--order", type=int, default=9, help="polynomial order with --edge")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the iteration's kernels from the host instead of one CUDA graph "
                         "(same kernels; lets a profiler list them one by one)")
    a = ap.parse_args(argv)
    if a.edge and a.mode not in ("solve", "ax"):
        ap.error("--edge applies to --mode solve and --mode ax only")
    return a


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over the ranks of the process group (x itself alone)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, n_global: int, steps: int, max_ms: float) -> float:
    """Unique DOFs solved by all ranks per second (each rank solves its own
    replica), in GDOF/s, over the slowest rank's time."""
    return world * n_global * steps / (max_ms * 1e-3) / 1e9


def oracle_iterations():
    p = os.path.join(ROOT, "oracle", "iteration_counts.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)["mixed_16cube_n9"]


def host_info():
    """Host thread count and CPU model of the machine the bench runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count(), model


def cpu_baseline(iters: int):
    """The FP64 oracle as it stands, on the host cores, on the same problem:
    a full Jacobi-PCG solve to 1e-10 on all cores (measured, the reported
    value), and a sample of `iters` iterations on one thread scaled to the
    oracle's own iteration count.  Returns the baseline and the oracle's
    solution continued to 1e-13 (the reference of the accuracy check)."""
    import oracle
    P = oracle.Problem(BOX)
    b = P.to_local(W.rhs_global(BOX, 0))
    nproc, model = host_info()
    n_all = oracle.threads()
    oracle.threads(1)
    t0 = time.perf_counter()
    P.pcg(b, tol=0.0, maxit=iters)
    per_it1 = (time.perf_counter() - t0) / iters
    oracle.threads(n_all)
    t0 = time.perf_counter()
    x, it, rel, _ = P.pcg_par(b, tol=RTOL, maxit=20000)
    t_all = time.perf_counter() - t0
    xo, _, rel_o, _ = P.pcg_par(b, tol=1e-13, maxit=20000, x0=x)
    full = oracle_iterations()
    one = {"ms_per_iteration": per_it1 * 1e3, "iterations_timed": iters}
    if full is not None:
        one["seconds_per_solve_extrapolated"] = per_it1 * full["iterations"]
        one["value"] = BOX.n_global / one["seconds_per_solve_extrapolated"] / 1e9
    base = {
        "value": BOX.n_global / t_all / 1e9,
        "unit": UNIT,
        "cores": n_all,
        "kind": "oracle",
        "sample": (f"one full FP64 Jacobi-PCG solve to 1e-10 of the C oracle on {n_all} host "
                   f"threads (OpenMP over elements, nodes and fixed chunks) on the same E=4096 "
                   f"N=9 problem: {it} iterations in {t_all:.1f} s; also {iters} iterations on "
                   f"1 thread: {per_it1 * 1e3:.1f} ms/iteration"),
        "seconds_per_solve": t_all,
        "iterations": it,
        "one_thread": one,
        "nproc": nproc,
        "cpu_model": model,
    }
    return base, xo


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        args = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                "-lms", "200"]
        if device_uuid:
            args += ["-i", device_uuid]
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(args, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


class NvmlEnergy:
    """The GPU's cumulative energy counter (NVML
    nvmlDeviceGetTotalEnergyConsumption, millijoules since the driver loaded;
    a read-only query) through the driver's own library."""

    def __init__(self, device_uuid: str | None):
        import ctypes as C
        self.C = C
        self.dev = None
        try:
            lib = C.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            dev = C.c_void_p()
            if device_uuid:
                ok = lib.nvmlDeviceGetHandleByUUID(device_uuid.encode(), C.byref(dev)) == 0
            else:
                ok = lib.nvmlDeviceGetHandleByIndex_v2(0, C.byref(dev)) == 0
            if ok:
                self.lib, self.dev = lib, dev
        except Exception:
            self.dev = None

    def read_mj(self):
        if self.dev is None:
            return None
        v = self.C.c_ulonglong(0)
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.dev, self.C.byref(v)) != 0:
            return None
        return int(v.value)


def energy_per_solve(run, sync, device_uuid, seconds=2.0, min_calls=10):
    """Joules per call of run() (the paper's energy view): the GPU's energy
    counter read before and after back-to-back calls (at least `min_calls`,
    and enough to cover about `seconds`).  Without the counter: None."""
    meter = NvmlEnergy(device_uuid)
    if meter.read_mj() is None:
        return None
    sync()
    t0 = time.perf_counter()
    run()
    sync()
    reps = max(min_calls, int(seconds / max(time.perf_counter() - t0, 1e-3)))
    e0 = meter.read_mj()
    t0 = time.perf_counter()
    for _ in range(reps):
        run()
    sync()
    wall = time.perf_counter() - t0
    e1 = meter.read_mj()
    if e0 is None or e1 is None or e1 <= e0:
        return None
    joules = (e1 - e0) * 1e-3
    return {"joules_per_solve": joules / reps, "solves": reps, "mean_watts": joules / wall,
            "wall_s": wall}


def fp64_peak_tflops(dev):
    """Measured FP64 rate of this GPU: cuBLAS DGEMM 4096^3 (2 n^3 flops), best
    of 3 after a warm-up, CUDA events."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    bm = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, bm)
    best = None
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, bm)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, bm
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def l2_flush(buf, k):
    """Evict L2 between timed steps: write `buf` (larger than L2), then read it
    back so the writes' dirty lines are written back before the next step."""
    buf.fill_(k & 0xFF)
    buf.view(dtype=__import__("torch").int32).sum()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# device source of the FP32 fused-step kernels (the ncu summary's traffic is
# valid while these are unchanged)
AX_SOURCES = ["paper_2405_11065_gb300/csrc/nb_ax_pen.cuh", "paper_2405_11065_gb300/csrc/nb_ax_tma.cuh",
              "paper_2405_11065_gb300/csrc/nb_ax_impl.cuh", "paper_2405_11065_gb300/csrc/nb_ax_f32.cu",
              "paper_2405_11065_gb300/csrc/nb_bulk.cuh", "paper_2405_11065_gb300/csrc/nb_cg_dev.cuh",
              "paper_2405_11065_gb300/csrc/nb_reduce.cuh"]


def profiled_traffic(sha, kernel):
    """DRAM bytes per launch of the FP32 fused-step kernel variant `kernel`
    from the committed ncu summary (lines "- dram_bytes_per_launch[<kernel>]:
    <bytes>"), if it was taken on the current device source."""
    p = os.path.join(ROOT, "profiles", "ax_fp32_cg_step_E4096_N9.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha") != sha:
        return None
    try:
        return float(vals[f"dram_bytes_per_launch[{kernel}]"])
    except (KeyError, ValueError):
        return None


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands on all host
    cores.  Each step is a bounded sample -- `per_step_iters` Jacobi-PCG
    iterations of the parallel oracle on the E=4096 N=9 problem -- and the
    value scales the mean step to the oracle's own iteration count to 1e-10."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    P = oracle.Problem(BOX)
    b = P.to_local(W.rhs_global(BOX, 0))
    full = oracle_iterations()
    nproc, model = host_info()
    cores = oracle.threads()
    per_step_iters = 100
    for _ in range(args.warmup):
        P.pcg_par(b, tol=0.0, maxit=10)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        P.pcg_par(b, tol=0.0, maxit=per_step_iters)
        times.append(time.perf_counter() - t0)
    step_s = sum(times) / len(times)
    t_solve = step_s / per_step_iters * full["iterations"]
    value = BOX.n_global / t_solve / 1e9
    sample = (f"each step: {per_step_iters} FP64 Jacobi-PCG iterations of the C oracle on "
              f"{cores} host threads ({model}) on the E=4096 N=9 problem; value scaled to the "
              f"{full['iterations']} iterations the oracle needs for 1e-10 "
              f"({t_solve:.1f} s per solve)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + " (FP64 CPU oracle)", "E": BOX.E, "N": BOX.N,
                       "n_local": BOX.n_local, "n_global": BOX.n_global,
                       "step": f"{per_step_iters} oracle iterations"},
            "seconds_per_solve_scaled": t_solve,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "nproc": nproc, "cpu_model": model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _rhs_local(nb, mesh, box, seed, dev):
    import torch
    bg = torch.from_numpy(W.rhs_global(box, seed)).to(dev)
    b = torch.empty(box.n_local, dtype=torch.float64, device=dev)
    mesh.to_local(nb.NB_FP64, bg, b, masked=True)
    return b


def run_sweep(args):
    """Operator throughput and CG time to 1e-10 on deformed cubes E = 8^3 ..
    32^3 at N in {5, 7, 9, 11, 15}: FP64, FP32 and tensor-core operators."""
    import torch
    import paper_2405_11065_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    flush = torch.empty(W.l2_flush_bytes(), dtype=torch.uint8, device=dev)
    peak, _ = measured_peaks()
    for box in W.sweep_boxes():
        mesh = nb.Mesh.from_box(ctx, box)
        nL = box.n_local
        line = {"mode": "sweep", "E": box.E, "N": box.N, "n_local": nL, "n_global": box.n_global}
        for pname, elt in (("fp64", 8), ("fp32", 4), ("tc_f16", 4), ("tc_bf16", 4)):
            prec = nb.PREC_NAMES[pname]
            if pname in ("fp64", "fp32"):
                mesh.autotune(prec, reps=2, flush=flush)
            ms = mesh.time_ax(prec, cg_step=False, reps=5, flush=flush)
            gbs = 8 * elt * nL / (ms * 1e-3) / 1e9
            line[pname] = {"ax_ms": ms, "ax_gdofs_local": nL / (ms * 1e-3) / 1e9,
                           "ax_gbs_algorithmic": gbs, "hbm_frac": gbs / peak}
        b = _rhs_local(nb, mesh, box, 0, dev)
        x = torch.zeros_like(b)
        mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP32))
        x.zero_()
        out = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP32))
        line["cg_fp32_refined"] = {"ms": out["seconds"] * 1e3, "iters": out["iters"],
                                   "outer": out["outer_iters"], "rel_res": out["rel_res"],
                                   "status": out["status"]}
        if nL <= 20_000_000:
            x.zero_()
            o64 = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP64))
            line["cg_fp64"] = {"ms": o64["seconds"] * 1e3, "iters": o64["iters"],
                               "rel_res": o64["rel_res"], "status": o64["status"]}
        print(json.dumps(line), flush=True)
        mesh.close()
        del b, x
        torch.cuda.empty_cache()
    return 0


def run_batched(args):
    """256 independent problems, E ~ U{8..512} (most cubic box), N in
    {5,7,9,11}, mixed precision with FP64 refinement, one graph per solve."""
    import torch
    import paper_2405_11065_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    probs = W.batched_problems(256)
    boxes = [bx for bx, _ in probs]
    t0 = time.perf_counter()
    batch = nb.Batch(ctx, boxes)
    setup_s = time.perf_counter() - t0
    flush = torch.empty(W.l2_flush_bytes(), dtype=torch.uint8, device=dev)
    batch.autotune(reps=3, flush=flush)
    ug = torch.from_numpy(np.concatenate([W.rhs_global(bx, s) for bx, s in probs])).to(dev)
    b = torch.empty(batch.n_local, dtype=torch.float64, device=dev)
    batch.to_local(ug, b)
    x = torch.zeros_like(b)
    opts = nb.default_opts(prec=nb.NB_FP32, maxiter=400000)
    batch.solve(b, x, opts)
    times = []
    for _ in range(max(args.steps, 1)):
        x.zero_()
        out = batch.solve(b, x, opts)
        times.append(out["seconds"])
    iters = [p["iters"] for p in out["problems"]]
    t = statistics.median(times)
    # the same problems solved one after the other by the single-problem path
    # (each with its own graph-captured solve), for comparison
    seq_ms = 0.0
    stream = torch.cuda.current_stream(dev)
    for p, (bx, _) in enumerate(probs):
        mesh = nb.Mesh.from_box(ctx, bx)
        lo = int(batch.l_off[p])
        bp = b[lo:lo + bx.n_local].contiguous()
        xp = torch.zeros_like(bp)
        mesh.solve(bp, xp, opts)
        xp.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mesh.solve(bp, xp, opts)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        seq_ms += e0.elapsed_time(e1)
        mesh.close()
    line = {"mode": "batched", "problems": len(boxes), "n_local": batch.n_local,
            "n_global": batch.n_global, "orders": sorted(set(bx.N for bx in boxes)),
            "setup_s": setup_s, "solve_ms": t * 1e3,
            "gdofs_solved_per_s": batch.n_global / t / 1e9,
            "batched_iterations": out["iters"], "max_problem_iters": max(iters),
            "median_problem_iters": float(np.median(iters)), "status": out["status"],
            "worst_rel_res": out["rel_res"], "launches": out["launches"],
            "sequential_single_solves_ms": seq_ms,
            "all_ok": all(p["status"] == 0 for p in out["problems"])}
    print(json.dumps(line), flush=True)
    return 0


def run_learned(args):
    """The learned-preconditioner workload (16^3 deformed box, N = 7)."""
    import torch
    import paper_2405_11065_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    box = W.LEARNED_16CUBE_N7
    mesh = nb.Mesh.from_box(ctx, box)
    model = nb.Model(ctx, box.N, 96, seed=7)
    snaps = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 800]  # across the ~900-iteration solve
    t0 = time.perf_counter()
    Xs, Ts = [], []
    for s in W.TRAIN_SEEDS:
        X, T = nb.Model.collect(mesh, _rhs_local(nb, mesh, box, s, dev), snaps, 120, seed=s)
        Xs.append(X)
        Ts.append(T)
    X, T = torch.cat(Xs), torch.cat(Ts)
    model.train(X, T, epochs=40, batch=256, lr=1e-3)
    loss = model.train(X, T, epochs=20, batch=256, lr=3e-4)
    model.attach(mesh)
    train_s = time.perf_counter() - t0
    res = []
    for s in W.HELDOUT_SEEDS:
        b = _rhs_local(nb, mesh, box, s, dev)
        row = {"seed": s}
        for name, pc in (("jacobi", nb.NB_PC_JACOBI), ("learned", nb.NB_PC_LEARNED)):
            x = torch.zeros_like(b)
            o = nb.default_opts(prec=nb.NB_FP32, pc=pc, rtol=1e-8)
            mesh.solve(b, x, o)
            x.zero_()
            out = mesh.solve(b, x, o)
            row[name] = {"iters": out["iters"], "ms": out["seconds"] * 1e3,
                         "status": out["status"], "rel_res": out["rel_res"]}
        res.append(row)
    line = {"mode": "learned", "E": box.E, "N": box.N, "pairs": int(sum(x.shape[0] for x in Xs)),
            "params": model.nparam, "train_s": train_s, "final_loss": loss, "rtol": 1e-8,
            "results": res}
    print(json.dumps(line), flush=True)
    return 0


def small_fp64(nb, ctx, dev):
    """The plain FP64 Jacobi-PCG workload: 2x2x2 affine box, N = 7, right-hand
    side U[-1,1) per unique node from seed 0; the relative residual after 100
    iterations, then the solve continued to 1e-10."""
    import torch
    box = W.SMALL_FP64
    mesh = nb.Mesh.from_box(ctx, box)
    b = _rhs_local(nb, mesh, box, 0, dev)
    x = torch.zeros_like(b)
    s100 = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP64, rtol=1e-30, maxiter=100))
    x.zero_()
    mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP64, rtol=RTOL))  # warm-up
    x.zero_()
    full = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP64, rtol=RTOL))
    mesh.close()
    return {"E": box.E, "N": box.N, "n_global": box.n_global, "deform": box.deform,
            "rel_res_after_100": s100["rel_res"], "iters_to_1e-10": full["iters"],
            "rel_res": full["rel_res"], "ms_to_1e-10": full["seconds"] * 1e3,
            "status": full["status"]}


def extra_workloads(nb, ctx, dev, flush, hbm_peak):
    """The other workloads, compact, for the default line: the plain FP64
    PCG on the 2x2x2 box, the roofline sweep at its largest size (E = 32^3 at
    N = 7 and 9), the 256-problem batch, and the learned preconditioner
    against Jacobi on one held-out right-hand side."""
    import torch
    out = {"fp64_2cube_N7": small_fp64(nb, ctx, dev)}
    sweep = []
    for N in (7, 9):
        box = W.Box(32, 32, 32, N, 0.05)
        mesh = nb.Mesh.from_box(ctx, box)
        nL = box.n_local
        mesh.autotune(nb.NB_FP32, reps=2, flush=flush)
        ms_ax = mesh.time_ax(nb.NB_FP32, cg_step=False, reps=5, flush=flush)
        ms_cg = mesh.time_ax(nb.NB_FP32, cg_step=True, reps=5, flush=flush)
        b = _rhs_local(nb, mesh, box, 0, dev)
        x = torch.zeros_like(b)
        o = nb.default_opts(prec=nb.NB_FP32, rtol=RTOL)
        mesh.solve(b, x, o)
        x.zero_()
        st = mesh.solve(b, x, o)
        sweep.append({"E": box.E, "N": N, "n_local": nL, "kernel": mesh.ax_variant_name(nb.NB_FP32),
                      "ax_ms": ms_ax, "ax_hbm_frac": 32 * nL / (ms_ax * 1e-3) / 1e9 / hbm_peak,
                      "cg_step_ms": ms_cg,
                      "cg_step_hbm_frac": 44 * nL / (ms_cg * 1e-3) / 1e9 / hbm_peak,
                      "mixed_solve_ms": st["seconds"] * 1e3, "iters": st["iters"],
                      "rel_res": st["rel_res"], "status": st["status"]})
        mesh.close()
        del b, x
        torch.cuda.empty_cache()
    out["sweep_32cube"] = sweep

    probs = W.batched_problems(256)
    boxes = [bx for bx, _ in probs]
    t0 = time.perf_counter()
    batch = nb.Batch(ctx, boxes)
    setup_s = time.perf_counter() - t0
    batch.autotune(reps=2, flush=flush)
    ug = torch.from_numpy(np.concatenate([W.rhs_global(bx, sd) for bx, sd in probs])).to(dev)
    b = torch.empty(batch.n_local, dtype=torch.float64, device=dev)
    batch.to_local(ug, b)
    x = torch.zeros_like(b)
    o = nb.default_opts(prec=nb.NB_FP32, maxiter=400000)
    batch.solve(b, x, o)
    x.zero_()
    st = batch.solve(b, x, o)
    iters = [p["iters"] for p in st["problems"]]
    out["batched_256"] = {"problems": len(boxes), "n_local": batch.n_local,
                          "n_global": batch.n_global, "setup_s": setup_s,
                          "solve_ms": st["seconds"] * 1e3,
                          "gdofs_solved_per_s": batch.n_global / st["seconds"] / 1e9,
                          "batched_iterations": st["iters"], "max_problem_iters": max(iters),
                          "median_problem_iters": float(np.median(iters)),
                          "all_ok": all(p["status"] == 0 for p in st["problems"])}
    batch.close()
    del b, x, ug
    torch.cuda.empty_cache()

    box = W.LEARNED_16CUBE_N7
    mesh = nb.Mesh.from_box(ctx, box)
    model = nb.Model(ctx, box.N, 96, seed=7)
    snaps = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 800]
    t0 = time.perf_counter()
    Xs, Ts = [], []
    for sd in W.TRAIN_SEEDS:
        X, T = nb.Model.collect(mesh, _rhs_local(nb, mesh, box, sd, dev), snaps, 120, seed=sd)
        Xs.append(X)
        Ts.append(T)
    X, T = torch.cat(Xs), torch.cat(Ts)
    model.train(X, T, epochs=40, batch=256, lr=1e-3)
    loss = model.train(X, T, epochs=20, batch=256, lr=3e-4)
    model.attach(mesh)
    train_s = time.perf_counter() - t0
    sd = W.HELDOUT_SEEDS[0]
    b = _rhs_local(nb, mesh, box, sd, dev)
    row = {"E": box.E, "N": box.N, "pairs": int(X.shape[0]), "params": model.nparam,
           "train_s": train_s, "final_loss": loss, "rtol": 1e-8, "heldout_seed": sd}
    for name, pc in (("jacobi", nb.NB_PC_JACOBI), ("learned", nb.NB_PC_LEARNED)):
        x = torch.zeros_like(b)
        o = nb.default_opts(prec=nb.NB_FP32, pc=pc, rtol=1e-8)
        mesh.solve(b, x, o)
        ms = []
        for _ in range(3):
            x.zero_()
            st = mesh.solve(b, x, o)
            ms.append(st["seconds"] * 1e3)
        row[name] = {"iters": st["iters"], "ms": statistics.median(ms), "status": st["status"],
                     "rel_res": st["rel_res"]}
    out["learned_16cube_N7"] = row
    mesh.close()
    return out


def run_extras(args):
    """Only the compact summary of the other workloads (one JSON line)."""
    import torch
    import paper_2405_11065_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    flush = torch.empty(W.l2_flush_bytes(), dtype=torch.uint8, device=dev)
    peak, _ = measured_peaks()
    print(json.dumps({"mode": "extras", **extra_workloads(nb, ctx, dev, flush, peak)}), flush=True)
    return 0


def run_learned_step(args):
    """Profiling aid: `--steps` flexible-CG steps with the learned
    preconditioner on the learned workload's mesh (E=4096, N=7) and an
    untrained network of its shape (the kernels' cost does not depend on the
    weights); host-launched with --no-graph so that a profiler lists every
    kernel."""
    import torch
    import paper_2405_11065_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    box = W.LEARNED_16CUBE_N7
    mesh = nb.Mesh.from_box(ctx, box)
    model = nb.Model(ctx, box.N, 96, seed=7)
    model.attach(mesh)
    b = _rhs_local(nb, mesh, box, 0, dev)
    x = torch.zeros_like(b)
    # one inner solve of exactly `steps` steps (restarted form, tight inner tolerance)
    o = nb.default_opts(prec=nb.NB_FP32, pc=nb.NB_PC_LEARNED, rtol=1e-8, maxiter=args.steps,
                        max_outer=1, restart=1, inner_rtol=1e-12,
                        use_graph=0 if args.no_graph else 1)
    st = mesh.solve(b, x, o)
    print(json.dumps({"mode": "learned-step", "iters": st["iters"], "ms": st["seconds"] * 1e3}),
          flush=True)
    return 0


def run_schwarz_step(args):
    """Profiling aid: `--steps` flexible-CG steps with the Schwarz
    preconditioner on the main workload's mesh (E=4096, N=9), host-launched
    with --no-graph so that a profiler lists every kernel."""
    import torch
    import paper_2405_11065_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    mesh = nb.Mesh.from_box(ctx, BOX)
    b = _rhs_local(nb, mesh, BOX, 0, dev)
    x = torch.zeros_like(b)
    pc = nb.NB_PC_SCHWARZ2 if args.mode == "schwarz2-step" else nb.NB_PC_SCHWARZ
    # one inner solve of exactly `steps` steps (restarted form, tight inner tolerance)
    o = nb.default_opts(prec=nb.NB_FP32, pc=pc, rtol=1e-10, maxiter=args.steps,
                        max_outer=1, restart=1, inner_rtol=1e-12,
                        use_graph=0 if args.no_graph else 1)
    st = mesh.solve(b, x, o)
    print(json.dumps({"mode": args.mode, "iters": st["iters"], "ms": st["seconds"] * 1e3}),
          flush=True)
    return 0


def run_batched_step(args):
    """Profiling aid: the batched workload's first `--steps` iterations
    (one refinement step), host-launched with --no-graph so that a profiler
    lists every kernel."""
    import torch
    import paper_2405_11065_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    probs = W.batched_problems(256)
    batch = nb.Batch(ctx, [bx for bx, _ in probs])
    ug = torch.from_numpy(np.concatenate([W.rhs_global(bx, s) for bx, s in probs])).to(dev)
    b = torch.empty(batch.n_local, dtype=torch.float64, device=dev)
    batch.to_local(ug, b)
    x = torch.zeros_like(b)
    out = batch.solve(b, x, nb.default_opts(prec=nb.NB_FP32, maxiter=args.steps, max_outer=1,
                                            use_graph=0 if args.no_graph else 1))
    print(json.dumps({"mode": "batched-step", "iters": out["iters"], "ms": out["seconds"] * 1e3}),
          flush=True)
    return 0


def run_vprec(args):
    """The precision study of Section 4.2 on the GPU: 100 CG iterations
    (Nekbone's fixed count) without preconditioner on the E=4096, N=9
    deformed box, every arithmetic operation of the loop rounded to t
    mantissa bits, t = 3 .. 52; the loop's final relative residual and the
    true binary64 one, |b - A x| / |b|."""
    import torch
    import paper_2405_11065_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    box = W.MIXED_16CUBE_N9
    mesh = nb.Mesh.from_box(ctx, box)
    b = _rhs_local(nb, mesh, box, 0, dev)
    x = torch.zeros_like(b)
    w = torch.empty_like(b)
    bn = math.sqrt(mesh.glsc3(nb.NB_FP64, b, b))
    rows = []
    t0 = time.perf_counter()
    for t in list(range(3, 53)):
        h = mesh.cg_vprec(t, 100, b, x)
        mesh.ax(nb.NB_FP64, x, w, assemble=True)
        r = b - w
        true_rel = math.sqrt(mesh.glsc3(nb.NB_FP64, r, r)) / bn
        rows.append({"t": t, "loop_rel_res": float(h[-1]), "true_rel_res": true_rel})
    ref = rows[-1]["true_rel_res"]
    stable = next((r["t"] for r in rows
                   if all(abs(q["true_rel_res"] - ref) <= 0.1 * ref for q in rows if q["t"] >= r["t"])),
                  None)
    # Monte Carlo Arithmetic at t = 23, 20 runs per mode (Section 4.2): the
    # residual history's mean, minimum and maximum, and the significant bits
    # s2 = -log2(sigma / |mu|) of the final residual over the runs
    mca = {}
    for mode in ("rr", "mca"):
        hs = np.array([mesh.cg_mca(mode, 23, 1000 + k, 100, b, x) for k in range(20)])
        mu, sd = hs.mean(axis=0), hs.std(axis=0, ddof=1)
        at = [9, 24, 49, 99]
        mca[mode] = {"iterations": [i + 1 for i in at],
                     "mean": [float(mu[i]) for i in at], "min": [float(hs[:, i].min()) for i in at],
                     "max": [float(hs[:, i].max()) for i in at],
                     "significant_bits_final": float(-math.log2(sd[-1] / abs(mu[-1])))
                     if sd[-1] > 0 else 52.0}
    line = {"mode": "vprec", "E": box.E, "N": box.N, "iterations": 100, "preconditioner": "none",
            "stable_from_t": stable, "seconds": time.perf_counter() - t0, "results": rows,
            "mca_t23_20_runs": mca}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode in ("sweep", "batched", "learned", "vprec", "learned-step", "batched-step",
                     "schwarz-step", "schwarz2-step", "extras"):
        return {"sweep": run_sweep, "batched": run_batched, "learned": run_learned,
                "vprec": run_vprec, "learned-step": run_learned_step,
                "batched-step": run_batched_step, "schwarz-step": run_schwarz_step,
                "schwarz2-step": run_schwarz_step, "extras": run_extras}[args.mode](args)
    rank, world, local = dist_env()
    cpu, x_oracle = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, x_oracle = cpu_baseline(args.cpu_iters)  # host only, before the first GPU call

    import torch
    import paper_2405_11065_gb300 as nb

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)  # legacy default stream: events are ordered
    ctx = nb.Context(local)                  # with the library's own blocking stream
    box = BOX  # --edge (solve and ax modes only, checked in parse): another box size
    if args.edge:
        box = W.Box(args.edge, args.edge, args.edge, args.order, BOX.deform)
    mesh = nb.Mesh.from_box(ctx, box)
    bg = torch.from_numpy(W.rhs_global(box, rank)).to(dev)
    b = torch.empty(box.n_local, dtype=torch.float64, device=dev)
    mesh.to_local(nb.NB_FP64, bg, b, masked=True)
    x = torch.zeros_like(b)
    flush = torch.empty(W.l2_flush_bytes(), dtype=torch.uint8, device=dev)
    if args.mode == "ax":
        prec = nb.PREC_NAMES[args.prec]
        if args.variant >= 0:
            mesh.set_ax_variant(prec, args.variant)
        for _ in range(args.warmup):
            mesh.time_ax(prec, cg_step=True, reps=1, flush=flush)
        ms = mesh.time_ax(prec, cg_step=True, reps=max(args.steps, 1), flush=flush)
        print(json.dumps({"mode": "ax", "prec": args.prec, "cg_step_ms": ms,
                          "kernel": mesh.ax_variant_name(prec),
                          "kernel_source_sha": source_sha(AX_SOURCES)}), flush=True)
        return 0

    # autotune the operator (per precision, this order) before timing
    tune = {}
    for pname, prec in (("fp32", nb.NB_FP32), ("fp64", nb.NB_FP64)):
        if args.no_autotune:
            tune[pname] = {"variant": -1, "ms": None}
            continue
        v, ms = mesh.autotune(prec, reps=3, flush=flush)
        tune[pname] = {"variant": v, "ms": ms}

    opts = nb.default_opts(prec=nb.NB_FP32, rtol=RTOL, use_graph=0 if args.no_graph else 1)
    for _ in range(args.warmup):
        x.zero_()
        mesh.solve(b, x, opts)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    dev_uuid = None
    try:
        dev_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = Clocks(dev_uuid)
    barrier()
    evs = []
    stats = []
    wall0 = time.perf_counter()
    for k in range(args.steps):
        l2_flush(flush, k)  # evict L2 between steps, outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = mesh.solve(b, x, opts)
        e1.record(stream)
        evs.append((e0, e1))
        stats.append(out)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, c in evs]
    total_ms = sum(step_ms)
    max_ms = max_over_ranks(total_ms, dev)
    ok = all(s["status"] == 0 and s["rel_res"] < RTOL for s in stats)
    if args.mode == "solve":
        if rank == 0:
            print(json.dumps({"mode": "solve", "ms_per_step": max_ms / args.steps, "ok": ok,
                              "iters": stats[-1]["iters"], "launches": stats[-1]["launches"]}),
                  flush=True)
        return 0 if ok else 1

    # correctness of the last solve on the device: FP64 residual
    w = torch.empty_like(b)
    mesh.ax(nb.NB_FP64, x, w, assemble=True)
    r = b - w
    c = torch.from_numpy(mesh.geom()[2]).to(dev)
    true_rel = float(torch.sqrt((c * r * r).sum() / (c * b * b).sum()))

    # plain FP64 PCG on the same GPU, same problem (the paper's comparison)
    o64 = nb.default_opts(prec=nb.NB_FP64, rtol=RTOL)
    x64 = torch.zeros_like(b)
    mesh.solve(b, x64, o64)
    fp64_ms, fp64_stats = [], None
    for _ in range(2):
        l2_flush(flush, 1)
        x64.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fp64_stats = mesh.solve(b, x64, o64)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        fp64_ms.append(e0.elapsed_time(e1))
    t64 = statistics.median(fp64_ms)
    tm = statistics.median(step_ms)
    # the same mixed solve with the overlapping Schwarz preconditioner (the
    # smoother of the paper's multigrid solveM), one level and with the
    # coarse-grid level
    def time_pc(pc):
        o_pc = nb.default_opts(prec=nb.NB_FP32, pc=pc, rtol=RTOL)
        xs = torch.zeros_like(b)
        mesh.solve(b, xs, o_pc)
        ms, st = [], None
        for _ in range(3):
            l2_flush(flush, 3)
            xs.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = mesh.solve(b, xs, o_pc)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms), st
    sw_t, sw_stats = time_pc(nb.NB_PC_SCHWARZ)
    sw2_t, sw2_stats = time_pc(nb.NB_PC_SCHWARZ2)
    sol_diff = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))

    # the mixed solution against the oracle's (all host cores, to 1e-13)
    oracle_diff = None
    if x_oracle is not None:
        xm = x.cpu().numpy()
        oracle_diff = float(np.linalg.norm(xm - x_oracle) / np.linalg.norm(x_oracle))

    # energy to solution, mixed vs FP64 (outside the timed region; the GPU's
    # cumulative energy counter read before and after at least 10 solves)
    def _mixed():
        x.zero_()
        mesh.solve(b, x, opts)

    def _fp64():
        x64.zero_()
        mesh.solve(b, x64, o64)

    sync = lambda: torch.cuda.synchronize(dev)
    en_m = energy_per_solve(_mixed, sync, dev_uuid)
    en_d = energy_per_solve(_fp64, sync, dev_uuid)
    energy = {"mixed": en_m, "fp64": en_d,
              "reduction_vs_fp64": (1.0 - en_m["joules_per_solve"] / en_d["joules_per_solve"])
              if en_m and en_d else None,
              "method": "NVML total energy counter (nvmlDeviceGetTotalEnergyConsumption) "
                        "read before and after >= 10 back-to-back solves"}

    # the paper's accuracy metric: AE_k = |r_m,k - r_d,k| between the residual
    # histories of an all-FP32 CG loop (the paper's mixed version, no
    # refinement) and the FP64 loop, and their mean MAE
    cap = 4000
    h64 = mesh.solve(b, torch.zeros_like(b), nb.default_opts(prec=nb.NB_FP64, rtol=RTOL),
                     history_cap=cap)["history"]
    h32 = mesh.solve(b, torch.zeros_like(b),
                     nb.default_opts(prec=nb.NB_FP32, rtol=RTOL, inner_rtol=RTOL, max_outer=1,
                                     restart=1),
                     history_cap=cap)["history"]
    kk = min(len(h64), len(h32))
    ae = np.abs(np.asarray(h32[:kk]) - np.asarray(h64[:kk]))
    accuracy = {"metric": "relative residual histories, FP32 CG loop vs FP64 CG loop",
                "fp64_iters": int(len(h64)), "fp32_loop_iters": int(len(h32)),
                "ae_at_fp64_convergence": float(ae[-1]) if kk else None,
                "mae": float(ae.mean()) if kk else None}

    # operator throughput and roofline of the dominant kernel
    hbm_peak, peak_kind = measured_peaks()
    nL = BOX.n_local
    ax = {}
    for pname, prec, elt in (("fp32", nb.NB_FP32, 4), ("fp64", nb.NB_FP64, 8)):
        ms_cg = mesh.time_ax(prec, cg_step=True, reps=20, flush=flush)
        ms_ax = mesh.time_ax(prec, cg_step=False, reps=20, flush=flush)
        ax[pname] = {"cg_step_ms": ms_cg, "ax_ms": ms_ax,
                     "ax_gdofs_local": nL / (ms_ax * 1e-3) / 1e9,
                     "ax_gdofs_unique": BOX.n_global / (ms_ax * 1e-3) / 1e9,
                     "ax_gbs_algorithmic": 8 * elt * nL / (ms_ax * 1e-3) / 1e9,
                     "cg_step_gbs_algorithmic": 11 * elt * nL / (ms_cg * 1e-3) / 1e9,
                     "variant": tune[pname]["variant"]}
    n = BOX.n
    ax["fp64"]["ax_gflops"] = (12 * n + 15) * nL / (ax["fp64"]["ax_ms"] * 1e-3) / 1e9
    fp64_peak = fp64_peak_tflops(dev)
    ax["fp64"]["fp64_peak_tflops_measured"] = fp64_peak
    ax["fp64"]["fp64_peak_kind"] = "cuBLAS DGEMM 4096^3 on this GPU (best of 3)"
    ax["fp64"]["frac_of_fp64_peak"] = ax["fp64"]["ax_gflops"] / (fp64_peak * 1e3)
    ax["fp64"]["frac_of_fp64_nominal_1250_gflops"] = ax["fp64"]["ax_gflops"] / 1250.0
    for pname, prec in (("fp32", nb.NB_FP32), ("fp64", nb.NB_FP64)):
        ax[pname]["kernel"] = mesh.ax_variant_name(prec)
    sha = source_sha(AX_SOURCES)
    bytes_cg = 11 * 4 * nL
    achieved = bytes_cg / (ax["fp32"]["cg_step_ms"] * 1e-3) / 1e9
    kname = mesh.ax_variant_name(nb.NB_FP32)
    traffic = profiled_traffic(sha, kname)
    roofline = {"kernel": kname + " (fused p-update + operator + pap, FP32)",
                "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_kind": f"{peak_kind} (STREAM copy)",
                "traffic": traffic, "algorithmic_bytes_per_launch": bytes_cg,
                "bytes_per_local_node": 44, "kernel_source_sha": sha}

    # end to end through the host-buffer entry point
    e2e = None
    if rank == 0 or world > 1:
        bh = torch.from_numpy(W.rhs_global(BOX, rank)).pin_memory()
        xh = torch.zeros(BOX.n_global, dtype=torch.float64).pin_memory()
        mesh.solve_host(bh, xh, opts)
        e2e_ms = []
        for _ in range(max(2, min(args.steps, 5))):
            l2_flush(flush, 2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outh = mesh.solve_host(bh, xh, opts)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            e2e_ms.append(e0.elapsed_time(e1))
        te = statistics.median(e2e_ms)
        e2e = {"value": world * BOX.n_global / (te * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 8 * BOX.n_global, "d2h_bytes_per_step": 8 * BOX.n_global,
               "ms_per_step": te, "status": outh["status"]}

    # the other workloads, compact (outside the timed region; one replica only)
    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = extra_workloads(nb, ctx, dev, flush, hbm_peak)

    launches = int(sum(s["launches"] for s in stats))
    value = whole_job_value(world, BOX.n_global, args.steps, max_ms)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 refinement)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "E": BOX.E, "N": BOX.N, "n_local": BOX.n_local,
                       "n_global": BOX.n_global, "deform": BOX.deform, "rhs": "U[-1,1) per unique node, seed = rank",
                       "l2": "flushed between timed steps (512 MB written, then read back)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches,
            "time_to_solution_ms": {"mixed_fp32_refined": tm, "fp64_pcg": t64,
                                    "mixed_schwarz": sw_t, "mixed_schwarz_two_level": sw2_t},
            "schwarz": {"iters": sw_stats["iters"], "outer": sw_stats["outer_iters"],
                        "rel_res": sw_stats["rel_res"], "status": sw_stats["status"]},
            "schwarz_two_level": {"iters": sw2_stats["iters"], "outer": sw2_stats["outer_iters"],
                                  "rel_res": sw2_stats["rel_res"], "status": sw2_stats["status"]},
            "gain_vs_fp64": (t64 - tm) / t64,
            "speedup_vs_fp64": t64 / tm,
            "iterations": {"mixed_inner": stats[-1]["iters"], "mixed_outer": stats[-1]["outer_iters"],
                           "fp64": fp64_stats["iters"]},
            "rel_res": {"mixed": stats[-1]["rel_res"], "fp64": fp64_stats["rel_res"],
                        "mixed_recomputed": true_rel},
            "mixed_vs_fp64_solution_rel_diff": sol_diff,
            "mixed_vs_oracle_solution_rel_diff": oracle_diff,
            "accuracy_ae_mae": accuracy, "energy": energy,
            "other_workloads": extras,
            "all_steps_converged": ok,
            "ax": ax,
            "wall_s_timed_region": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
