"""Benchmark of the GB300 pressure multigrid (arXiv 1410.8568, Sec. 2.3).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload drop_film_128|drop_film_256|drop_film_512|sphere_32|batch64|serve_stream]

Metric: Poisson multigrid solves per second to a relative residual of 1e-10,
mixed precision (FP32 V(2,2) cycles inside FP64 iterative refinement) next to
the plain FP64 path on the same inputs, with p50/p99 latency.

One step = one pressure solve of a time step: the new density goes in
(face coefficients of Eqs. 11-12, coarse-level coefficients, coarsest-grid
inverse) and Eq. 9 is solved from a cold start to ||r|| <= 1e-10 ||b||.  Inputs
are resident in HBM when the timed region starts; L2 is flushed (a 256 MB
write) before every step, outside the step's events.  Each step is bracketed by
CUDA events on the solver's stream; `value` = steps / summed step time.

`e2e` repeats the step through mg_step_host with pinned host buffers (density
and right-hand side copied in, pressure copied out, inside the timed region).

`roofline` is for the dominant kernel (the finest-level red-black half-sweep,
FP32): its launches are timed with CUDA events on the solver stream in a second
pass of the same steps (host-driven loop, one event pair per launch).

`cpu_baseline` / `--impl reference`: the FP64 CPU oracle (oracle/, plain C with
OpenMP over z-planes) solving the same problem on the host cores.

Multi-GPU: the solve does not shard here (replicas only): each rank solves its
own copy; value = all ranks' solves / the slowest rank's time.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Poisson MG solves/s to 1e-10 rel. residual, mixed vs FP64 on GB300; p50/p99 ms"
TOL = 1e-10
L2_FLUSH_BYTES = 256 << 20
# largest grid whose oracle p* the bench computes on the host (512^3: about a
# minute on 16 cores and ~10 GB of host memory)
ORACLE_MAX_CELLS = 512 ** 3

WORKLOADS = {
    "drop_film_128": dict(kind="config2", n=128,
                          desc="drop_film_128^3_1000to1: film depth 0.1 + drop R 0.125 at z 0.3, periodic x,y, Neumann z, Fourier-divergence RHS"),
    "drop_film_256": dict(kind="config2", n=256,
                          desc="drop_film_256^3_1000to1: film depth 0.1 + drop R 0.125 at z 0.3, periodic x,y, Neumann z, Fourier-divergence RHS"),
    "drop_film_512": dict(kind="config3", n=512,
                          desc="drop_film_512^3_1000to1: film + drop + 0-4 droplets, periodic x,y, Neumann z, Fourier-divergence RHS"),
    "drop_film_1024": dict(kind="config3", n=1024,
                           desc="drop_film_1024^3_1000to1: film + drop + 0-4 droplets, periodic x,y, Neumann z, Fourier-divergence RHS"),
    "sphere_32": dict(kind="config1", n=32,
                      desc="sphere_32^3_1000to1: R 0.2 centred, Neumann walls, N(0,1) RHS"),
    "projection_128": dict(kind="projection", n=128,
                           desc="projection step at 128^3: S = div u*/dt of a Fourier MAC velocity field on the "
                                "drop/film density (1000:1, periodic x,y, Neumann z), solve, u = u* - dt grad p / rho"),
    "batch64": dict(kind="batch", n=0,
                    desc="batch of 64 grids, n in {32,48,64,96,128}^3, seeded spheres R 0.05-0.2, ratio {10,100,1000}, "
                         "Neumann walls, N(0,1) RHS; one batched graph launch per solve of all 64"),
    "serve_stream": dict(kind="serve", n=0,
                         desc="served stream: Poisson arrivals, n log-uniform in [64,512] rounded to "
                              "{64,96,128,192,256,384,512}, drop/film fields, ratio 10-1000, continuous batching"),
}


PROLONG = {"trilinear": 0, "flux": 1}
SOLVER = {"mg": 0, "pcg": 1}


def reduce_max(value, dist):
    """Largest value over the ranks: the job takes as long as its slowest rank."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_value(world, units_per_rank, total_ms):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / (total_ms / 1000.0)


def make_problem(name):
    from paper_1410_8568_gb300 import inputs as I
    w = WORKLOADS[name]
    if w["kind"] == "config1":
        return I.config1(w["n"])
    if w["kind"] == "config2":
        return I.config2(w["n"])
    return I.config3(w["n"])


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources that define the profiled smoother kernels: the flat
    half-sweep (mg_tiles.cu), the one-pass sweeps (mg_fused.cu, mg_staged.cu), the per-quad
    relaxation they share (mg_stencil.cuh, mg_xprec.cuh) and the views and
    launch helpers (mg_device.cuh, mg_launch.cuh)."""
    h = hashlib.sha256()
    for f in ("mg_tiles.cu", "mg_fused.cu", "mg_staged.cu", "mg_stencil.cuh", "mg_xprec.cuh", "mg_device.cuh",
              "mg_launch.cuh"):
        with open(os.path.join(ROOT, "paper_1410_8568_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, kernel="smooth"):
    """DRAM bytes per launch of the dominant kernel (the finest-level half-sweep,
    "smooth", or one-pass sweep, "sweep") from the committed ncu summary, or None
    if absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "%s_level0_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None
        self.windows = []

    def window(self, t0, t1):
        """Keep the samples taken between wall times t0 and t1 (time.time())."""
        self.windows.append((t0, t1))

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if self.windows and not any(a <= ts <= b for a, b in self.windows):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "sampled": "every 200 ms, kept inside the timed regions (%d windows)" % len(self.windows)}


def level_shapes(shape):
    """Multigrid levels of a grid: all axes halved while every axis is even and > 2."""
    out = [tuple(shape)]
    while all(n % 2 == 0 and n > 2 for n in out[-1]):
        out.append(tuple(n // 2 for n in out[-1]))
    return out


def count_launches(shape, iters, steps, nu1=2, nu2=2, inner=3, tail_cells=4096, mixed=True, pcg=False,
                   xp=False, onepass=False, staged=False):
    """Kernels of one solve step: coefficient set-up, prologue, refinement (or CG) steps, epilogue.
    In FP32 cycles the levels of at most tail_cells cells (below the finest) run in one launch;
    with more than one V-cycle per refinement step each step starts with a step-control kernel.
    onepass: the finest level runs one launch per red-black sweep instead of two; staged: with a
    staged shape, the post-sweeps of a step's last cycle still run as half-sweep pairs."""
    lv = level_shapes(shape)
    L = len(lv)
    lt = next((l for l in range(1, L - 1) if math.prod(lv[l]) <= tail_cells), L) if mixed else L
    normal = lt if lt < L else L - 1
    setup = 1 + (L - 1) + 1            # faces from density, coarsening per level, coarsest inverse
    prologue = 6                       # begin, sum b, mean, residual, finalize, loop control
    if not pcg:
        prologue += 2 + (1 if xp else 0)  # b - mean b, its norm (+ float forms of b and p)
    # half-sweeps, restriction, prolongation per regular level (below the finest the
    # restriction into a level does its zero-start red half-sweep); tail or coarsest
    cycle = normal * (2 * nu1 + 1 + 1 + 2 * nu2) - (normal - 1) + 1
    if pcg:
        prologue += inner * cycle + 3  # first preconditioning: V-cycles, z and its sums, direction
        per_step = 4 + 3 + 1           # A d, alpha, update, test; z, beta, direction; loop control
    else:
        per_step = 3 + (1 if inner > 1 else 0)  # residual, finalize, loop control (+ step control)
    epilogue = 3                       # sum p, mean, p - mean
    if onepass and not pcg:
        cycle -= nu1 + nu2
        per_step += nu2 if staged else 0
    return setup + prologue + iters * cycle + steps * per_step + epilogue


def cpu_oracle_solve(P, faces, tol=TOL):
    import oracle
    t = time.perf_counter()
    r = oracle.solve(P.shape, P.bc, faces, P.rhs, tol=tol, max_cycles=200)
    return time.perf_counter() - t, r


def single_config(args, P, world):
    """config of the single-grid workloads (both arms)."""
    return {"workload": WORKLOADS[args.workload]["desc"], "grid": list(P.shape),
            "bc": list(P.bc), "density_ratio": P.ratio, "tol": TOL,
            "precision": "mixed: FP32 V(2,2) red-black cycles inside FP64 iterative refinement",
            "prolongation": args.prolongation, "solver": args.solver, "sweep": args.sweep,
            "step": "set density (faces, coarse faces, coarsest inverse) + cold-start solve",
            "l2": "flushed before every step (256 MB write, outside the step events)",
            "parallelism": "replicas" if world > 1 else "single"}


# grids above this size time the oracle by single V-cycles (a whole 512^3
# oracle solve takes about a minute on 16 cores)
REFERENCE_WHOLE_SOLVE_CELLS = 128 ** 3


def run_reference(args, name):
    """--impl reference: the FP64 CPU oracle as it stands, on the host cores.
    Small grids: one whole oracle solve to 1e-10 per step.  Larger grids: one
    oracle solve to 1e-10 first (untimed: it gives the cycles C a solve
    needs), and one call that stops before its first cycle (its set-up: the
    hierarchy, b - mean b and the starting residual, time s0); then every step
    is one oracle call of a single V(2,2) cycle, a solve is estimated from
    each step as s0 + C x (step time - s0), and solves/s = steps / the sum of
    those estimates."""
    import oracle
    P = make_problem(name)
    faces = oracle.faces_from_density(P.shape, P.bc, P.rho)
    cores = oracle.num_threads()
    whole = P.cells <= REFERENCE_WHOLE_SOLVE_CELLS
    if not whole:
        t_full, r = cpu_oracle_solve(P, faces)
        C = r.cycles
        t = time.perf_counter()
        oracle.solve(P.shape, P.bc, faces, P.rhs, tol=0.0, max_cycles=0)
        s0 = time.perf_counter() - t
    times = []
    for s in range(args.warmup + args.steps):
        if whole:
            dt, r = cpu_oracle_solve(P, faces)
        else:
            t = time.perf_counter()
            oracle.solve(P.shape, P.bc, faces, P.rhs, tol=0.0, max_cycles=1)
            dt = time.perf_counter() - t
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    if whole:
        value = len(times) / tot
        sample = "%d whole FP64 oracle solves of the workload to 1e-10 (%d V(2,2) cycles each)" % (
            len(times), r.cycles)
        solve_s = [t for t in times]
    else:
        solve_s = [s0 + C * max(t - s0, 0.0) for t in times]
        value = len(times) / sum(solve_s)
        sample = ("%d oracle calls of one V(2,2) cycle each on the workload; a whole oracle solve to 1e-10 "
                  "needs %d cycles (one measured before the steps: %.1f s) and its set-up (hierarchy, "
                  "b - mean b, starting residual) takes %.2f s (a call that stops before its first cycle); "
                  "a solve = set-up + %d x (step time - set-up)" % (len(times), C, t_full, s0, C))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": single_config(args, P, args.gpus),
        "p50_ms": 1000.0 * statistics.median(solve_s), "p99_ms": 1000.0 * float(np.percentile(solve_s, 99)),
        "latency": "per solve (whole solves, or C x the one-cycle step time)",
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _line(args, world, name, value, ms, p50, p99, extra):
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[name]["desc"], "tol": TOL,
                       "precision": "mixed: FP32 V(2,2) red-black cycles inside FP64 iterative refinement",
                       "prolongation": args.prolongation, "solver": args.solver,
                       "parallelism": "replicas" if world > 1 else "single"},
            "p50_ms": p50, "p99_ms": p99}
    line.update(extra)
    return line


def run_projection(args, rank, world, local_rank, dist):
    """One projection step per step: divergence, solve to 1e-10, velocity update."""
    import torch

    from paper_1410_8568_gb300 import gbmg
    from paper_1410_8568_gb300 import inputs as I

    n = WORKLOADS[args.workload]["n"]
    shape, bc, rho_np, u_np, dt = I.projection_problem(n, ratio=1000.0, dt=1e-2)
    rho = torch.from_numpy(rho_np).cuda()
    u0 = [torch.from_numpy(a).cuda() for a in u_np]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    res = {}
    for prec in (gbmg.MIXED, gbmg.FP64):
        with torch.cuda.stream(stream):
            S = gbmg.Solver(shape, bc, rho=rho, precision=prec, stream=stream,
                            prolongation=PROLONG[args.prolongation], solver=SOLVER[args.solver])
            u = [a.clone() for a in u0]
            p = torch.zeros_like(rho)
            src = torch.empty_like(rho)

            def step():
                for a, b in zip(u, u0):
                    a.copy_(b)
                p.zero_()
                return S.projection_step(u, dt, p, src, tol=TOL)

            for _ in range(args.warmup):
                step()
            stream.synchronize()
            if dist is not None:
                dist.barrier()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                st = step()
                ev[k][1].record(stream)
                if st.status != gbmg.OK:
                    raise RuntimeError("projection failed: %s" % gbmg.strerror(st.status))
            stream.synchronize()
        times = [a.elapsed_time(b) for a, b in ev]
        tot = sum(times)
        tot = reduce_max(tot, dist)
        # divergence left in the projected field, relative to the field's before
        div = torch.empty_like(rho)
        S.divergence(u, 1.0, div)
        S.divergence(u0, 1.0, src)
        res[prec] = dict(value=job_value(world, args.steps, tot), ms=tot / args.steps,
                         p50=statistics.median(times), p99=float(np.percentile(times, 99)), iters=st.iters,
                         div_ratio=(torch.linalg.vector_norm(div) / torch.linalg.vector_norm(src)).item())
        S.close()
    if rank == 0:
        m, f = res[gbmg.MIXED], res[gbmg.FP64]
        line = _line(args, world, args.workload, m["value"], m["ms"], m["p50"], m["p99"], {
            "iters": m["iters"], "divergence_after_over_before": m["div_ratio"],
            "step": "restore u*, p = 0; divergence + solve to 1e-10 + velocity update (timed, L2 flushed between steps)",
            "fp64": {"value": f["value"], "unit": "solves/s", "ms_per_step": f["ms"], "iters": f["iters"],
                     "divergence_after_over_before": f["div_ratio"]},
            "mixed_over_fp64": m["value"] / f["value"],
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": None})
        print(json.dumps(line))


def run_batch(args, rank, world, local_rank, dist):
    """64 independent grids of uneven sizes solved by one batched graph launch."""
    import torch

    import oracle
    from paper_1410_8568_gb300 import gbmg
    from paper_1410_8568_gb300 import inputs as I

    probs = I.config4_batch(64)
    rho = [torch.from_numpy(P.rho).cuda() for P in probs]
    rhs = [torch.from_numpy(P.rhs).cuda() for P in probs]
    ps = [torch.zeros_like(r) for r in rhs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    cells = sum(P.cells for P in probs)
    res = {}
    for prec in (gbmg.MIXED, gbmg.FP64):
        with torch.cuda.stream(stream):
            solvers = [gbmg.Solver(P.shape, P.bc, rho=r, precision=prec, stream=stream, prolongation=PROLONG[args.prolongation],
                                   solver=SOLVER[args.solver])
                       for P, r in zip(probs, rho)]
            B = gbmg.Batch(solvers)

        def step():
            for S, r, p in zip(solvers, rho, ps):
                S.set_density(r)
                p.zero_()
            return B.solve(rhs, ps, tol=TOL)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
            times = []
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            if dist is not None:
                dist.barrier()
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                sts = step()
                ev[k][1].record(stream)
            stream.synchronize()
        times = [a.elapsed_time(b) for a, b in ev]
        bad = [st.status for st in sts if st.status != gbmg.OK]
        if bad:
            raise RuntimeError("batch solve failed: %s" % bad)
        tot = sum(times)
        tot = reduce_max(tot, dist)
        errs = []
        if rank == 0:
            # error against the oracle's p* on the 4 smallest grids of the batch
            for g in sorted(range(len(probs)), key=lambda g: probs[g].cells)[:4]:
                P = probs[g]
                f = oracle.faces_from_density(P.shape, P.bc, P.rho)
                pstar = oracle.solve_exact(P.shape, P.bc, f, P.rhs).x
                x = ps[g].cpu().numpy()
                errs.append(float(np.linalg.norm(x - pstar) / np.linalg.norm(pstar)))
        res[prec] = dict(ms=tot / args.steps, value=job_value(world, 64 * args.steps, tot),
                         p50=statistics.median(times), p99=float(np.percentile(times, 99)),
                         iters=[st.iters for st in sts], err=max(errs) if errs else None)
        B.close()
        for S in solvers:
            S.close()
    if rank == 0:
        m, f = res[gbmg.MIXED], res[gbmg.FP64]
        line = _line(args, world, args.workload, m["value"], m["ms"], m["p50"], m["p99"], {
            "batch": {"grids": 64, "cells": cells, "cycles_min": min(m["iters"]), "cycles_max": max(m["iters"]),
                      "step": "set density of every grid + one batched solve (cold start) of all 64"},
            "err_vs_oracle_max_4_smallest": m["err"],
            "fp64": {"value": f["value"], "unit": "solves/s", "ms_per_step": f["ms"], "p50_ms": f["p50"],
                     "p99_ms": f["p99"], "err_vs_oracle_max_4_smallest": f["err"]},
            "mixed_over_fp64": m["value"] / f["value"],
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": None})
        print(json.dumps(line))


def run_serve(args, rank, world, local_rank, dist):
    """Poisson-arrival request stream through the continuous-batching server:
    for each offered load (a fraction of the measured capacity of the mixed
    path), the same seeded stream of requests in mixed precision and in FP64."""
    import torch

    from paper_1410_8568_gb300 import gbmg
    from paper_1410_8568_gb300 import inputs as I

    stream_spec = I.config5_stream(count=args.requests, rate=1.0)
    # one field per (edge, ratio bucket); the stream's ratios are log-uniform in
    # [10, 1000] and are mapped to the nearest of 10, 100, 1000
    buckets = (10.0, 100.0, 1000.0)

    def bucket(ratio):
        return min(buckets, key=lambda b: abs(math.log(b) - math.log(ratio)))

    fields, rhs_of = {}, {}
    for _, n, ratio, seed in stream_spec:
        rb = bucket(ratio)
        if (n, rb) in fields:
            continue
        shape = (n, n, n)
        if n not in rhs_of:
            rng = np.random.default_rng(I.config_seed(5, n))
            rhs_of[n] = torch.from_numpy(I.rhs_fourier_divergence(shape, I.DROP_FILM_BC, rng)).cuda()
        rho = torch.from_numpy(I.density_field(shape, 0.1, [((0.5, 0.5, 0.3), 0.125)], rb)).cuda()
        faces = [torch.empty_like(rho) for _ in range(3)]
        gbmg.faces_from_density(shape, I.DROP_FILM_BC, rho, *faces)
        fields[(n, rb)] = (shape, I.DROP_FILM_BC, faces, rhs_of[n])
        del rho
    torch.cuda.synchronize()
    sizes = sorted({n for _, n, _, _ in stream_spec})

    def solo_times(prec):
        """Service time of each edge alone (new coefficients + cold-start solve,
        as a request costs the server), the launch shapes tuned first."""
        svc = {}
        for n in sizes:
            (shape, bc, faces, rhs), = [v for (m, _), v in fields.items() if m == n][:1]
            with gbmg.Solver(shape, bc, faces=faces, precision=prec) as S:
                p = torch.zeros_like(rhs)
                S.solve(rhs, p)
                torch.cuda.synchronize()
                t = time.perf_counter()
                S.set_faces(*faces)
                S.solve(rhs, p.zero_())
                svc[n] = time.perf_counter() - t
        return svc

    def run_stream(prec, rate):
        srv = gbmg.Server(hbm_budget_bytes=args.hbm_budget << 30, max_slots=args.slots, precision=prec)
        arrivals = [a / rate for a, _, _, _ in stream_spec]
        pending, lat = {}, []
        k = done = 0
        t0 = time.perf_counter()
        while done < len(stream_spec):
            now = time.perf_counter() - t0
            while k < len(stream_spec) and arrivals[k] <= now:
                _, n, ratio, seed = stream_spec[k]
                shape, bc, faces, rhs = fields[(n, bucket(ratio))]
                p = torch.zeros_like(rhs)
                torch.cuda.synchronize()
                pending[srv.submit(shape, bc, faces, rhs, p, tol=TOL)] = (p, n)
                k += 1
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    rc, st = r
                    if rc != gbmg.OK:
                        raise RuntimeError("served solve failed: %s" % gbmg.strerror(rc))
                    lat.append((pending.pop(t)[1], st.ms))
                    done += 1
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        info = srv.info()
        srv.close()
        ms = [v for _, v in lat]
        per_size = {}
        for n in sizes:
            v = [m for e, m in lat if e == n]
            if v:
                per_size["%d^3" % n] = {"requests": len(v), "p50_ms": statistics.median(v),
                                        "p99_ms": float(np.percentile(v, 99))}
        return {"value": len(stream_spec) / wall, "wall_s": wall, "p50_ms": statistics.median(ms),
                "p99_ms": float(np.percentile(ms, 99)), "max_in_flight": info["max_in_flight"],
                "peak_bytes": info["peak_bytes"], "per_size": per_size}

    svc = solo_times(gbmg.MIXED)
    mean_svc = sum(svc[n] for _, n, _, _ in stream_spec) / len(stream_spec)
    capacity = 1.0 / mean_svc
    solo_fp64 = solo_times(gbmg.FP64)
    runs = {}
    for load in args.load:
        rate = load * capacity
        runs[load] = {"arrival_rate_per_s": rate,
                      "mixed": run_stream(gbmg.MIXED, rate), "fp64": run_stream(gbmg.FP64, rate)}
    if rank == 0:
        head = runs[0.8] if 0.8 in runs else runs[args.load[0]]
        m, f = head["mixed"], head["fp64"]
        loads = {("%g" % k): v for k, v in runs.items()}
        line = _line(args, world, args.workload, m["value"], 1000.0 * m["wall_s"] / len(stream_spec),
                     m["p50_ms"], m["p99_ms"], {
            "serve": {"requests": len(stream_spec), "slots": args.slots, "hbm_budget_gib": args.hbm_budget,
                      "capacity_solves_per_s": capacity,
                      "capacity_rule": "1 / mean solo service time (new coefficients + cold-start solve) of "
                                       "the stream's requests, mixed path",
                      "solo_ms": {"%d^3" % n: 1000.0 * v for n, v in svc.items()},
                      "solo_fp64_ms": {"%d^3" % n: 1000.0 * v for n, v in solo_fp64.items()},
                      "headline_load": 0.8 if 0.8 in runs else args.load[0],
                      "latency": "submission to completion, ms",
                      "lanes": "size lanes of up to 64^3, 128^3, 256^3 and larger grids, one stream each, "
                               "smaller grids at higher stream priority",
                      "tuning": "launch shapes of every size tuned before the stream starts",
                      "loads": loads},
            "fp64": {"value": f["value"], "unit": "solves/s", "p50_ms": f["p50_ms"], "p99_ms": f["p99_ms"]},
            "mixed_over_fp64": m["value"] / f["value"],
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": None})
        print(json.dumps(line))


# Algorithmic bytes per finest cell of the level-0 kernels (FP32 cycle, s = 4 B):
# a full red + black sweep reads x, b and the 3 face arrays and writes x (6 s),
# so each of its two half-sweep launches counts half of that; the residual +
# restriction reads x, b, 3 faces and writes r/8 (5.125 s); the prolongation +
# correction reads e/8 and reads and writes x (2.125 s).
ALG_BPC = {"half": 12.0, "sweep": 24.0, "restrict": 20.5, "prolong": 8.5}
# Bytes the unfused kernels actually move per finest cell: a half-sweep reads
# all of x and the 3 face arrays, the colour's sectors of b (the whole b: the
# two cells of a colour share the quad's sector) and writes the quad (x).
ACT_BPC = {"half": 20.0, "sweep": 24.0}
# The one-pass sweep (both colours in one launch, two iterate buffers) reads
# the old iterate, b and the 3 face arrays once and writes the new iterate: the
# algorithmic bytes (its halo rows and planes are re-read through L2).
# FP64 residual of a refinement step: reads p, b - mean b and 3 FP64 faces,
# writes the FP32 residual (44 B); 6 differences, 1 product and 5 fused
# multiply-adds, the subtraction from b and the scale (14 FP64 operations) and
# the FP64 -> FP32 conversion, which this GPU also issues to its FP64 pipe.
RES_BPC, RES_FP64_OPS = 44.0, 15.0


def oracle_reference_run(P, tol=TOL):
    """The oracle's p* (iterated to rounding level) and the time it took:
    (p*, seconds, cycles run, cycles that reached tol)."""
    import oracle
    faces = oracle.faces_from_density(P.shape, P.bc, P.rho)
    t = time.perf_counter()
    r = oracle.solve_exact(P.shape, P.bc, faces, P.rhs)
    dt = time.perf_counter() - t
    hist = r.history
    reach = next((k for k in range(len(hist)) if hist[k] <= tol * r._bnorm), len(hist) - 1)
    return r.x, dt, r.cycles, reach


def oracle_single_thread(P, cycles):
    """The oracle on one host thread, a bounded sample: its set-up (a call that
    stops before the first cycle) and one V(2,2) cycle, each timed; a solve =
    set-up + `cycles` cycles."""
    import oracle
    faces = oracle.faces_from_density(P.shape, P.bc, P.rho)
    threads = oracle.num_threads()
    oracle.set_threads(1)
    try:
        t = time.perf_counter()
        oracle.solve(P.shape, P.bc, faces, P.rhs, tol=0.0, max_cycles=0)
        s0 = time.perf_counter() - t
        t = time.perf_counter()
        oracle.solve(P.shape, P.bc, faces, P.rhs, tol=0.0, max_cycles=1)
        s1 = time.perf_counter() - t
    finally:
        oracle.set_threads(threads)
    cyc = max(s1 - s0, 1e-9)
    return {"value": 1.0 / (s0 + cycles * cyc), "unit": "solves/s", "cores": 1,
            "sample": "one thread: set-up %.2f s and one V(2,2) cycle %.2f s, timed; a solve = set-up + %d "
                      "cycles" % (s0, cyc, cycles)}


def run_single(args, rank, world, local_rank, dist):
    """One grid per step: new density in, cold-start solve to 1e-10 (mixed,
    FP64, extended-precision outer iteration), end to end through the host
    entry point, per-launch timing of the level-0 kernels."""
    import torch

    from paper_1410_8568_gb300 import gbmg

    P = make_problem(args.workload)
    N = P.cells
    rho_h = torch.from_numpy(P.rho).pin_memory()
    rhs_h = torch.from_numpy(P.rhs).pin_memory()
    rho = rho_h.cuda()
    rhs = rhs_h.cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    clocks = ClockSampler(local_rank)
    clocks.start()

    def timed(solver, steps, host=False, window=False):
        """Per-step device times (ms) and the last stats."""
        p = torch.zeros_like(rhs)
        ph = torch.zeros(P.rho.shape, dtype=torch.float64).pin_memory()
        st = None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0 = time.time()
        with torch.cuda.stream(stream):
            for s in range(steps):
                flush.fill_(float(s))
                if host:
                    # the caller's starting iterate (zero) is prepared before the
                    # step; its copy to the device is part of the step
                    ph.zero_()
                ev[s][0].record(stream)
                if host:
                    st = solver.step_host(rho_h.numpy(), rhs_h.numpy(), ph.numpy(), tol=TOL)
                else:
                    p.zero_()
                    solver.set_density(rho)
                    st = solver.solve(rhs, p, tol=TOL)
                ev[s][1].record(stream)
                if st.status != gbmg.OK:
                    raise RuntimeError("solve failed: %s" % gbmg.strerror(st.status))
            stream.synchronize()
        if window:
            clocks.window(t0, time.time())
        times = [a.elapsed_time(b) for a, b in ev]
        return times, st, p

    # the headline (FP32 cycles in the FP64 outer iteration), the FP64 path, and
    # the extended-precision outer iteration (multigrid iteration only)
    modes = [("mixed", gbmg.MIXED, gbmg.OUTER_FP64), ("fp64", gbmg.FP64, gbmg.OUTER_FP64)]
    if args.solver == "mg":
        modes.append(("mixed_xp", gbmg.MIXED, gbmg.OUTER_XP))
    results = {}
    solvers = {}
    for key, prec, outer in modes:
        with torch.cuda.stream(stream):
            sweep = {"auto": gbmg.SWEEP_AUTO, "half": gbmg.SWEEP_HALF}.get(args.sweep)
            solvers[key] = gbmg.Solver(P.shape, P.bc, rho=rho, precision=prec, stream=stream, outer=outer,
                                       prolongation=PROLONG[args.prolongation], solver=SOLVER[args.solver],
                                       sweep=int(args.sweep) if sweep is None else sweep)
        S = solvers[key]
        timed(S, args.warmup)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        times, st, p = timed(S, args.steps, window=True)
        torch.cuda.synchronize()
        tot = reduce_max(sum(times), dist)
        # host copy of the last step's result, taken at once for the oracle comparison
        x_host = p.cpu().numpy().copy() if (rank == 0 and N <= ORACLE_MAX_CELLS) else None
        results[key] = dict(ms=tot / args.steps, value=job_value(world, args.steps, tot),
                            p50=statistics.median(times), p99=float(np.percentile(times, 99)),
                            iters=st.iters, gamma=st.gamma, rel_res=st.rel_res,
                            levels=S.num_levels(), x=x_host, inner=S.resolved_params()["inner_cycles"],
                            refine_steps=st.steps)
        if key == "mixed_xp":
            # its residual kernel, per-launch events (NVTX range for a profiler:
            # ncu --nvtx --nvtx-include "profile_pass_xp/")
            S.profile(True)
            try:
                torch.cuda.nvtx.range_push("profile_pass_xp")
                nvtx_xp = True
            except (RuntimeError, AttributeError):
                nvtx_xp = False
            timed(S, 3)
            if nvtx_xp:
                torch.cuda.nvtx.range_pop()
            n_x, ms_x = S.profile_read(gbmg.K_RESIDUAL, 0)
            S.profile(False)
            results[key]["residual_avg_launch_us"] = 1000.0 * ms_x / max(1, n_x)
        if key != "mixed":
            S.close()  # frees its hierarchy before the next one is built
            del solvers[key]

    # end to end through the host entry point (pinned buffers, copies inside)
    S = solvers["mixed"]
    timed(S, 2, host=True)
    e2e_times, _, _ = timed(S, args.steps, host=True, window=True)
    e2e_tot = reduce_max(sum(e2e_times), dist)
    clock_rec = clocks.stop()

    # roofline of the dominant kernel: the finest-level sweep (one-pass) or
    # half-sweep, per-launch events
    v0 = S.tile_choice(gbmg.TILE_HALF, 0)
    sv = S.tile_choice(gbmg.TILE_SWEEP, 0)
    kk = "sweep" if sv > 0 else "half"
    S.profile(True)
    prof_steps = max(3, min(args.steps, 10))
    # an NVTX range lets a profiler select these host-loop launches
    # (ncu --nvtx --nvtx-include "profile_pass/")
    try:
        torch.cuda.nvtx.range_push("profile_pass")
        nvtx = True
    except (RuntimeError, AttributeError):
        nvtx = False
    timed(S, prof_steps)
    if nvtx:
        torch.cuda.nvtx.range_pop()
    n_l, ms_l = S.profile_read(gbmg.K_SMOOTH, 0)
    n_r, ms_r = S.profile_read(gbmg.K_RESIDUAL, 0)
    peak, peak_kind = read_peaks()
    per_kernel = {}
    for name, kind in (("restrict", gbmg.K_RESTRICT), ("prolong", gbmg.K_PROLONG)):
        n_k, ms_k = S.profile_read(kind, 0)
        if n_k:
            us = 1000.0 * ms_k / n_k
            b = ALG_BPC[name] * N
            per_kernel[name] = {"avg_launch_us": us, "algorithmic_bytes_per_launch": b,
                                "achieved_gbs": b / (us * 1e3), "frac": b / (us * 1e3) / peak, "bound": "hbm"}
    S.profile(False)
    fp64_rate = gbmg.probe_fp64_rate(stream=stream)
    res_us = 1000.0 * ms_r / max(1, n_r)
    residual = {"avg_launch_us": res_us, "launches_timed": n_r,
                "bytes_per_launch": RES_BPC * N, "achieved_gbs": RES_BPC * N / (res_us * 1e3),
                "hbm_frac": RES_BPC * N / (res_us * 1e3) / peak,
                "fp64_ops_per_cell": RES_FP64_OPS,
                "fp64_ops_per_s": RES_FP64_OPS * N / (res_us * 1e-6),
                "fp64_frac": RES_FP64_OPS * N / (res_us * 1e-6) / fp64_rate,
                "bound": "fp64 pipe (min of HBM and FP64 issue rate: the larger fraction)"}
    avg_s = ms_l / n_l / 1000.0
    bytes_launch = ALG_BPC[kk] * N
    achieved = bytes_launch / avg_s / 1e9
    traffic = profiled_traffic(args.workload, "sweep" if sv > 0 else "smooth")

    # error of each result against the FP64 oracle's converged solution p*, and
    # the oracle's own time (its p* run: mean cycle time x the cycles it needed
    # to reach the tolerance)
    errors, cpu = {}, None
    if rank == 0 and N <= ORACLE_MAX_CELLS:
        import oracle
        pstar, dt, ncyc, reach = oracle_reference_run(P)
        nrm = np.linalg.norm(pstar)
        for key in ("mixed", "fp64", "mixed_xp"):
            if key in results:
                errors[key] = float(np.linalg.norm(results[key]["x"] - pstar) / nrm)
        if not args.no_cpu_baseline:
            t_solve = dt / ncyc * reach
            cpu = {"value": 1.0 / t_solve, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
                   "sample": "the oracle's p* run on this workload (%d V(2,2) cycles to rounding level, %.1f s), "
                             "timed; solves/s = 1 / (mean cycle time x the %d cycles that reached 1e-10)" %
                             (ncyc, dt, reach),
                   "single_thread": oracle_single_thread(P, reach)}
    elif rank == 0 and not args.no_cpu_baseline:
        import oracle
        faces = oracle.faces_from_density(P.shape, P.bc, P.rho)
        t = time.perf_counter()
        oracle.solve(P.shape, P.bc, faces, P.rhs, tol=0.0, max_cycles=2)
        dt = (time.perf_counter() - t) * results["fp64"]["iters"] / 2.0
        cpu = {"value": 1.0 / dt, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "2 FP64 oracle V(2,2) cycles of the workload, scaled to %d cycles per solve" %
                         results["fp64"]["iters"]}

    if rank == 0:
        m, f = results["mixed"], results["fp64"]
        launches = args.steps * count_launches(P.shape, m["iters"], m["refine_steps"], inner=m["inner"],
                                               pcg=args.solver == "pcg", onepass=sv > 0,
                                               staged=sv > 0 and gbmg.sweep_shape(sv)[2] > 0)
        xp = results.get("mixed_xp")
        line = {
            "metric": METRIC, "value": m["value"], "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": single_config(args, P, world),
            "p50_ms": m["p50"], "p99_ms": m["p99"],
            "iters": m["iters"], "refine_steps": m["refine_steps"], "inner_cycles": m["inner"],
            "gamma": m["gamma"], "rel_res": m["rel_res"],
            "err_vs_oracle": errors.get("mixed"),
            "fp64": {"value": f["value"], "unit": "solves/s", "ms_per_step": f["ms"], "p50_ms": f["p50"],
                     "p99_ms": f["p99"], "iters": f["iters"], "refine_steps": f["refine_steps"],
                     "inner_cycles": f["inner"], "gamma": f["gamma"], "rel_res": f["rel_res"],
                     "err_vs_oracle": errors.get("fp64")},
            "mixed_over_fp64": m["value"] / f["value"],
            "mixed_xp": None if xp is None else {
                "precision": "FP32 V(2,2) cycles in the extended-precision outer iteration (three-float "
                             "iterate, float-pair faces and b, error-free FP32 residual; FP64 only in "
                             "the set-up and final conversion)",
                "value": xp["value"], "unit": "solves/s", "ms_per_step": xp["ms"],
                "p50_ms": xp["p50"], "p99_ms": xp["p99"], "iters": xp["iters"],
                "refine_steps": xp["refine_steps"], "rel_res": xp["rel_res"],
                "err_vs_oracle": errors.get("mixed_xp"),
                "residual_avg_launch_us": xp["residual_avg_launch_us"],
                "over_mixed": xp["value"] / m["value"]},
            "err_note": None if errors else "oracle p* not computed above %d cells" % ORACLE_MAX_CELLS,
            "e2e": {"value": job_value(world, args.steps, e2e_tot), "unit": "solves/s",
                    "h2d_bytes_per_step": 3 * 8 * N, "d2h_bytes_per_step": 8 * N},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": ("FP32 one-pass red-black sweep of level 0 (both colours in one launch), "
                                    "shape %d (%d threads, %d planes per block, tile of %d cells along x; "
                                    "0: whole rows)" % ((sv,) + gbmg.sweep_shape(sv)))
                                   if sv > 0 else
                                   ("FP32 half-sweep of level 0 (one red or black colour), launch shape %d "
                                    "(%d threads x %d quads)" % ((v0,) + gbmg.tile_shape(v0))),
                         "bytes_rule": "algorithmic: 6 s = 24 B per cell per full red+black sweep (%s)" %
                                       ("one launch" if sv > 0 else "half per colour launch: 12 B x cells"),
                         "bytes_per_launch": bytes_launch,
                         "actual_bytes_per_launch": ACT_BPC[kk] * N,
                         "frac_on_actual_bytes": ACT_BPC[kk] * N / avg_s / 1e9 / peak,
                         "traffic_over_algorithmic": None if traffic is None else traffic / bytes_launch,
                         "avg_launch_us": avg_s * 1e6, "launches_timed": n_l, "peak_source": peak_kind,
                         "level0_kernels": per_kernel,
                         "residual_fp64": residual,
                         "fp64_peak": {"fma_per_s": fp64_rate, "gflops": 2e-9 * fp64_rate,
                                       "how": "mg_probe_fp64_rate: 8 independent FP64 FMA chains per thread, "
                                              "8 blocks of 256 threads per SM, best of 3 event-timed launches"}},
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clock_rec,
        }
        print(json.dumps(line))
    for S in solvers.values():
        S.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="drop_film_512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prolongation", default="trilinear", choices=["trilinear", "flux"],
                    help="prolongation of the V-cycle: trilinear or flux-conserving (Sec. 2.3 item 4)")
    ap.add_argument("--solver", default="mg", choices=["mg", "pcg"],
                    help="outer iteration: V-cycles in FP64 refinement (mg) or V-cycle-preconditioned CG (pcg)")
    ap.add_argument("--sweep", default="auto",
                    help="finest-level red-black sweep of the single-grid workloads: auto (timed at create), "
                         "half (two half-sweep launches) or a one-pass shape 1..6")
    ap.add_argument("--requests", type=int, default=500, help="serve_stream: requests in the stream")
    ap.add_argument("--load", type=float, nargs="+", default=[0.5, 0.8, 1.0],
                    help="serve_stream: arrival rates as fractions of the measured capacity of the mixed path")
    ap.add_argument("--slots", type=int, default=8, help="serve_stream: most requests on the GPU at once")
    ap.add_argument("--hbm-budget", type=int, default=64, help="serve_stream: GiB of device memory for hierarchies")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, args.workload)
        return

    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__
    __graft_entry__.build()

    kind = WORKLOADS[args.workload]["kind"]
    run = {"batch": run_batch, "serve": run_serve, "projection": run_projection}.get(kind, run_single)
    run(args, rank, world, local_rank, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
