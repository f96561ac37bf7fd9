"""Benchmark: milliseconds to a 1e-8 relative residual, AMG-DD vs the plain
V-cycle on the same hierarchy, one GB300 per process.

Workload: 3D 7-point Poisson on a 128^3 interior grid (2,097,152 unknowns,
Dirichlet), b ~ U[-1,1] (seed 0), x0 = 0, 512 box subdomains of 16^3,
padding 2 on every level, 2 AlgFAC V(1,1)-cycles per AMG-DD iteration, FP64.
One step = one AMG-DD solve to 1e-8 (residual, restriction, composite-grid
FAC cycles and owned corrections, repeated until converged). The inputs
(7.1 GB of composite-grid operators, 183 MB fine matrix) exceed the 126 MB L2,
so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

`--impl reference` times the CPU oracle (plain C, all host cores) on the
same workload: every step is one AMG-DD iteration, scaled by the number of
iterations to 1e-8.
"""
from __future__ import annotations

import argparse
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

import amgdd_inputs as I  # noqa: E402

WORKLOAD = "poisson3d_128"
METRIC = "ms to 1e-8 rel. residual & HBM GB/s: AMG-DD vs plain V-cycle, 1 GB300"
TOL = 1e-8


def _config(w):
    n = int(len(w["rowptr"]) - 1)
    e = w["shape"][0]
    return {
        "workload": "3D 7-point Poisson %d^3 (N=%d), %d subdomains of 16^3, padding %d, "
                    "2 AlgFAC V(1,1) per iteration, FP64, b~U[-1,1] seed 0, x0=0" % (e, n, w["nsub"], w["padding"]),
        "n": n, "nnz": int(len(w["col"])), "nsub": int(w["nsub"]),
        "padding": int(w["padding"]), "n_fac": int(w["n_fac"]), "tol": TOL,
        "l2_policy": "inputs larger than L2 (composite operators 7 GB, fine matrix 183 MB)",
    }


# FAC kernel of each autotuner candidate: the single-column kernel (schedules
# 1-9, source kernels.cu), the several-column kernel (source fac_multi.cuh),
# the one with each grid's work vectors in shared memory (fac_vsm.cu) or the
# one cycling each grid with a cluster of blocks (fac_cluster.cu)
FAC_KERNELS = {"k_fac_all_grids": "kernels.cu", "k_fac_all_grids_r": "fac_multi.cuh",
               "k_fac_grids_vsm": "fac_vsm.cu", "k_fac_cluster": "fac_cluster.cu", "k_fac_teams": "fac_multi.cuh"}


def _fac_kernel(candidate):
    if candidate is None or candidate < 9:
        return "k_fac_all_grids"
    if candidate in (26, 27):
        return "k_fac_grids_vsm"
    if candidate == 31:
        return "k_fac_teams"
    return "k_fac_cluster" if candidate >= 28 else "k_fac_all_grids_r"


def _measured_traffic(workload, kernel, candidate):
    """DRAM bytes per FAC launch from the committed ncu summary of this
    workload (profiles/<kernel>_<workload>_dram.md) for this kernel, when
    that summary was taken with the same candidate and the kernel source is
    unchanged since (sha1); None otherwise."""
    if workload is None:
        return None
    import hashlib
    summ = os.path.join(ROOT, "profiles", "%s_%s_dram.md" % (kernel, workload))
    src = os.path.join(ROOT, "paper_1906_10575_gb300", "csrc", FAC_KERNELS[kernel])
    try:
        txt = open(summ).read()
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    fields = dict(l.split(": ", 1) for l in txt.splitlines()
                  if l.startswith(("source_sha1:", "traffic_bytes", "candidate:")))
    if fields.get("source_sha1") != sha:
        return None
    if candidate is not None and fields.get("candidate") not in (None, str(candidate)):
        return None
    return int(fields["traffic_bytes_per_launch"])


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# FP64 peak of a GB300: 1.25 TFLOP/s nominal dense (2 DFMA per SM per clock at
# 2.07 GHz boost on 152 SMs is 1.26 TFLOP/s).
FP64_PEAK_TFLOPS = 1.25
# FP64 FMA throughput measured on this machine's GB300 with 8 independent fma
# chains per thread (1.198 TFLOP/s)
FP64_PROBE_TFLOPS = 1.198


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_fac_bytes(st, nfac, si=2, sv=8.0):
    """Bytes one all-grids FAC launch must move: the per-composite-grid formula
    sum_c sum_{l<L} [3 M(A_l real rows) + [c>1] M(A_{l+1} real rows) + 2 M(P_l)
    + 8 * k * |Dbar_l|] summed over grids, with M(X) = nnz*(8 + si) + 4*rows,
    si = 2 (16-bit local columns) and k = 8 vector touches per point and
    level visit. A_l real rows are read by the pre- and post-smoothing sweeps
    and by s_l + A_l t_l; P_l and R_l = P_l^T once each."""
    L = st.num_levels - 1

    def M(nnz, rows):
        return nnz * (sv + si) + 4.0 * rows

    tot = 0.0
    for c in range(1, nfac + 1):
        for l in range(L):
            bar = st.comp_real[l] + st.comp_ghost[l]
            tot += 3 * M(st.comp_nnz_real[l], st.comp_real[l])
            if c > 1:
                tot += M(st.comp_nnz_real[l + 1], st.comp_real[l + 1])
            tot += 2 * M(st.comp_nnz_P[l], bar)
            tot += sv * 8 * bar
    return tot


def algorithmic_fac_flops(st, nfac):
    """FP64 flops of one FAC launch under the same count: 2 per operator
    entry of the formula above, plus the dense coarsest products."""
    L = st.num_levels - 1
    fma = 0.0
    for c in range(1, nfac + 1):
        for l in range(L):
            fma += 3 * st.comp_nnz_real[l] + 2 * st.comp_nnz_P[l]
            if c > 1:
                fma += st.comp_nnz_real[l + 1]
        fma += st.nsub * float(st.n[L]) ** 2
    return 2.0 * fma


def algorithmic_solve_bytes(st, fac_bytes, iters):
    """Per AMG-DD iteration: residual (A_0 + 3 vectors), restriction chain
    (R_l + 2 vectors), the FAC launch; plus one final residual."""
    L = st.num_levels - 1
    res = 12.0 * st.nnz[0] + 4.0 * st.n[0] + 24.0 * st.n[0]
    rst = sum(12.0 * st.nnz_P[l] + 4.0 * st.n[l + 1] + 8.0 * (st.n[l] + st.n[l + 1]) for l in range(L))
    return iters * (res + rst + fac_bytes) + res


def vcycle_bytes(st, iters):
    """Per V(1,1)-cycle: A_l read by 4 half-sweeps (C, F, F, C: two full
    sweeps), the residual and the level-0 residual check; P_l, R_l once."""
    L = st.num_levels - 1
    b = 0.0
    for l in range(L):
        b += 3 * (12.0 * st.nnz[l] + 4.0 * st.n[l]) + 2 * 12.0 * st.nnz_P[l] + 10 * 8.0 * st.n[l]
    b += 12.0 * st.nnz[0] + 28.0 * st.n[0]
    return iters * b


def run_reference(args, w):
    """CPU oracle arm: each step is one AMG-DD iteration on all host cores."""
    from oracle import Oracle
    cores = os.cpu_count()
    o = Oracle(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"],
               interp=args.interp, coarsen=args.coarsen)
    b = w["b"]
    # iterations to 1e-8 (identical on every implementation of the same arithmetic)
    t0 = time.perf_counter()
    _, hist = o.amgdd_solve(b, w["n_fac"], tol=TOL, maxit=100)
    full = (time.perf_counter() - t0) * 1e3
    iters = len(hist) - 1
    x = np.zeros(o.n)
    for _ in range(max(0, args.warmup - 1)):
        x = o.amgdd_iteration(b, x, w["n_fac"])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        x = o.amgdd_iteration(b, x, w["n_fac"])
        times.append((time.perf_counter() - t0) * 1e3)
    per_iter = statistics.median(times)
    value = per_iter * iters
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "ms",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(per_iter, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(_config(w), interp=args.interp, coarsen=args.coarsen),
        "iterations": iters, "full_solve_ms": round(full, 1),
        "cpu_baseline": {"value": round(value, 3), "unit": "ms", "cores": cores, "kind": "oracle",
                         "cpu_model": _cpu_model(),
                         "sample": "one AMG-DD iteration over all 512 composite grids per step "
                                   "(OpenMP over grids), x %d iterations to 1e-8" % iters},
        "e2e": {"value": round(value, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def max_over_ranks(values, dist=None):
    """Element-wise maximum of per-rank timings over all ranks (the slowest
    replica sets the whole-job time); identity without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def _cpu_model():
    """Host CPU model from lscpu (Arm hosts have no 'model name' in
    /proc/cpuinfo), else from /proc/cpuinfo, else the platform string."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(w, iters, interp="direct", coarsen="rs", one_thread_budget_s=150.0):
    """The oracle's full AMG-DD solve to 1e-8 (Algorithm 2 with AlgFAC on
    every composite grid, OpenMP over grids) timed on all host cores and on
    one thread. The one-thread solve runs in full when its estimate (all-core
    time x cores) stays within one_thread_budget_s; otherwise one iteration
    at one thread is timed and scaled by the iteration count, which the
    sample text then says."""
    from oracle import Oracle, set_threads
    cores = os.cpu_count()
    o = Oracle(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], interp=interp, coarsen=coarsen)
    b = w["b"]
    all_threads = set_threads(cores)
    t0 = time.perf_counter()
    _, hist = o.amgdd_solve(b, w["n_fac"], tol=TOL, maxit=200)
    t_all = time.perf_counter() - t0
    it = len(hist) - 1
    set_threads(1)
    if t_all * all_threads <= one_thread_budget_s:
        t0 = time.perf_counter()
        o.amgdd_solve(b, w["n_fac"], tol=TOL, maxit=200)
        t_one = time.perf_counter() - t0
        how = "full solve"
    else:
        t0 = time.perf_counter()
        o.amgdd_iteration(b, np.zeros(o.n), w["n_fac"])
        t_one = (time.perf_counter() - t0) * it
        how = "one iteration x %d (full solve estimated above %.0f s)" % (it, one_thread_budget_s)
    set_threads(all_threads)
    return {"value": round(t_all * 1e3, 2), "unit": "ms", "cores": all_threads, "kind": "oracle",
            "all_cores_ms": round(t_all * 1e3, 2), "one_thread_ms": round(t_one * 1e3, 2),
            "iterations": it, "cpu_model": _cpu_model(),
            "sample": "the oracle's whole AMG-DD solve to 1e-8 (%d iterations, all %d composite grids) on %d "
                      "threads; one thread: %s" % (it, w["nsub"], all_threads, how)}


def _ev_ms(stream, fn, k=1):
    """Mean CUDA-event time of k calls of fn on `stream` (ms)."""
    import torch
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(k):
        fn()
    a1.record(stream)
    a1.synchronize()
    return a0.elapsed_time(a1) / k


def run_extra(args, name, stream, dist, local, emit=True):
    """The other configurations, one JSON line each (not the headline):

    kappa3d_256 -- 256^3 variable-coefficient diffusion, 4096 composite grids,
      FP32 AlgFAC inside FP64 refinement; AMG-DD against the FP64 V-cycle on
      the same hierarchy, and the final error against the FP64 AMG-DD
      solution (whose iterates equal the CPU oracle's bit for bit).
    batched_64 -- 64 independent Poisson systems as one block-diagonal matrix,
      4 right-hand sides, FP32 AlgFAC inside FP64 refinement, one
      several-column FAC launch per iteration in a CUDA graph; against four
      single-column FP64 V-cycle solves on the same hierarchy.
    aniso2d_512 -- 2D rotated anisotropic diffusion (the paper's second test
      problem as finite differences), FP64, AMG-DD against the V-cycle.
    poisson2d_64 -- 2D 5-point Poisson 64^2, 16 composite grids, padding 1,
      FP64: the small case, where every launch of either method is latency
      bound and the whole problem fits L2, so a 256 MB buffer is written
      before every timed solve to start each one from a cold L2; ms only (no
      bandwidth fraction for an L2-resident problem)."""
    import torch
    from paper_1906_10575_gb300 import Solver, capi

    shape = (args.edge, args.edge) if name == "poisson2d_64" and args.edge > 0 else None
    w = I.workload(name, seed=0, nsys=args.nsys if "nsys" in I.WORKLOADS[name] else None, shape=shape)
    if args.padding >= 0:
        w["padding"] = args.padding
    n = int(len(w["rowptr"]) - 1)
    hbm, peak_kind = _peaks()
    multi = "nsys" in I.WORKLOADS[name]
    small = name == "poisson2d_64"
    prec = int(w.get("precision", 0))
    maxit = 2000
    t0 = time.perf_counter()
    s = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=w["n_fac"],
               interp=args.interp, coarsen=args.coarsen,
               precision=prec, schedule=args.schedule, stream=stream,
               max_coarse=16 * (len(w["edges"]) if multi else 1))
    setup_s = time.perf_counter() - t0
    st = s.stats
    nrhs = w["nrhs"] if multi else 1
    Bh = w["B"] if multi else w["b"][:, None]
    B = torch.from_numpy(np.ascontiguousarray(Bh)).cuda()
    X = torch.zeros_like(B)
    solve = (lambda: s.solve_multi(B, X, tol=TOL, max_iter=maxit, stream=stream)) if multi else \
        (lambda: s.solve(B[:, 0], X[:, 0], tol=TOL, max_iter=maxit, stream=stream))
    tune = None
    if args.candidate >= 0:
        capi.amgdd_set_fac_kernel(s.h, nrhs, args.candidate)
        tune = {"best_candidate": args.candidate, "ms_per_candidate": None}
    elif not args.no_autotune:
        # FP32 composite grids are compared with the oracle within rounding
        # anyway, so there the group-per-row candidates take part
        best, tms = capi.amgdd_autotune(s.h, nrhs, reps=2, stream=stream, allow_reordered=prec == 1)
        tune = {"best_candidate": best, "ms_per_candidate": [round(float(t), 3) for t in tms],
                "reordered_allowed": prec == 1}
    # the small workload fits L2: write a buffer twice its size before every
    # timed solve (outside the timed region)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda") if small else None

    def cold():
        if flush is not None:
            flush.fill_(1.0)
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        # the FAC launch alone, first (direct launches, before any solve):
        # from the restricted residuals of B (x = 0)
        off = int(s.offsets[-1])
        Rcols = []
        for j in range(nrhs):
            r = torch.zeros(off, dtype=torch.float64, device="cuda")
            capi.amgdd_residual(s.h, B[:, j].contiguous(), torch.zeros(n, dtype=torch.float64, device="cuda"),
                                r[:n], stream)
            capi.amgdd_restrict(s.h, r, stream)
            Rcols.append(r)
        Xf = torch.zeros_like(X)
        if multi:
            Rm = torch.stack(Rcols, 1).contiguous()
            fac = lambda: capi.amgdd_fac_multi(s.h, Rm, Xf, stream)  # noqa: E731
        else:
            xf = torch.zeros(n, dtype=torch.float64, device="cuda")
            fac = lambda: capi.amgdd_fac(s.h, Rcols[0], xf, stream)  # noqa: E731
        fac()
        fac_ms = _ev_ms(stream, fac, 3)
        for _ in range(args.warmup):
            X.zero_()
            solve()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        times = []
        for _ in range(args.steps):
            X.zero_()
            cold()
            info = {}
            times.append(_ev_ms(stream, lambda: info.update(solve())))
        clocks = clk.stop()
        Xmix = X.clone()
        # FP64 V-cycle on the same hierarchy, column by column
        xv = torch.zeros(n, dtype=torch.float64, device="cuda")
        v_ms, v_it = 0.0, []
        for j in range(nrhs):
            bj = B[:, j].contiguous()
            xv.zero_()
            s.vcycle_solve(bj, xv, tol=TOL, max_iter=maxit, stream=stream)
            xv.zero_()
            cold()
            iv = {}
            v_ms += _ev_ms(stream, lambda: iv.update(s.vcycle_solve(bj, xv, tol=TOL, max_iter=maxit,
                                                                     stream=stream)))
            v_it.append(iv["iterations"])
    s.close()
    ms = statistics.median(times)
    ms, v_ms = max_over_ranks([ms, v_ms], dist)
    fac_b = algorithmic_fac_bytes(st, w["n_fac"], sv=4.0 if prec else 8.0)
    # several columns: the operator once, the vector touches once per column
    if multi:
        L = st.num_levels - 1
        vec = sum(4.0 * 8 * (st.comp_real[l] + st.comp_ghost[l]) for l in range(L)) * w["n_fac"]
        fac_b = fac_b + (nrhs - 1) * vec
    fac_gbs = fac_b / (fac_ms * 1e-3) / 1e9
    fac_kern = _fac_kernel(tune["best_candidate"] if tune else (None if not multi else 9))
    fac_cand = tune["best_candidate"] if tune else None
    fac_line = {"kernel": fac_kern, "candidate": fac_cand, "ms_per_launch": round(fac_ms, 3),
                "algorithmic_bytes": fac_b, "achieved_gbs": round(fac_gbs, 1), "peak_gbs": hbm,
                "hbm_frac": None if small else round(fac_gbs / hbm, 4),
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind}
    # DRAM traffic of the committed ncu capture of this workload and kernel
    # (1 pass, full size), when it matches the current source and candidate
    traffic = _measured_traffic("batched_64" if multi and args.nsys == 64 and args.padding < 0 else None,
                                fac_kern, fac_cand)
    if traffic is not None:
        fac_line["traffic"] = traffic
        fac_line["dram_gbs"] = round(traffic / (fac_ms * 1e-3) / 1e9, 1)
        fac_line["dram_frac"] = round(traffic / (fac_ms * 1e-3) / 1e9 / hbm, 4)
    err = None
    if not multi and prec == 1 and not args.no_fp64_check:
        # FP64 AMG-DD on the same problem: reference solution for the error
        s64 = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=w["n_fac"],
                     interp=args.interp, coarsen=args.coarsen,
                     stream=stream)
        x64 = torch.zeros(n, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            i64 = s64.solve(B[:, 0], x64, tol=TOL, max_iter=maxit, stream=stream)
            torch.cuda.synchronize()
        err = {"rel_error_vs_fp64_amgdd": float(torch.linalg.vector_norm(Xmix[:, 0] - x64)
                                                / torch.linalg.vector_norm(x64)),
               "fp64_iterations": i64["iterations"], "fp64_final_relres": i64["final_relres"]}
        s64.close()
    it = info["iterations"]
    if multi:
        desc = ("%d independent 3D 7-point Poisson systems (edges %s drawn from {32,48,64,80,96}, N=%d total), "
                "boxes of 16^3 (%d subdomains), padding %d, %d right-hand sides U[-1,1], "
                "FP32 AlgFAC / FP64 refinement" % (len(w["edges"]), ",".join(map(str, sorted(set(w["edges"])))),
                                                     n, w["nsub"], w["padding"], nrhs))
    elif small:
        desc = ("2D 5-point Poisson %d^2 (N=%d), %d subdomains of 16^2, padding %d, 2 AlgFAC V(1,1) per "
                "iteration, FP64, b~U[-1,1] seed 0, x0=0" % (w["shape"][0], n, w["nsub"], w["padding"]))
    elif "aniso" in I.WORKLOADS[name]:
        desc = ("2D rotated anisotropic diffusion theta=3pi/16, eps=1e-3, 9-point, 512^2 (N=%d), %d subdomains "
                "of 32^2, padding %d, FP64, b~U[-1,1] seed 0" % (n, w["nsub"], w["padding"]))
    else:
        desc = ("3D 7-point diffusion 256^3 (N=%d), kappa on 8^3 blocks of 32^3 i.i.d. {1,1e3}, %d subdomains "
                "of 16^3, padding %d, FP32 AlgFAC / FP64 refinement, b~U[-1,1] seed 0" % (n, w["nsub"],
                                                                                          w["padding"]))
    line = {
        "metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": False,
        "dtype": "f32 AlgFAC / f64 refinement" if prec else "f64",
        "data": "synthetic",
        "config": {"workload": desc, "n": n, "nnz": int(len(w["col"])), "nsub": int(w["nsub"]), "nrhs": nrhs,
                   "l2_policy": ("L2-resident problem; 256 MB written before every timed solve" if small
                                 else "inputs larger than L2"), "interp": args.interp,
                   "coarsen": args.coarsen},
        "iterations": it, "final_relres": info["final_relres"],
        "vcycle_fp64": {"ms_all_columns": round(v_ms, 3), "iterations": v_it},
        "amgdd_over_vcycle_time": round(ms / v_ms, 3),
        "ms_per_iteration": {"amgdd": round(ms / max(1, info["iterations"]), 4),
                             "vcycle": round(v_ms / max(1, sum(v_it)), 4)},
        "fac": fac_line,
        "composite_overhead": round(st.composite_overhead, 3), "levels": st.num_levels,
        "coarsest": int(st.n[st.num_levels - 1]), "setup_s": round(setup_s, 1),
        "device_gb": round(st.device_bytes / 1e9, 2),
        "host_peak_gb": round(__import__("resource").getrusage(__import__("resource").RUSAGE_SELF).ru_maxrss / 1e6, 1),
        "gpu_launches_per_step": int(info["kernel_launches"]),
        "clocks": clocks, "fp64_check": err, "autotune": tune,
    }
    if multi:
        line["edges"] = list(map(int, w["edges"]))
    if emit:
        print(json.dumps(line))
    return line


def run_adjoint(args, stream):
    """96^3 diffusion with kappa = exp(g) (g a Gaussian random field, length
    0.1, variance 1), loss 1/2 |x - x_t|^2: the differentiable solve's pieces
    timed separately (host setup of A(kappa); forward AMG-DD solve; adjoint
    AMG-DD solve with the same handle, A being symmetric; the gradient
    kernel), and the oracle's forward solve, adjoint solve and gradient on the
    host cores beside them."""
    import torch
    from paper_1906_10575_gb300 import Solver, capi
    from oracle import Oracle, kappa_gradient
    n = 96
    tol = 1e-10
    kappa = I.lognormal_kappa(n, seed=0)
    b = I.uniform_rhs(n ** 3, 1)
    xt = I.uniform_rhs(n ** 3, 2)
    rp, ci, v = I.diffusion3d(kappa)
    part, nsub = I.box_partition((n, n, n), (16, 16, 16))
    t0 = time.perf_counter()
    s = Solver(rp, ci, v, part, nsub, 2, n_fac=2, stream=stream, interp=args.interp, coarsen=args.coarsen)
    setup_s = time.perf_counter() - t0
    if not args.no_autotune:
        capi.amgdd_autotune(s.h, 1, reps=2, stream=stream)
    kd = torch.from_numpy(kappa.reshape(-1)).cuda()
    bd = torch.from_numpy(b).cuda()
    xtd = torch.from_numpy(xt).cuda()
    x = torch.zeros_like(bd)
    lam = torch.zeros_like(bd)
    g = torch.zeros_like(bd)
    fw, bw, gk = [], [], []
    with torch.cuda.stream(stream):
        for k in range(args.warmup + args.steps):
            x.zero_()
            lam.zero_()
            torch.cuda.synchronize()
            i1 = {}
            t_f = _ev_ms(stream, lambda: i1.update(s.solve(bd, x, tol=tol, max_iter=200, stream=stream)))
            gx = (x - xtd).contiguous()
            i2 = {}
            t_b = _ev_ms(stream, lambda: i2.update(s.solve(gx, lam, tol=tol, max_iter=200, stream=stream)))
            t_g = _ev_ms(stream, lambda: capi.amgdd_kappa_grad_3d((n, n, n), kd, x, lam, g, stream), 10)
            if k >= args.warmup:
                fw.append(t_f)
                bw.append(t_b)
                gk.append(t_g)
    s.close()
    hbm, peak_kind = _peaks()
    ms_g = statistics.median(gk)
    grad_bytes = 32.0 * n ** 3
    o = Oracle(rp, ci, v, part, nsub, 2, interp=args.interp, coarsen=args.coarsen)
    t0 = time.perf_counter()
    xo, ho = o.amgdd_solve(b, 2, tol=tol, maxit=200)
    lo, _ = o.amgdd_solve(xo - xt, 2, tol=tol, maxit=200)
    go = kappa_gradient(kappa, xo, lo)
    cpu_s = time.perf_counter() - t0
    gg = g.cpu().numpy()
    line = {
        "metric": "ms for the gradient of a loss through an AMG-DD diffusion solve (forward + adjoint solve + "
                  "gradient kernel), 1 GB300",
        "value": round(statistics.median(fw) + statistics.median(bw) + ms_g, 3), "unit": "ms", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "3D 7-point diffusion 96^3, kappa = exp(Gaussian random field, length 0.1, "
                               "variance 1) seed 0, 216 subdomains of 16^3, padding 2, loss 1/2|x - x_t|^2, "
                               "solves to 1e-10", "interp": args.interp, "coarsen": args.coarsen},
        "forward_ms": round(statistics.median(fw), 3), "forward_iterations": i1["iterations"],
        "adjoint_ms": round(statistics.median(bw), 3), "adjoint_iterations": i2["iterations"],
        "gradient_kernel_ms": round(ms_g, 4),
        "gradient_kernel_gbs": round(grad_bytes / (ms_g * 1e-3) / 1e9, 1),
        "gradient_kernel_note": "28 MB per launch, L2-resident: the HBM roofline does not apply",
        "host_setup_s": round(setup_s, 2),
        "gradient_vs_oracle_max_rel": float(np.abs(gg - go).max() / np.abs(go).max()),
        "cpu_baseline": {"value": round(cpu_s * 1e3, 1), "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "the oracle's forward and adjoint AMG-DD solves to 1e-10 and its gradient "
                                   "(all 216 composite grids, OpenMP over grids)"},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision measurement")
    ap.add_argument("--no-multi", action="store_true", help="skip the four-right-hand-side measurement")
    ap.add_argument("--no-small-case", action="store_true",
                    help="skip the 2D 64^2 measurement reported beside the headline")
    ap.add_argument("--hybrid-level", type=int, default=6,
                    help="switch level of the hybrid AMG-DD measurement (0 = skip)")
    ap.add_argument("--schedule", type=int, default=0, help="FAC kernel variant (0 = library default)")
    ap.add_argument("--n", type=int, default=128,
                    help="grid edge (default 128, the benchmark workload; smaller edges "
                         "are for profiling captures only)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "kappa3d_256", "batched_64", "aniso2d_512", "adjoint_96",
                             "poisson2d_64"],
                    help="poisson3d_128 (default, the headline) or one of the other "
                         "configurations, printed as a line of their own")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default FAC kernel instead of timing every candidate and "
                         "keeping the fastest")
    ap.add_argument("--interp", default="direct", choices=["direct", "exti"],
                    help="interpolation of the hierarchy: direct (default) or extended+i, "
                         "truncated to 4 entries per row")
    ap.add_argument("--padding", type=int, default=-1,
                    help="padding eta on every level instead of the workload's (-1, the default, keeps "
                         "it; not for adjoint_96)")
    ap.add_argument("--coarsen", default="rs", choices=["rs", "hmis"],
                    help="C/F splitting of the hierarchy: rs (default, Ruge-Stueben first pass) or hmis "
                         "(over the subdomains)")
    ap.add_argument("--candidate", type=int, default=-1,
                    help="use this FAC kernel candidate instead of autotuning (profiling captures)")
    ap.add_argument("--edge", type=int, default=0,
                    help="poisson2d_64: grid edge (default 64, the workload; other edges size the "
                         "latency-bound regime)")
    ap.add_argument("--nsys", type=int, default=64,
                    help="batched_64: number of systems (default 64, the workload; fewer are for "
                         "profiling captures only)")
    ap.add_argument("--no-fp64-check", action="store_true",
                    help="kappa3d_256: skip the FP64 AMG-DD solve used for the final error")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload != WORKLOAD:
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle arm runs the headline "
                                  "workload only; %s is measured on the GPU path" % args.workload}))
            return
        import torch
        torch.cuda.set_device(local)
        if args.workload == "adjoint_96":
            run_adjoint(args, torch.cuda.Stream())
        else:
            run_extra(args, args.workload, torch.cuda.Stream(), None, local)
        return
    w = I.workload(WORKLOAD, seed=0, shape=(args.n,) * 3)
    if args.padding >= 0:
        w["padding"] = args.padding

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, w)
        return

    import torch
    from paper_1906_10575_gb300 import Solver, capi

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    s = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=w["n_fac"],
               interp=args.interp, coarsen=args.coarsen,
               schedule=args.schedule, stream=stream)
    st = s.stats
    b = torch.from_numpy(w["b"]).cuda()
    x = torch.zeros_like(b)
    tune = None
    cand = None
    if args.candidate >= 0:
        cand = args.candidate
        capi.amgdd_set_fac_kernel(s.h, 1, cand)
    elif not args.no_autotune:
        cand, tms = capi.amgdd_autotune(s.h, 1, reps=2, stream=stream)
        tune = {"best_candidate": cand, "ms_per_candidate": [round(float(t), 3) for t in tms]}

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, k):
        times, infos = [], []
        for _ in range(k):
            x.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = fn(b, x, tol=TOL, max_iter=200, stream=stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        return times, infos

    with torch.cuda.stream(stream):
        # dominant kernel alone, first (direct launches, before any solve
        # graph): the all-grids FAC launch
        r_all = torch.zeros(int(s.offsets[-1]), dtype=torch.float64, device="cuda")
        capi.amgdd_residual(s.h, b, torch.zeros_like(b), r_all[:s.n], stream)
        capi.amgdd_restrict(s.h, r_all, stream)
        xf = torch.zeros_like(b)
        for _ in range(2):
            capi.amgdd_fac(s.h, r_all, xf, stream)
        nf = 5
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nf):
            capi.amgdd_fac(s.h, r_all, xf, stream)
        e1.record(stream)
        e1.synchronize()
        fac_ms = e0.elapsed_time(e1) / nf
        barrier()
        timed(s.solve, args.warmup)
        barrier()
        clk = ClockSampler(local)
        t_dd, i_dd = timed(s.solve, args.steps)
        clocks = clk.stop()
        x64 = x.clone()
        barrier()
        timed(s.vcycle_solve, args.warmup)
        t_v, i_v = timed(s.vcycle_solve, args.steps)
        barrier()
        # end to end through the C ABI with host buffers
        hb = torch.from_numpy(w["b"]).pin_memory()
        hx = torch.empty_like(hb).pin_memory()
        t_e2e = []
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            db = hb.to("cuda", non_blocking=True)
            dx = torch.zeros_like(db)
            s.solve(db, dx, tol=TOL, max_iter=200, stream=stream)
            hx.copy_(dx, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if k >= args.warmup:
                t_e2e.append(e0.elapsed_time(e1))

    # the paper's convergence setting: b = 0, random x0, relres relative to
    # the initial residual; convergence factor rho = relres_k^(1/k)
    paper_mode = {}
    with torch.cuda.stream(stream):
        zb = torch.zeros_like(b)
        x0 = torch.from_numpy(np.random.default_rng(7).uniform(-1.0, 1.0, s.n)).cuda()
        for name, fn in (("amgdd", s.solve), ("vcycle", s.vcycle_solve)):
            xz = x0.clone()
            inf = fn(zb, xz, tol=TOL, max_iter=400, stream=stream)
            k = inf["iterations"]
            paper_mode[name] = {"iterations": k, "final_relres": inf["final_relres"],
                                "rho": round(float(inf["final_relres"]) ** (1.0 / max(k, 1)), 4)}
    paper_mode["setting"] = "b = 0, x0 ~ U[-1,1] seed 7, relres = |A x_k| / |A x_0|"

    # mixed precision (FP32 AlgFAC inside FP64 refinement) on the same
    # workload: reported beside the FP64 headline
    mixed = None
    if not args.no_mixed:
        s.close()
        sm = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=w["n_fac"],
                    interp=args.interp, coarsen=args.coarsen,
                    precision=1, stream=stream)
        cand_m = None
        if not args.no_autotune:
            cand_m, _ = capi.amgdd_autotune(sm.h, 1, reps=2, stream=stream)
        with torch.cuda.stream(stream):
            def tm(k):
                ts, inf = [], None
                for _ in range(k):
                    x.zero_()
                    torch.cuda.synchronize()
                    a0 = torch.cuda.Event(enable_timing=True)
                    a1 = torch.cuda.Event(enable_timing=True)
                    a0.record(stream)
                    inf = sm.solve(b, x, tol=TOL, max_iter=200, stream=stream)
                    a1.record(stream)
                    a1.synchronize()
                    ts.append(a0.elapsed_time(a1))
                return ts, inf
            tm(args.warmup)
            t_m, i_m = tm(args.steps)
            capi.amgdd_fac(sm.h, r_all, xf, stream)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(nf):
                capi.amgdd_fac(sm.h, r_all, xf, stream)
            a1.record(stream)
            a1.synchronize()
            fac_m = a0.elapsed_time(a1) / nf
        ms_m = max_over_ranks([statistics.median(t_m)], dist)[0]
        # final error of the mixed solution against the FP64 solution (the
        # FP64 iterate equals the CPU oracle's bit for bit)
        err = float(torch.linalg.vector_norm(x - x64) / torch.linalg.vector_norm(x64))
        mixed = {"ms": round(ms_m, 3), "iterations": i_m["iterations"], "final_relres": i_m["final_relres"],
                 "rel_error_vs_fp64_solution": err,
                 "fac_ms_per_launch": round(fac_m, 3),
                 "fac_gbs_algorithmic_fp32": round(algorithmic_fac_bytes(sm.stats, w["n_fac"], sv=4.0)
                                                   / (fac_m * 1e-3) / 1e9, 1),
                 "fac_candidate": cand_m,
                 "dtype": "f32 AlgFAC / f64 refinement"}
        sm.close()

    # hybrid AMG-DD (Algorithm 3): V-cycle on the fine levels, one AMG-DD
    # cycle on level --hybrid-level
    hybrid = None
    if args.hybrid_level > 0:
        sh = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=w["n_fac"],
                    interp=args.interp, coarsen=args.coarsen,
                    hybrid_level=args.hybrid_level, stream=stream)
        with torch.cuda.stream(stream):
            timed(sh.hybrid_solve, args.warmup)
            t_h, i_h = timed(sh.hybrid_solve, args.steps)
        ms_h = max_over_ranks([statistics.median(t_h)], dist)[0]
        hybrid = {"level": args.hybrid_level, "ms": round(ms_h, 3), "iterations": i_h[-1]["iterations"],
                  "final_relres": i_h[-1]["final_relres"]}
        sh.close()

    # four right-hand sides of the same matrix at once (FP64): every operator
    # entry feeds four fma chains
    multi = None
    if not args.no_multi:
        sq = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=w["n_fac"],
                    interp=args.interp, coarsen=args.coarsen,
                    stream=stream)
        Bm = torch.from_numpy(np.ascontiguousarray(np.stack([I.uniform_rhs(sq.n, j) for j in range(4)], 1))).cuda()
        Xm = torch.zeros_like(Bm)
        cand_q = None
        if not args.no_autotune:
            cand_q, _ = capi.amgdd_autotune(sq.h, 4, reps=2, stream=stream)
        with torch.cuda.stream(stream):
            def tmm(k):
                ts, inf = [], None
                for _ in range(k):
                    Xm.zero_()
                    torch.cuda.synchronize()
                    a0 = torch.cuda.Event(enable_timing=True)
                    a1 = torch.cuda.Event(enable_timing=True)
                    a0.record(stream)
                    inf = sq.solve_multi(Bm, Xm, tol=TOL, max_iter=200, stream=stream)
                    a1.record(stream)
                    a1.synchronize()
                    ts.append(a0.elapsed_time(a1))
                return ts, inf
            tmm(args.warmup)
            t_mm, i_mm = tmm(args.steps)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            capi.amgdd_iterate_multi(sq.h, Bm, Xm, stream)
            a0.record(stream)
            for _ in range(nf):
                capi.amgdd_iterate_multi(sq.h, Bm, Xm, stream)
            a1.record(stream)
            a1.synchronize()
            it_mm = a0.elapsed_time(a1) / nf
        ms_mm = max_over_ranks([statistics.median(t_mm)], dist)[0]
        multi = {"nrhs": 4, "ms_all_columns": round(ms_mm, 3), "ms_per_column": round(ms_mm / 4, 3),
                 "iterations": i_mm["iterations"], "final_relres_max": i_mm["final_relres"],
                 "ms_per_iteration": round(it_mm, 3), "fac_candidate": cand_q,
                 "dtype": "f64"}
        sq.close()

    ms_dd = statistics.median(t_dd)
    ms_v = statistics.median(t_v)
    ms_e2e = statistics.median(t_e2e)
    ms_dd, ms_v, ms_e2e = max_over_ranks([ms_dd, ms_v, ms_e2e], dist)
    it_dd = i_dd[-1]["iterations"]
    it_v = i_v[-1]["iterations"]
    hbm, peak_kind = _peaks()
    fac_b = algorithmic_fac_bytes(st, w["n_fac"])
    fac_f = algorithmic_fac_flops(st, w["n_fac"])
    fac_gbs = fac_b / (fac_ms * 1e-3) / 1e9
    exec_tfs = 2.0 * st.fac_fma / (fac_ms * 1e-3) / 1e12
    frac_hbm = fac_gbs / hbm
    # the FAC launch is bound by HBM: its algorithmic bytes over the launch
    # time against the measured copy bandwidth; the FP64 pipe, counted with
    # the fmas the kernel executes (zero entries skipped), is reported beside
    kern = _fac_kernel(cand)
    roof = {"bound": "hbm", "achieved": round(fac_gbs, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(frac_hbm, 4), "traffic": _measured_traffic("poisson3d_128" if args.n == 128 and args.padding < 0 and
                                         args.coarsen == "rs" and args.interp == "direct" else None, kern, cand),
            "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind,
            "kernel": kern, "candidate": cand, "ms_per_launch": round(fac_ms, 3),
            "algorithmic_bytes": fac_b,
            "fp64": {"executed_fma": int(st.fac_fma), "achieved_tflops": round(exec_tfs, 4),
                     "frac_of_probe": round(exec_tfs / FP64_PROBE_TFLOPS, 4), "probe_tflops": FP64_PROBE_TFLOPS,
                     "probe_source": "FP64 fma throughput measured on this pool's GB300 (8 independent "
                                     "chains per thread)",
                     "frac_of_nominal": round(exec_tfs / FP64_PEAK_TFLOPS, 4), "nominal_tflops": FP64_PEAK_TFLOPS,
                     "algorithmic_flops": fac_f}}
    dd_bytes = algorithmic_solve_bytes(st, fac_b, it_dd)
    v_bytes = vcycle_bytes(st, it_v)
    # the fastest either solve could be on this GPU: its algorithmic bytes at
    # the measured copy bandwidth (AMG-DD: every iteration's residual,
    # restriction chain and FAC launch, plus the final residual)
    dd_lb = dd_bytes / (hbm * 1e9) * 1e3
    v_lb = v_bytes / (hbm * 1e9) * 1e3
    launches = int(i_dd[-1]["kernel_launches"])
    line = {
        "metric": METRIC, "value": round(ms_dd, 3), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_dd, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(_config(w), interp=args.interp, coarsen=args.coarsen),
        "iterations": it_dd, "final_relres": i_dd[-1]["final_relres"],
        "gbs": round(dd_bytes / (ms_dd * 1e-3) / 1e9, 1),
        "amgdd_lower_bound_ms": round(dd_lb, 3),
        "vcycle": {"ms": round(ms_v, 3), "iterations": it_v, "final_relres": i_v[-1]["final_relres"],
                   "gbs": round(v_bytes / (ms_v * 1e-3) / 1e9, 1), "lower_bound_ms": round(v_lb, 3),
                   "kernel_launches": int(i_v[-1]["kernel_launches"])},
        "amgdd_over_vcycle_time": round(ms_dd / ms_v, 3),
        "composite_overhead": round(st.composite_overhead, 3),
        "operator_complexity": round(st.operator_complexity, 3),
        "setup_s": round(st.setup_seconds, 2),
        "roofline": roof,
        "gpu_launches": launches * args.steps, "gpu_launches_per_step": launches,
        "e2e": {"value": round(ms_e2e, 3), "unit": "ms", "h2d_bytes_per_step": 8 * s.n,
                "d2h_bytes_per_step": 8 * s.n},
        "clocks": clocks,
        "autotune": tune,
        "paper_mode": paper_mode,
        "mixed_precision": mixed,
        "multi_rhs": multi,
        "hybrid": hybrid,
    }
    if not args.no_small_case:
        # the small latency-bound case (2D 64^2, where AMG-DD beats the
        # V-cycle on one GPU), measured in the same run beside the headline
        sa = argparse.Namespace(**vars(args))
        sa.padding, sa.candidate, sa.interp, sa.coarsen, sa.edge = -1, -1, "direct", "rs", 0
        sa.steps, sa.warmup, sa.no_autotune, sa.schedule = 5, 3, False, 0
        sl = run_extra(sa, "poisson2d_64", stream, dist, local, emit=False)
        line["small_case"] = {
            "workload": sl["config"]["workload"], "l2_policy": sl["config"]["l2_policy"],
            "amgdd_ms": sl["value"], "amgdd_iterations": sl["iterations"],
            "vcycle_ms": sl["vcycle_fp64"]["ms_all_columns"],
            "vcycle_iterations": sl["vcycle_fp64"]["iterations"][0],
            "amgdd_over_vcycle_time": sl["amgdd_over_vcycle_time"], "ms_per_iteration": sl["ms_per_iteration"],
            "fac_kernel": sl["fac"]["kernel"], "fac_candidate": sl["fac"]["candidate"],
            "fac_ms_per_launch": sl["fac"]["ms_per_launch"],
            "launches_per_solve": sl["gpu_launches_per_step"]}
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(w, it_dd, args.interp, args.coarsen)
    if rank == 0:
        print(json.dumps(line))
    if s.h:
        s.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
