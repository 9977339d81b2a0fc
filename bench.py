#!/usr/bin/env python
"""Benchmark of the HSS-structured multifrontal solver on one GB300 (or N
independent replicas on N GPUs).

Metric: factor + solve time to a true relative residual of 1e-10 on the 3D
7-point Poisson problem on a 64^3 grid (n = 262144), HSS compression on
fronts with n_f >= 1024 at relative tolerance 1e-4, d0 = 128 and dd = 64
sample columns, one right-hand side uniform on [-1, 1] (seed 1), sampling
matrix from seed 0.  Two forms are timed on the same GPU: the mixed form
(FP32 fronts, sampling, ID and ULV preconditioning FP64 GMRES(30); the
headline ``value``) and the plain FP64 form (``fp64_ms_per_step``).

One step = hssmf_factor + hssmf_solve (GMRES to 1e-10) on device-resident
inputs; the factor storage (GBs) is far larger than L2, so no flush is
needed.  ``e2e`` repeats the step through the C ABI with host buffers
(values, right-hand side and solution copied inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own system on its own GPU
(replicas: the method has no data-parallel exchange at this size); the
reported time is the maximum over ranks.
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

WORKLOAD = dict(dims=(64, 64, 64), hss_min_front=1024, hss_tol=1e-4, d0=128, dd=64, seed=0,
                rhs_seed=1, nrhs=1)
WORKLOAD_NAME = ("3D 7-point Poisson 64^3 (n=262144), geometric ND (8^3 leaves), HSS on fronts >= 1024, "
                 "eps=1e-4, d0=128, dd=64, 1 RHS U[-1,1] seed 1, GMRES(30) to rel. residual 1e-10")
# --config grf100: the 100^3 anisotropic variable-coefficient diffusion (kappa =
# exp(Gaussian random field, correlation length 8 cells, sigma 1), anisotropy
# 1:1:10, harmonic-mean faces), HSS on fronts >= 2048; 1 and 64 RHS.  At eps
# 1e-2 GMRES(30) stalls on this coefficient contrast (~1.4e3), so the timed
# tolerance is 1e-4 (--hss-tol overrides it)
GRF100 = dict(dims=(100, 100, 100), hss_min_front=2048, hss_tol=1e-4, d0=128, dd=64, seed=0, rhs_seed=1, nrhs=1,
              grf=True, multi_rhs=64)
GRF100_NAME = ("3D anisotropic variable-coefficient diffusion 100^3 (n=1e6), kappa=exp(GRF corr 8, sigma 1), "
               "anisotropy 1:1:10, HSS on fronts >= 2048, eps={eps:g}, d0=128, dd=64, 1 RHS U[-1,1] seed 1, "
               "GMRES(30) to rel. residual 1e-10")
# --config batch256: 256 independent upwinded 2D convection-diffusion systems
# (sides uniform on 32..256, one velocity per system with components uniform on
# [-50, 50], nu 1), factored and solved together, 16 RHS each, eps 1e-6, HSS on
# fronts >= 256, refinement to 1e-10 in every system
BATCH256 = dict(nsys=256, hss_min_front=256, hss_tol=1e-6, d0=128, dd=64, seed=0, rhs_seed=1, nrhs=16,
                batch=True, multi_rhs=0)
BATCH256_NAME = ("batch of 256 upwinded 2D convection-diffusion systems (sides U{{32..256}}, velocity U[-50,50]^2 per "
                 "system, nu 1, seed 0; n={n}), one elimination forest with levels batched over all systems, HSS on "
                 "fronts >= 256, eps=1e-6, d0=128, dd=64, 16 RHS U[-1,1] seed 1, iterative refinement to rel. "
                 "residual 1e-10 in every system and column")
METRIC = "factor+solve time to rel. residual 1e-10 (mixed FP32/FP64 vs FP64), 1 GB300"
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 FMA units x clock (80.6)
# DRAM bytes of an ID launch per algorithmic byte (ncu: 10.73 MB for 4 nodes of
# 832 x 800 of rank 720 on the exchange kernel, 11.57 MB algorithmic)
ID_TRAFFIC_PER_ALG_BYTE = 0.93


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax = max(smax, float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _problem():
    import problems
    if WORKLOAD.get("batch"):
        sides, _, A = problems.batch_convdiff2d(WORKLOAD["nsys"], seed=WORKLOAD["seed"])
        WORKLOAD["grids"] = [(k, k, 1) for k in sides]
        WORKLOAD["sys_off"] = [0] + list(__import__("numpy").cumsum([k * k for k in sides]))
        b = problems.rhs_uniform(A.n, WORKLOAD["nrhs"], WORKLOAD["rhs_seed"])
        return A, b
    if WORKLOAD.get("grf"):
        A = problems.grid_anisotropic_grf(WORKLOAD["dims"][0], 8.0, 1.0, (1.0, 1.0, 10.0), seed=WORKLOAD["seed"])
    else:
        A = problems.grid_poisson(WORKLOAD["dims"])
    b = problems.rhs_uniform(A.n, WORKLOAD["nrhs"], WORKLOAD["rhs_seed"])
    return A, b


def problems_rhs(n, nrhs):
    import problems
    return problems.rhs_uniform(n, nrhs, WORKLOAD["rhs_seed"])


def _solver(A, precision):
    import paper_1502_07405_gb300 as P
    o = P.Options.defaults(hss_min_front=WORKLOAD["hss_min_front"], hss_tol=WORKLOAD["hss_tol"],
                           d0=WORKLOAD["d0"], dd=WORKLOAD["dd"], seed=WORKLOAD["seed"],
                           precision=precision)
    s = P.Solver(o)
    if WORKLOAD.get("batch"):
        s.analyze_grids(WORKLOAD["grids"], A.rowptr, A.colind)
    else:
        s.analyze_grid(WORKLOAD["dims"], A.rowptr, A.colind)
    return s


def _relres(A, x, b):
    """Largest relative residual over the right-hand sides (and, for a batch,
    over the systems)."""
    import numpy as np
    x = x.reshape(A.n, -1)
    b = b.reshape(A.n, -1)
    r = b - A.to_scipy() @ x
    if not WORKLOAD.get("batch"):
        return float((np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0)).max())
    off = WORKLOAD["sys_off"]
    return float(max((np.linalg.norm(r[off[g]:off[g + 1]], axis=0) /
                      np.linalg.norm(b[off[g]:off[g + 1]], axis=0)).max() for g in range(len(off) - 1)))


def _device_rhs(b):
    """b as a device tensor: a vector, or a column-major view for several RHS."""
    import numpy as np
    import torch
    if b.shape[1] == 1:
        return torch.tensor(np.ascontiguousarray(b[:, 0]), device="cuda")
    return torch.tensor(np.ascontiguousarray(b.T), device="cuda").t()


def _time_steps(s, vals, bt, steps, warmup, ws, split=None):
    """CUDA-event timing of factor + solve on the default stream (the
    solver's stream); returns per-step ms (max over ranks).  With ``split``
    a list, each step's own (factor ms, solve ms, iterations) is appended."""
    import torch
    for _ in range(warmup):
        s.factor(vals)
        s.solve(bt)
    torch.cuda.synchronize()
    out = []
    for _ in range(steps):
        _barrier(ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.factor(vals)
        x = s.solve(bt)
        e1.record()
        torch.cuda.synchronize()
        out.append(_barrier_max(e0.elapsed_time(e1), ws))
        if split is not None:
            st = s.get_stats()
            split.append((st["t_factor_ms"], st["t_solve_ms"], st["iterations"]))
    return out, x


def _time_fp64(s, vals, bt, steps, ws, A, b):
    """Factor + GMRES of the plain FP64 form (one untimed warm-up).  Where
    GMRES(30) stops at maxit short of 1e-10, the step time still counts the
    whole run and the second value records the residual reached."""
    import numpy as np
    import torch
    import paper_1502_07405_gb300 as P
    x = torch.empty_like(bt)
    info = None

    def step():
        nonlocal info
        s.factor(vals)
        try:
            s.solve(bt, x)
        except P.HssmfError as e:
            if e.status != P.ERR_NOCONV:
                raise
            info = {"iterations": s.opts.maxit}

    step()
    torch.cuda.synchronize()
    out = []
    for _ in range(steps):
        _barrier(ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        out.append(_barrier_max(e0.elapsed_time(e1), ws))
    if info is not None:
        info["relres"] = _relres(A, x.cpu().numpy(), b)
        info["note"] = "GMRES(30) reached maxit before 1e-10; fp64_ms_per_step times factor + maxit iterations"
    return out, info


def _profile_range(args, start):
    """With --profile-range, the timed steps are the only part of the run a
    profiler started with --profile-from-start off records (warm-up steps,
    which include the autotuner's trials, stay outside)."""
    if not args.profile_range:
        return
    import torch
    torch.cuda.synchronize()
    (torch.cuda.profiler.start if start else torch.cuda.profiler.stop)()


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    A, b = _problem()
    vals = torch.tensor(A.values, device="cuda")
    bt = _device_rhs(b)
    if args.form == "fp64":  # profiling of the plain FP64 form alone
        s64 = _solver(A, 0)
        for _ in range(args.warmup):
            s64.factor(vals)
            s64.solve(bt)
        _profile_range(args, True)
        t64, _ = _time_steps(s64, vals, bt, args.steps, 0, ws)
        _profile_range(args, False)
        if rank == 0:
            print(json.dumps({"form": "fp64", "ms_per_step": t64, "stats": s64.get_stats()}), flush=True)
        s64.close()
        return
    # mixed form (headline) -------------------------------------------------
    s = _solver(A, 1)
    clocks = Clocks(local)
    for _ in range(args.warmup):
        s.factor(vals)
        s.solve(bt)
    torch.cuda.synchronize()
    clocks.start()
    split = []
    _profile_range(args, True)
    times, x = _time_steps(s, vals, bt, args.steps, 0, ws, split)
    _profile_range(args, False)
    clk = clocks.stop()
    med = int(np.argsort(times)[len(times) // 2])  # the median step and its own factor / solve split
    st = s.get_stats()
    relres = _relres(A, x.cpu().numpy(), b)
    if args.form == "mixed":  # profiling of the mixed form alone
        if rank == 0:
            print(json.dumps({"form": "mixed", "ms_per_step": times, "relres": relres,
                              "stats": st}), flush=True)
        s.close()
        return
    # one profiled step for the phase split and the dominant kernel
    s.set_profiling(True)
    s.factor(vals)
    s.solve(bt)
    torch.cuda.synchronize()
    phases = s.get_phase_times()
    stp = s.get_stats()
    s.set_profiling(False)
    # the same factorization with 32 (64 for grf100) right-hand sides (solve time, GMRES per column)
    nmulti = WORKLOAD.get("multi_rhs", 32)
    rhs32 = None
    if nmulti:
        b32 = problems_rhs(A.n, nmulti)
        b32t = torch.tensor(np.ascontiguousarray(b32.T), device="cuda").t()  # column-major view
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x32 = s.solve(b32t)
        e1.record()
        torch.cuda.synchronize()
        t32 = e0.elapsed_time(e1)
        rhs32 = {"nrhs": nmulti, "solve_ms": round(t32, 2), "max_relres": _relres(A, x32.cpu().numpy(), b32),
                 "iterations_max": s.get_stats()["iterations"]}
    # e2e through the C ABI with host buffers --------------------------------
    vals_h = np.ascontiguousarray(A.values)
    b_h = np.asfortranarray(b)
    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        _barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.factor(vals_h)
        xh = s.solve(b_h)
        e2e_t.append(_barrier_max((time.perf_counter() - t0) * 1e3, ws))
    s.close()
    # plain FP64 form ---------------------------------------------------------
    s64 = _solver(A, 0)
    fp64_steps = args.fp64_steps if args.fp64_steps is not None else max(1, min(args.steps, 3))
    t64, fp64_conv = _time_fp64(s64, vals, bt, fp64_steps, ws, A, b)
    st64 = s64.get_stats()
    s64.close()
    ms = float(times[med])
    # roofline of the dominant kernel: the interpolative decompositions
    # (algorithmic bytes m d + k (m - k) elements and flops per ID, over the
    # wall time of the ID phases: CUDA events on the solver's stream around
    # each batch's ID launches, which run concurrently on side streams)
    hbm, src = _peaks()
    t_id = phases["id_kernels"]
    achieved_bw = stp["id_bytes"] / (t_id * 1e-3) / 1e9 if t_id > 0 else 0.0
    achieved = stp["id_flops"] / (t_id * 1e-3) / 1e12 if t_id > 0 else 0.0
    peak = FP32_SIMT_TFLOPS
    roof = {"kernel": ("k_cpqr_id_rx / k_cpqr_id_push / k_cpqr_id_rr / k_cpqr_id_smem (interpolative "
                       "decompositions, Section 2.2)"),
            "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 1), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 5),
            "traffic": round(ID_TRAFFIC_PER_ALG_BYTE * stp["id_bytes"] / max(stp["id_launches"], 1)),
            "traffic_note": ("DRAM bytes per launch scaled from ncu captures of the exchange and shared-memory "
                             "ID kernels on 832 x 800 nodes (dram read + write = 0.93 x the algorithmic bytes: the "
                             "input is read once and nothing is re-read; profiles/ncu_id_*_832x800.md)"),
            "peak_source": ("FP32 FMA peak from unit counts and the maximum SM clock: 152 SMs x 128 lanes x "
                            "2 flop x 2.07 GHz"),
            "launches": stp["id_launches"],
            "alg_flops_per_launch": stp["id_flops"] / max(stp["id_launches"], 1),
            "alg_bytes_per_launch": stp["id_bytes"] / max(stp["id_launches"], 1),
            "avg_launch_ms": t_id / max(stp["id_launches"], 1),
            "timing_note": ("achieved = flops of every ID / wall time of the ID phases; the launches of a batch "
                            "overlap on side streams, so avg_launch_ms is wall time per launch"),
            "hbm_achieved_gbs": round(achieved_bw, 2), "hbm_frac": round(achieved_bw / hbm, 5),
            "hbm_peak": hbm, "hbm_peak_source": src,
            "share_of_factor": round(t_id / max(stp["t_factor_ms"], 1e-9), 3),
            "note": ("latency-bound: one pivot per step, each step a reduction over the node's columns and an "
                     "exchange across the CTAs that hold the node")}
    # the solve reads the factorization once per application (the paper's
    # solution bandwidth): factor bytes x applications / solve time
    apps = st["iterations"] + 1
    t_sol = phases["solve"]
    sol_bw = stp["factor_bytes"] * apps / (t_sol * 1e-3) / 1e9 if t_sol > 0 else 0.0
    solve_roof = {"bound": "hbm", "achieved": round(sol_bw, 1), "peak": hbm, "unit": "GB/s",
                  "frac": round(sol_bw / hbm, 4), "applications": apps, "factor_bytes": stp["factor_bytes"]}
    dense_mf = _dense_mf(stp)
    line = {
        "metric": METRIC, "value": round(ms, 2), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 factor + f64 GMRES", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME.format(n=A.n) if WORKLOAD.get("batch") else WORKLOAD_NAME,
                   "form": ("mixed (FP32 factorization, FP64 refinement)" if WORKLOAD.get("batch")
                            else "mixed (FP32 HSS factorization preconditioning FP64 GMRES)"),
                   "l2": "no flush: factor storage and inputs are GBs, far larger than L2",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "fp64_ms_per_step": round(float(np.median(t64)), 2),
        "mixed_over_fp64_speedup": round(float(np.median(t64)) / ms, 3),
        "iterations": st["iterations"], "relres": relres,
        "fp64_iterations": st64["iterations"] if fp64_conv is None else fp64_conv["iterations"],
        "factor_ms": round(split[med][0], 2), "solve_ms": round(split[med][1], 2),
        "split_note": "factor_ms and solve_ms are the median step's own (host-synchronous C ABI timers)",
        "max_hss_rank": st["max_rank"], "max_d": st["max_d"], "hss_fronts": st["n_hss_fronts"],
        "factor_flops": st["factor_flops"], "phases_ms": {k: round(v, 2) for k, v in phases.items()},
        "gpu_launches": st["gpu_launches"],
        "e2e": {"value": round(float(np.median(e2e_t)), 2), "unit": "ms",
                "h2d_bytes_per_step": int(A.values.nbytes + b.nbytes),
                "d2h_bytes_per_step": int(b.nbytes)},
        "roofline": roof,
        "solve_roofline": solve_roof,
        "multi_rhs": rhs32,
        "clocks": clk,
        "dense_mf": dense_mf,
    }
    if fp64_conv is not None:
        line["fp64_not_converged"] = fp64_conv
    if ws > 1:
        line["systems_per_s"] = round(ws / (ms * 1e-3), 4)
    if rank == 0:
        if ws == 1 and args.config == "poisson64" and not args.no_secondary:
            line["secondary"] = {name: _secondary(name) for name in ("batch256", "grf100")}
        if ws == 1 and not args.no_cpu and not WORKLOAD.get("grf") and not WORKLOAD.get("batch"):
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _dense_mf(st_any):
    """The plain dense multifrontal method on the same elimination tree, from
    the symbolic structure alone: factor flops 2/3 ns^3 + 2 ns^2 nu + 2 ns nu^2
    and stored factor entries ns^2 + 2 ns nu per front, beside the library's
    own HSS-structured counts."""
    import numpy as np
    import paper_1502_07405_gb300 as P
    A, _ = _problem()
    s = _solver(A, 1)
    nf = s.get_stats()["n_fronts"]
    _, sb, se, _, nu = s.get_symbolic(nf)
    s.close()
    ns = (se - sb).astype(np.float64)
    nu = nu.astype(np.float64)
    flops = float(np.sum(2.0 / 3.0 * ns ** 3 + 2.0 * ns ** 2 * nu + 2.0 * ns * nu ** 2))
    ents = float(np.sum(ns ** 2 + 2.0 * ns * nu))
    return {"factor_flops": flops, "factor_bytes_fp32": 4.0 * ents, "factor_bytes_fp64": 8.0 * ents,
            "hss_factor_flops": st_any["factor_flops"], "hss_factor_bytes_fp32": st_any["factor_bytes"]}


SECONDARY = {"batch256": (BATCH256, BATCH256_NAME), "grf100": (GRF100, GRF100_NAME)}


def _secondary(name):
    """One more workload on the same GPU, mixed form only: analyze, one
    untimed factor + solve, then two timed steps (CUDA events); errors are
    reported, not raised, so that the headline line still prints."""
    import numpy as np
    import torch
    global WORKLOAD_NAME
    saved, saved_name = dict(WORKLOAD), WORKLOAD_NAME
    try:
        WORKLOAD.clear()
        WORKLOAD.update(SECONDARY[name][0])
        A, b = _problem()
        WORKLOAD_NAME = SECONDARY[name][1].format(n=A.n, eps=WORKLOAD["hss_tol"])
        vals = torch.tensor(A.values, device="cuda")
        bt = _device_rhs(b)
        s = _solver(A, 1)
        split = []
        times, x = _time_steps(s, vals, bt, 2, 1, 1, split)
        st = s.get_stats()
        rel = _relres(A, x.cpu().numpy(), b)
        s.close()
        med = int(np.argsort(times)[len(times) // 2])
        return {"workload": WORKLOAD_NAME, "ms_per_step": round(float(times[med]), 2), "steps": 2, "warmup": 1,
                "factor_ms": round(split[med][0], 2), "solve_ms": round(split[med][1], 2),
                "iterations": int(split[med][2]), "relres": rel, "hss_fronts": st["n_hss_fronts"],
                "max_hss_rank": st["max_rank"], "max_d": st["max_d"], "form": "mixed (FP32 factorization, FP64 "
                "outer iteration)"}
    except Exception as e:  # pragma: no cover - reported in the line
        return {"error": f"{type(e).__name__}: {e}"}
    finally:
        WORKLOAD.clear()
        WORKLOAD.update(saved)
        WORKLOAD_NAME = saved_name
        torch.cuda.empty_cache()


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _blas_threads():
    """Threads the oracle's BLAS uses in this process (the environment's
    limit, else every core)."""
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        v = os.environ.get(k)
        if v and v.isdigit():
            return int(v)
    return _cores()


def _calibration():
    path = os.path.join(ROOT, "oracle", "poisson64_calibration.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def _sample_subprocess(threads, depth=None):
    """One oracle sample step in a child process whose BLAS uses ``threads``
    threads (the limit must be set before numpy loads); returns seconds."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads))
    code = ("import json, sys; sys.path.insert(0, %r); from oracle import bench_sample as S; "
            "print(json.dumps(S.sample_step(%s)))" % (ROOT, "" if depth is None else int(depth)))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])[0]


def _scale(cal, depth):
    """Whole oracle run / one sample of this depth, both timed on the
    calibration machine (None without a record)."""
    try:
        return float(cal["samples"][str(depth)]["ratio"])
    except (TypeError, KeyError, ValueError):
        return None


def _sample_text(cal, depth, t_ms, extra=""):
    scale = _scale(cal, depth)
    if scale is None:
        return (f"oracle (numpy FP64) on the depth-{depth} subtree of the 64^3 elimination tree ({t_ms:.0f} ms); "
                f"no calibration record, so value is the unscaled sample time")
    smp = cal["samples"][str(depth)]
    return (f"oracle (numpy FP64) factorization of the depth-{depth} subtree of the 64^3 elimination tree "
            f"({smp['fronts']} fronts, {smp['hss_fronts']} HSS) plus one solve sweep over it: {t_ms:.0f} ms{extra}; "
            f"scaled by {scale:.1f} = whole oracle run ({cal['full_s']:.0f} s: factor + {cal['iterations']} GMRES "
            f"iterations, rel. residual {cal['relres']:.1e}) / the same sample ({smp['seconds']:.2f} s), both "
            f"measured back to back on {cal['machine']['machine']} x{cal['machine']['cpus']} "
            f"(oracle/poisson64_calibration.json, written by oracle/bench_sample.py)")


def cpu_baseline():
    """The oracle on a bounded sample of the same workload (all cores, then
    one thread), scaled to the whole factor + GMRES by the calibration."""
    from oracle import bench_sample as S
    cal = _calibration()
    depth = S.BASELINE_DEPTH
    n = _cores()
    t_all = sorted(_sample_subprocess(n, depth) for _ in range(2))[0]
    t_one = _sample_subprocess(1, depth)
    scale = _scale(cal, depth)
    k = scale if scale is not None else 1.0
    return {"value": round(t_all * 1e3 * k, 1), "unit": "ms", "cores": n, "kind": "oracle",
            "sample": _sample_text(cal, depth, t_all * 1e3, f" on {n} BLAS threads ({t_one * 1e3:.0f} ms on 1)"),
            "sample_ms": round(t_all * 1e3, 1), "sample_ms_1thread": round(t_one * 1e3, 1),
            "value_1thread": round(t_one * 1e3 * k, 1), "scale": None if scale is None else round(scale, 2)}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, each step one bounded
    sample of the 64^3 workload (no GPU library is loaded)."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    import numpy as np
    from oracle import bench_sample as S
    cal = _calibration()
    A, b = S._problem()
    for _ in range(args.warmup):  # untimed: a leaf front of the same tree
        S.sample_step(9, A, b)
    times = [S.sample_step(S.SAMPLE_DEPTH, A, b)[0] * 1e3 for _ in range(args.steps)]
    t_one = _sample_subprocess(1, S.SAMPLE_DEPTH)
    ms = float(np.median(times)) if times else float("nan")
    scale = _scale(cal, S.SAMPLE_DEPTH)
    k = scale if scale is not None else 1.0
    value = ms * k
    threads = _blas_threads()
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME,
                       "form": "CPU oracle (numpy FP64), one bounded sample of the workload per step",
                       "l2": "no flush: CPU run", "parallelism": "1 process, BLAS threads"},
            "value_note": ("value = projected time of the whole factor + solve (the metric); ms_per_step = the "
                           "measured time of one sample step"),
            "cpu_baseline": {"value": round(value, 1), "unit": "ms", "cores": threads, "kind": "oracle",
                             "sample": _sample_text(cal, S.SAMPLE_DEPTH, ms, f" on {threads} BLAS threads (median "
                                                    f"of {len(times)}; {t_one * 1e3:.0f} ms on 1)"),
                             "sample_ms": round(ms, 1), "sample_ms_1thread": round(t_one * 1e3, 1),
                             "value_1thread": round(t_one * 1e3 * k, 1),
                             "scale": None if scale is None else round(scale, 2)},
            "e2e": {"value": round(value, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--profile-range", action="store_true",
                    help="mark the timed steps for a profiler run with --profile-from-start off")
    ap.add_argument("--nsys", type=int, default=None,
                    help="--config batch256 with this many systems instead (profiling captures only)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batch256 and grf100 measurements that follow the 64^3 benchmark")
    ap.add_argument("--form", choices=["both", "mixed", "fp64"], default="both",
                    help="forms to time (profiling runs use one)")
    ap.add_argument("--small", action="store_true",
                    help="32^3 grid instead of 64^3 (profiling captures only; not a bench line)")
    ap.add_argument("--config", choices=["poisson64", "grf100", "batch256"], default="poisson64",
                    help="workload: the 64^3 Poisson benchmark (default), the 100^3 anisotropic one, or the "
                         "batch of 256 convection-diffusion systems")
    ap.add_argument("--hss-tol", type=float, default=None, help="override the workload's HSS tolerance")
    ap.add_argument("--fp64-steps", type=int, default=None, help="timed steps of the FP64 form (default min(steps, 3))")
    args = ap.parse_args()
    global WORKLOAD_NAME
    if args.config == "batch256":
        WORKLOAD.clear()
        WORKLOAD.update(BATCH256)
        WORKLOAD_NAME = BATCH256_NAME
        if args.nsys is not None:
            WORKLOAD["nsys"] = args.nsys
            WORKLOAD_NAME = BATCH256_NAME.replace("batch of 256", f"batch of {args.nsys}")
    elif args.config == "grf100":
        WORKLOAD.clear()
        WORKLOAD.update(GRF100)
        if args.hss_tol is not None:
            WORKLOAD["hss_tol"] = args.hss_tol
        WORKLOAD_NAME = GRF100_NAME.format(eps=WORKLOAD["hss_tol"])
    elif args.hss_tol is not None:
        ap.error("--hss-tol applies to --config grf100 only")
    if args.small:
        WORKLOAD["dims"] = (32, 32, 32)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
