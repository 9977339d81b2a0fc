"""Bounded samples of the 64^3 Poisson benchmark for timing the oracle.

Test infrastructure, like the rest of this package: only the benchmark's
CPU baseline and reference arm use it; nothing in the GPU library imports it.

The whole oracle factorization + GMRES of the 64^3 workload takes hours of
CPU time, so a benchmark step times a bounded sample of it: one subtree of
the 64^3 elimination tree (the front reached from the root by taking the
first child ``depth`` times, with all its descendants), factored exactly as
in the whole factorization (multifrontal.factor_subtree: same ordering,
update sets and random sketch), followed by one forward and backward sweep
of the multifrontal solve over those fronts.  The benchmark scales the
sample's time to the whole workload by the ratio of the two times measured
once, back to back on one machine, by ``calibrate`` (the full oracle run
and the same sample), stored in poisson64_calibration.json beside this file.

    python -m oracle.bench_sample            # writes the calibration record
"""
from __future__ import annotations

import json
import os
import platform
import time

import numpy as np

from . import krylov
from . import multifrontal as mf

DIMS = (64, 64, 64)
OPTS = dict(hss_tol=1e-4, d0=128, dd=64, hss_min_front=1024, hss_leaf=128, seed=0)
RHS_SEED = 1
SAMPLE_DEPTH = 6  # a reference-arm step: 15 fronts (a 16 x 16 x 8 box's subtree), one HSS front
BASELINE_DEPTH = 5  # the CPU baseline of a benchmark line: 31 fronts, three HSS fronts
CALIBRATION = os.path.join(os.path.dirname(os.path.abspath(__file__)), "poisson64_calibration.json")


def _problem():
    import problems
    A = problems.grid_poisson(DIMS).to_scipy()
    b = problems.rhs_uniform(A.shape[0], 1, RHS_SEED)[:, 0]
    return A, b


def sample_step(depth=SAMPLE_DEPTH, A=None, b=None):
    """One sample: the subtree's factorization and one solve sweep over it.
    Returns (seconds, number of fronts, number of HSS fronts)."""
    if A is None:
        A, b = _problem()
    t0 = time.perf_counter()
    fz, sub = mf.factor_subtree(A, DIMS, mf.Options(**OPTS), depth)
    mf.apply_inverse(fz, b)
    t = time.perf_counter() - t0
    n_hss = sum(1 for i in sub if isinstance(fz.data[i], mf.HSSFront))
    return t, len(sub), n_hss


def full_run(A=None, b=None):
    """The whole oracle step: factorization + GMRES(30) to 1e-10."""
    if A is None:
        A, b = _problem()
    t0 = time.perf_counter()
    fz = mf.factor(A, DIMS, mf.Options(**OPTS))
    tf = time.perf_counter() - t0
    x, its, rel = krylov.gmres(A, lambda v: mf.apply_inverse(fz, v), b, rtol=1e-10)
    return tf, time.perf_counter() - t0 - tf, its, rel, mf.hss_stats(fz)


def machine():
    try:
        blas = np.show_config(mode="dicts")["Build Dependencies"]["blas"]["name"]
    except Exception:  # pragma: no cover
        blas = "unknown"
    threads = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS") if os.environ.get(k)}
    return {"platform": platform.platform(), "machine": platform.machine(), "cpus": os.cpu_count(),
            "blas": blas, "thread_env": threads}


def calibrate(path=CALIBRATION, reps=3):
    A, b = _problem()
    tf, ts, its, rel, hs = full_run(A, b)
    rec = {"workload": "64^3 Poisson, HSS fronts >= 1024, eps 1e-4, d0 128, dd 64, GMRES(30) to 1e-10",
           "full_factor_s": tf, "full_solve_s": ts, "full_s": tf + ts, "iterations": int(its),
           "relres": float(rel), "hss_fronts": len(hs), "max_rank": max(r for _, _, r, _, _ in hs),
           "samples": {}, "machine": machine(), "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    for depth in (SAMPLE_DEPTH, BASELINE_DEPTH):
        runs = [sample_step(depth, A, b) for _ in range(reps)]
        t = float(np.median([r[0] for r in runs]))
        rec["samples"][str(depth)] = {"fronts": runs[0][1], "hss_fronts": runs[0][2], "seconds": t,
                                      "ratio": (tf + ts) / t}
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1)
    return rec


if __name__ == "__main__":
    print(json.dumps(calibrate(), indent=1))
