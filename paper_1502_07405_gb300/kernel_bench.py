"""Single-kernel timing through the C ABI, for profiling one kernel family
at a time on synthetic inputs (ncu captures, roofline checks).

    python -m paper_1502_07405_gb300.kernel_bench gemm --m 4096 --n 128 --k 8192 --b-exact
    python -m paper_1502_07405_gb300.kernel_bench id --d 832 --m 800 --jobs 8 --mode -1

``gemm`` runs hssmf_gemm_f32 (the tensor-core GEMMs of the FP32 form: the
TMA pipeline over pre-split operands, or with --in-loop the factorization's
kernel; with --b-exact the shape of the sampling products S = U R of
Section 4.3); ``id`` runs hssmf_batched_id on matrices with a geometric
singular-value decay (Section 2.2 interpolative decompositions).  Prints one
JSON line with the CUDA-event time per call (the calls synchronize; the
allocation of the entry points' scratch is inside the timed region for
``id``).
"""
from __future__ import annotations

import argparse
import ctypes as C
import json

import numpy as np


def _gemm(args):
    import torch
    from . import lib
    f = lib.hssmf_gemm_f32
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_void_p, C.c_longlong,
                  C.c_void_p, C.c_longlong, C.c_float, C.c_void_p, C.c_longlong, C.c_int, C.c_void_p]
    m, n, k = args.m, args.n, args.k
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(m * k, device="cuda", generator=g)  # column-major m x k (k x m with --ta)
    B = torch.randn(n, k, device="cuda", generator=g)  # column-major k x n
    if args.b_exact:
        B = B.to(torch.bfloat16).to(torch.float32)
    Cm = torch.zeros(n, m, device="cuda")
    times = []
    for it in range(args.warmup + args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = f(args.ta, 0, m, n, k, 1.0, A.data_ptr(), k if args.ta else m, B.data_ptr(), k, 1.0, Cm.data_ptr(), m,
               int(args.b_exact) | (2 if args.in_loop else 0), None)
        e1.record()
        torch.cuda.synchronize()
        if st != 0:
            raise RuntimeError(f"hssmf_gemm_f32 returned {st}")
        if it >= args.warmup:
            times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    flops = 2.0 * m * n * k
    return {"kernel": "k_gemm_tc" if args.in_loop else "k_gemm_tma", "m": m, "n": n, "k": k, "ta": args.ta,
            "b_exact": bool(args.b_exact), "ms": ms,
            "tflops": flops / ms * 1e-9, "a_bytes": 4 * m * k, "a_gbs": 4.0 * m * k / ms * 1e-6}


def _id(args):
    import torch
    from . import lib
    f = lib.hssmf_batched_id
    f.restype = C.c_int
    d, m, jobs = args.d, args.m, args.jobs
    rng = np.random.default_rng(0)
    r = min(d, m)
    Ys = []
    for _ in range(jobs):
        Q1 = rng.standard_normal((d, r)).astype(np.float32)
        Q2 = rng.standard_normal((r, m)).astype(np.float32)
        s = (10.0 ** (-np.arange(r) / (r / args.decades))).astype(np.float32)
        Ys.append(((Q1 * s) @ Q2).T.reshape(-1))
    dt = torch.float64 if args.prec == 0 else torch.float32
    Yd = torch.tensor(np.concatenate(Ys), dtype=dt, device="cuda")
    mm = np.full(jobs, m, np.int32)
    dd = np.full(jobs, d, np.int32)
    y_off = (np.arange(jobs, dtype=np.int64) * d * m)
    p_off = (np.arange(jobs, dtype=np.int64) * m)
    x_off = (np.arange(jobs, dtype=np.int64) * (m * m // 4 + 1))
    piv = torch.zeros(jobs * m, dtype=torch.int32, device="cuda")
    X = torch.zeros(jobs * (m * m // 4 + 1), dtype=dt, device="cuda")
    ranks = np.zeros(jobs, np.int32)
    lp = lambda a: a.ctypes.data_as(C.c_void_p)
    times = []
    for it in range(args.warmup + args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = f(args.prec, jobs, C.c_void_p(Yd.data_ptr()), lp(y_off), lp(mm), lp(dd), C.c_double(args.eps),
               lp(ranks), C.c_void_p(piv.data_ptr()), lp(p_off), C.c_void_p(X.data_ptr()), lp(x_off),
               int(args.mode), None)
        e1.record()
        torch.cuda.synchronize()
        if st != 0:
            raise RuntimeError(f"hssmf_batched_id returned {st}")
        if it >= args.warmup:
            times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    k = int(ranks.max())
    esz = 8 if args.prec == 0 else 4
    alg = jobs * esz * (m * d + k * (m - k))
    return {"kernel": "batched_id", "d": d, "m": m, "jobs": jobs, "mode": args.mode, "prec": args.prec,
            "rank": k, "ms": ms, "us_per_step": 1e3 * ms / max(k, 1), "alg_bytes": alg}


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="what", required=True)
    g = sub.add_parser("gemm")
    g.add_argument("--m", type=int, default=4096)
    g.add_argument("--n", type=int, default=128)
    g.add_argument("--k", type=int, default=8192)
    g.add_argument("--b-exact", action="store_true")
    g.add_argument("--ta", type=int, default=0, help="1: op(A) = A^T (A stored k x m)")
    g.add_argument("--in-loop", action="store_true",
                   help="the factorization's kernel (FP32 tiles staged and split in its loop)")
    g.add_argument("--reps", type=int, default=5)
    g.add_argument("--warmup", type=int, default=2)
    i = sub.add_parser("id")
    i.add_argument("--d", type=int, default=832)
    i.add_argument("--m", type=int, default=800)
    i.add_argument("--jobs", type=int, default=8)
    i.add_argument("--mode", type=int, default=-1, help="use_cluster of hssmf_batched_id")
    i.add_argument("--prec", type=int, default=1)
    i.add_argument("--eps", type=float, default=1e-4)
    i.add_argument("--decades", type=float, default=4.5, help="singular values fall this many decades")
    i.add_argument("--reps", type=int, default=3)
    i.add_argument("--warmup", type=int, default=1)
    args = ap.parse_args()
    out = _gemm(args) if args.what == "gemm" else _id(args)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
