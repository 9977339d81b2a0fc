"""bench.py's multi-process plumbing on CPU: two gloo ranks, the barrier and
the max-over-ranks reduction that every timed value goes through, and the
reference arm's rank-0-only rule."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ws, r, local = bench._dist()
    bench._barrier(ws)
    m = bench._barrier_max(10.0 * (rank + 1), ws)  # per-rank times 10 and 20 ms
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"ws": ws, "rank": r, "local": local, "max": m}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert [g["rank"] for g in got] == [0, 1] and all(g["ws"] == 2 for g in got)
    assert all(g["max"] == 20.0 for g in got)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup = 1, 0

    bench.run_reference(Args())  # returns at once: no oracle run, no output
    assert capsys.readouterr().out == ""


def test_relres_takes_the_worst_system_and_column(monkeypatch):
    """bench._relres: the largest relative residual over the right-hand sides,
    and over the systems of a batch (each system's own norms)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import problems
    mats = [problems.grid_poisson((4, 4, 1)), problems.grid_poisson((3, 5, 1), scale=10.0)]
    A = problems.block_diag(mats)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((A.n, 2))
    b = A.to_scipy() @ x
    xe = x.copy()
    xe[16:, 1] += 1e-3  # error in the second system, second column only
    monkeypatch.setattr(bench, "WORKLOAD", dict(batch=True, sys_off=[0, 16, 31]))
    r2 = np.linalg.norm(b[16:, 1] - mats[1].to_scipy() @ xe[16:, 1]) / np.linalg.norm(b[16:, 1])
    assert bench._relres(A, xe, b) == pytest.approx(r2, rel=1e-12)
    monkeypatch.setattr(bench, "WORKLOAD", dict())
    rg = np.linalg.norm(b[:, 1] - A.to_scipy() @ xe[:, 1]) / np.linalg.norm(b[:, 1])
    assert bench._relres(A, xe, b) == pytest.approx(rg, rel=1e-12)
    assert rg < r2  # the whole-vector residual hides the per-system one


def test_reference_arm_scales_the_sample_and_loads_no_gpu_library(tmp_path):
    """The reference arm times the oracle alone: in a fresh process, with a
    small sample (a leaf front of the 64^3 tree) and a stand-in calibration
    record, its value is the sample time times the recorded ratio, and
    neither the package nor libhssmf.so is loaded."""
    import subprocess
    code = f"""
import json, sys
sys.path.insert(0, {ROOT!r})
import bench
from oracle import bench_sample as S
S.SAMPLE_DEPTH = 9
bench._sample_subprocess = lambda threads, depth=None: 0.25
bench._calibration = lambda: {{"samples": {{"9": {{"ratio": 100.0, "fronts": 1, "hss_fronts": 0, "seconds": 9.0}}}},
    "full_s": 900.0, "iterations": 9, "relres": 1e-11, "machine": {{"machine": "x", "cpus": 8}}}}
class Args:
    steps, warmup = 2, 1
bench.run_reference(Args())
maps = open("/proc/self/maps").read()
print(json.dumps({{"lib": "libhssmf" in maps, "pkg": "paper_1502_07405_gb300" in sys.modules}}))
"""
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, check=True, cwd=str(tmp_path))
    lines = [json.loads(x) for x in out.stdout.strip().splitlines()]
    ref, loaded = lines[0], lines[1]
    assert ref["impl"] == "reference" and ref["steps"] == 2
    assert ref["value"] == pytest.approx(ref["ms_per_step"] * 100.0, rel=1e-3)
    assert ref["cpu_baseline"]["sample_ms_1thread"] == 250.0
    assert loaded == {"lib": False, "pkg": False}
