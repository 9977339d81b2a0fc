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
