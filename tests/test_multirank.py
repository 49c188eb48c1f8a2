"""The benchmark's multi-rank host logic with world size 2 on the gloo
backend (CPU): barrier, max over ranks, whole-job value, and that only rank
0 of the reference arm does any work."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    secs = 1.0 + rank            # rank 1 is the slower one
    mx = bench.max_over_ranks(secs, world)
    val = bench.job_value(1000, secs, world)
    bench.barrier(world)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": mx, "value": val}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["max"] == 2.0
        assert got["value"] == pytest.approx(2 * 1000 / 2.0)


def _ref_worker(rank, world, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import contextlib
    import io
    import types
    import bench
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(types.SimpleNamespace(steps=1, warmup=0))
    with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as f:
        f.write(buf.getvalue())


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    mp.start_processes(_ref_worker, args=(2, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    assert (tmp_path / "ref1.txt").read_text() == ""
    line = json.loads((tmp_path / "ref0.txt").read_text().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
