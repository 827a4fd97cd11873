"""World-size-2 checks of bench.py's multi-process path on CPU (gloo): ranks time the
same replica workload, the job is charged the slowest rank, only rank 0 reports, and
the reference arm runs on rank 0 alone."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    r, local, w = bench.dist_setup("gloo")
    assert (r, local, w) == (rank, rank, ws)
    bench.barrier(w)
    out[rank] = bench.allmax(10.0 + rank, w)     # per-rank step times 10 ms and 11 ms
    # the reference arm returns immediately on ranks other than 0
    class A:
        gpus, steps, warmup = ws, 1, 3
    if rank != 0:
        assert bench.run_reference(A()) is None
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_rank0_only():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    assert out[0] == 11.0 and out[1] == 11.0


def test_bench_gpus_2_starts_two_ranks_itself():
    """python bench.py --gpus 2 without a torchrun environment launches 2 ranks (here on
    CPU with gloo, no GPU work) and rank 0 reports n_gpus = 2."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK",
                                                               "MASTER_ADDR", "MASTER_PORT")}
    env["CUDA_VISIBLE_DEVICES"] = ""
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--launch-check"],
                         capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [json.loads(x) for x in res.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, res.stdout
    assert lines[0]["n_gpus"] == 2 and lines[0]["ms_per_step"] == 2.0 and lines[0]["backend"] == "gloo"
