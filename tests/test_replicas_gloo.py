"""The multi-GPU path of bench.py runs replicas (every rank computes the whole
step; nothing on the path exchanges data).  Its host logic is checked here with
two gloo ranks on the CPU: the job time is the slowest rank's, the throughput is
world x the per-rank units, every rank sees the same numbers, and only rank 0
of the reference arm prints."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = [9.5, 11.25][rank]                 # the ranks' own step times
        t = bench.max_over_ranks(local_ms, world, "cpu")
        value = bench.replica_throughput(2889, world, t * 1e-3)
        dist.barrier()
        # the reference arm: only rank 0 runs and prints
        class Args:
            case, steps, warmup = "tiny", 1, 0
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(Args, rank, world)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"t": t, "value": value, "printed": buf.getvalue()}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_agree_on_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    assert r[0]["t"] == r[1]["t"] == 11.25
    assert r[0]["value"] == r[1]["value"] == pytest.approx(2 * 2889 / 11.25e-3)
    assert r[1]["printed"] == ""


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_throughput(100, 1, 0.5) == 200.0
