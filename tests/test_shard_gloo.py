"""Column-block partition of the full reduced Hessian over ranks, and the gather.

Two and three gloo ranks on the CPU each compute their own block of columns of
H with the oracle (the same arithmetic per column as a single rank), gather the
blocks on rank 0, and rank 0 checks that the gathered H equals the single-rank
H bit for bit.  An uneven split (n_p = 107 over 2 and 3 ranks) exercises the
padding of the collective.
"""
import json
import os
import socket
import sys

import numpy as np
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
    from oracle import OracleGrid
    from paper_2201_00241_gb300 import gridgen as gg
    from paper_2201_00241_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        g = gg.make_case("case118")
        o = OracleGrid(g)
        st = o.plant()
        c0, n = shard.column_range(o.n_p, world, rank)
        E = np.zeros((o.n_p, n))
        E[c0 + np.arange(n), np.arange(n)] = 1.0
        block = o.hessvec(st.x, st.p, st.pd, st.qd, E)
        H = shard.gather_columns(block, o.n_p, world, rank, dst=0)
        if rank == 0:
            full = o.hessvec(st.x, st.p, st.pd, st.qd, np.eye(o.n_p))
            res = {"equal": bool(np.array_equal(H, full)), "shape": list(H.shape)}
        else:
            res = {"none": H is None}
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partition_and_gather_equal_single_rank_hessian(tmp_path, world):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "rank0.json"))
    assert r0["equal"] and r0["shape"] == [107, 107]
    for k in range(1, world):
        assert json.load(open(tmp_path / f"rank{k}.json"))["none"]


def test_column_ranges_cover_every_column_once():
    sys.path.insert(0, ROOT)
    from paper_2201_00241_gb300 import shard
    for n_p in (1, 7, 107, 2889):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                c0, n = shard.column_range(n_p, world, r)
                seen.extend(range(c0, c0 + n))
                assert n in (n_p // world, -(-n_p // world))
            assert seen == list(range(n_p))
    with pytest.raises(ValueError):
        shard.column_range(10, 2, 2)
