"""The multi-process path of bench.py on CPU: world size 2 over gloo (no GPU).
The slowest rank sets the time (max over ranks), the barrier joins both ranks,
and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import argparse
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(ws),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    got_ws, got_rank, _ = bench.dist_setup()
    m = bench.max_over_ranks(10.0 + rank, ws)
    bench.barrier(ws)
    # the reference arm: every rank but 0 returns at once without work
    ran = None
    if rank != 0:
        ran = bench.run_reference(argparse.Namespace(steps=1, warmup=0))
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{got_ws} {got_rank} {m} {ran}\n")


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    for r in range(ws):
        got_ws, got_rank, m, ran = open(tmp_path / f"rank{r}.txt").read().split()
        assert int(got_ws) == ws and int(got_rank) == r
        assert float(m) == 11.0            # max over ranks
        if r != 0:
            assert ran == "None"
