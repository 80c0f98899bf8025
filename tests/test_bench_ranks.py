"""Host logic of bench.py under torchrun (replicas on N ranks): the timing
is the slowest rank's and the work is summed over the ranks.  Runs as two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times, counts = bench.reduce_over_ranks([10.0 + rank, 5.0 - rank], [100 + rank, 7], "cpu")
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%r %r\n" % (times, counts))
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        got = (tmp_path / ("rank%d.txt" % rank)).read_text().strip()
        assert got == "[11.0, 5.0] [201, 14]", got


def test_reduce_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks([1.5, 2.5], [3, 4]) == ([1.5, 2.5], [3, 4])
