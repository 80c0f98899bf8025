"""Element-by-element parity at more than 1e7 strings: the 127-qubit
heavy-hex kicked Ising circuit (theta = pi/4, Z_62) for 6 steps at delta = 2e-5, where
the operator holds 12,716,456 strings.  The single-threaded oracle needs
minutes for this, so the oracle runs sharded by owner(z) over CPU gloo ranks
(one oracle per rank; the sharding is exact, see test_shard_ranks.py, which
checks it against the unsharded oracle); the CUDA path runs unsharded in one
context.  Sets and coefficients must be bit-exact, in the canonical order of
orqa_export; <M_t> within 1e-10."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
STEPS, DELTA, SIZE = 6, 2e-5, 12716456

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_rank(rank, world, port, out_dir):
    import torch.distributed as dist
    for p in (ROOT, HERE):
        if p not in sys.path:
            sys.path.insert(0, p)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2506_13241_gb300 import shard, workloads as W
    from shardlib import OracleShard
    wl = W.workload("heavyhex")
    ev = shard.ShardedEvolution(OracleShard(wl["n"], oracle), shard.TorchComm())
    ev.set_terms(wl["observable"])
    mags = []
    for _ in range(STEPS):
        for layer in wl["layers"]:
            ev.apply_layer(layer, DELTA)
        mags.append(ev.expect())
    x, z, c = ev.engine.planes()
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), x=x, z=z, c=c, mags=np.array(mags))
    dist.destroy_process_group()


def test_heavyhex_over_1e7_strings(tmp_path):
    import torch
    import torch.multiprocessing as mp
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paritylib import canonical_key_order
    from paper_2506_13241_gb300 import build, orqa, workloads as W
    build.build()
    # the oracle side first, in CPU processes (none of them touches the GPU)
    world = max(2, min(16, os.cpu_count() or 2))
    mp.start_processes(_oracle_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    parts = [np.load(tmp_path / ("rank%d.npz" % r)) for r in range(world)]
    x = np.concatenate([p["x"] for p in parts])
    z = np.concatenate([p["z"] for p in parts])
    c = np.concatenate([p["c"] for p in parts])
    mo = parts[0]["mags"]
    order = canonical_key_order(x, z)
    x, z, c = x[order], z[order], c[order]
    assert len(c) == SIZE
    # the CUDA path, unsharded
    wl = W.workload("heavyhex")
    ctx = orqa.Context(wl["n"], 4 * SIZE)
    ctx.set_labels(wl["observable"])
    mg = []
    for _ in range(STEPS):
        for layer in wl["layers"]:
            ctx.apply_layer(layer, DELTA)
        mg.append(ctx.expect())
    gx, gz, gc = ctx.export()
    assert len(gc) == SIZE
    assert np.array_equal(gx, x) and np.array_equal(gz, z)
    bad = np.nonzero(gc.view(np.uint64) != c.view(np.uint64))[0]
    assert bad.size == 0, "%d coefficients differ, first row %d" % (bad.size, bad[0])
    assert np.max(np.abs(np.array(mg) - mo)) < 1e-10
