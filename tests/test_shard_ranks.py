"""The z-hash sharded evolution (paper_2506_13241_gb300.shard) on CPU ranks:
gloo process groups of 2 and 4 ranks, each rank's part of the operator held
by the CPU oracle (tests/shardlib.py), the owner map and the exchange
protocol from the package.  Sharding must not change the result: the union
of the ranks' operators equals the single-process oracle's operator bit for
bit after every step (X layers run without any exchange), no string is held
by two ranks, every string sits on its owner, and <M_t> summed over the
ranks equals the single-process value."""
import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir, steps, delta):
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
    n = wl["n"]
    ev = shard.ShardedEvolution(OracleShard(n, oracle), shard.TorchComm())
    ev.set_terms(wl["observable"])
    mags, sizes = [], []
    for _ in range(steps):
        for layer in wl["layers"]:
            ev.apply_layer(layer, delta)
        mags.append(ev.expect())
        sizes.append(ev.engine.size())
    x, z, c = ev.engine.planes()
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), x=x, z=z, c=c, mags=np.array(mags),
             sizes=np.array(sizes), exchanged=ev.exchanged, total=ev.size())
    dist.destroy_process_group()


def _run(world, tmp_path, steps, delta):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), steps, delta), nprocs=world,
                       join=True, start_method="spawn")
    return [dict(np.load(tmp_path / ("rank%d.npz" % r))) for r in range(world)]


def _check_against_oracle(parts, oracle_mod, steps, delta):
    import paritylib
    from paper_2506_13241_gb300 import orqa as B, workloads as W
    wl = W.workload("heavyhex")
    n = wl["n"]
    mo, op = oracle_mod.run_layers(n, wl["observable"], wl["layers"], steps, delta)
    world = len(parts)
    x = np.concatenate([p["x"] for p in parts])
    z = np.concatenate([p["z"] for p in parts])
    c = np.concatenate([p["c"] for p in parts])
    # every string on its owner rank, none on two ranks
    for r, p in enumerate(parts):
        if len(p["c"]):
            assert np.all(B.orqa_shard_owner(n, p["z"], world) == r)
    key = np.concatenate([x, z], axis=1)
    assert len(np.unique(key, axis=0)) == len(key)
    got = paritylib.canonical(paritylib.planes_to_codes(x, z, n), c)
    paritylib.assert_bit_exact(got, paritylib.oracle_canonical(op, n), "sharded over %d ranks" % world)
    for p in parts:
        assert int(p["total"]) == len(op)
        assert np.max(np.abs(p["mags"] - np.array(mo))) < 1e-10
    return op


@pytest.mark.slow
def test_two_ranks_match_single_oracle(tmp_path, oracle_mod):
    """The 127-qubit heavy-hex kicked Ising circuit (theta = pi/4, Z_62, 5
    steps, delta = 1e-4) sharded over two gloo ranks."""
    parts = _run(2, tmp_path, 5, 1e-4)
    _check_against_oracle(parts, oracle_mod, 5, 1e-4)
    assert all(int(p["exchanged"]) > 0 for p in parts)  # the ZZ layers did move strings


@pytest.mark.slow
def test_four_ranks_balance(tmp_path, oracle_mod):
    """Four ranks: same result, and owner(z) spreads the 426,052 strings of
    step 5 within 5% of the mean per rank (the paper reports max/min shard
    sizes near 1 above 1e5 strings per process, App. C)."""
    parts = _run(4, tmp_path, 5, 1e-4)
    _check_against_oracle(parts, oracle_mod, 5, 1e-4)
    final = np.array([int(p["sizes"][-1]) for p in parts])
    assert final.sum() == 426052
    assert final.max() / final.mean() < 1.05 and final.min() / final.mean() > 0.95


def test_local_shards_match_single_oracle(oracle_mod):
    """The single-process driver (LocalShards) over three oracle shards on a
    random 40-qubit operator with random ZZ edges at all Clifford angles and
    random X subsets: union equal to the unsharded oracle after every layer."""
    import random

    import paritylib
    from paper_2506_13241_gb300 import shard
    from shardlib import OracleShard
    n = 40
    rng = random.Random(31)
    terms = [("".join(rng.choice("IXYZ") for _ in range(n)), rng.uniform(-1, 1)) for _ in range(60)]
    terms = list({lab: c for lab, c in terms}.items())
    ev = shard.LocalShards([OracleShard(n, oracle_mod) for _ in range(3)])
    ev.set_terms(terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    for step in range(3):
        edges = set()
        while len(edges) < 40:
            a, b = rng.sample(range(n), 2)
            edges.add((min(a, b), max(a, b)))
        zz = [("rzz", a, b, rng.choice([-math.pi / 2, math.pi / 2, math.pi])) for a, b in sorted(edges)]
        xx = [("rx", q, None, rng.choice([0.3, -0.7, math.pi / 4])) for q in sorted(rng.sample(range(n), 6))]
        for layer in (zz, xx):
            ev.apply_layer(layer, 1e-3)
            for g in layer:
                op.apply(g, 1e-3)
            planes = [e.planes() for e in ev.engines]
            x = np.concatenate([p[0] for p in planes])
            z = np.concatenate([p[1] for p in planes])
            c = np.concatenate([p[2] for p in planes])
            got = paritylib.canonical(paritylib.planes_to_codes(x, z, n), c)
            paritylib.assert_bit_exact(got, paritylib.oracle_canonical(op, n), "local shards step %d" % step)
        assert abs(ev.expect() - op.expect_zero()) < 1e-12
    assert ev.exchanged > 0


def test_owner_map_properties():
    """owner(z) depends on z alone (so an X layer never moves a string), is
    in range, and spreads distinct z planes evenly."""
    from paper_2506_13241_gb300 import orqa as B, shard
    rng = np.random.default_rng(3)
    z = rng.integers(0, 2 ** 63, size=(20000, 2), dtype=np.uint64)
    for R in (1, 2, 3, 7, 512):
        o = shard.owners(z, 127, R)
        assert o.min() >= 0 and o.max() < R
        if R > 1:
            counts = np.bincount(o, minlength=R)
            assert counts.max() < 1.25 * len(z) / R + 40
    assert np.array_equal(shard.owners(z[:, :1], 60, 5), shard.owners(z[:, :1].copy(), 60, 5))
    with pytest.raises(B.OrqaError):
        shard.owners(z, 127, 0)
    assert shard.moves_z([("rzz", 0, 1, -math.pi / 2)]) and not shard.moves_z([("rx", 0, None, 0.3)])
