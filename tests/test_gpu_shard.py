"""The z-hash sharded evolution on the GPU: R liborqa contexts on one GPU
driven by shard.LocalShards (orqa_shard_split on every shard, records
exchanged by device copies, orqa_shard_append), against one unsharded
context and the oracle.  The union of the shards must equal the unsharded
operator bit for bit, every string must sit on its owner (the device owner
map equals the host one), and the summed <M_t> must agree to 1e-10."""
import math

import numpy as np
import pytest

from paritylib import assert_bit_exact, canonical, gpu_canonical, oracle_canonical, planes_to_codes
from paper_2506_13241_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orqa():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2506_13241_gb300 import build, orqa as binding
    build.build()
    return binding


def shards_union(ev, n):
    parts = [e.ctx.export() for e in ev.engines]
    x = np.concatenate([p[0] for p in parts])
    z = np.concatenate([p[1] for p in parts])
    c = np.concatenate([p[2] for p in parts])
    return parts, canonical(planes_to_codes(x, z, n), c)


@pytest.mark.parametrize("R", [2, 3])
def test_sharded_heavyhex_matches_unsharded(orqa, oracle_mod, R):
    from paper_2506_13241_gb300 import shard
    wl = W.workload("heavyhex")
    n = wl["n"]
    ev = shard.LocalShards([shard.GpuShard(orqa.Context(n, 1 << 19)) for _ in range(R)])
    ev.set_terms(wl["observable"])
    ref = orqa.Context(n, 1 << 20)
    ref.set_labels(wl["observable"])
    for t in range(wl["steps"]):
        for layer in wl["layers"]:
            ev.apply_layer(layer, wl["delta"])
            ref.apply_layer(layer, wl["delta"])
        parts, got = shards_union(ev, n)
        assert_bit_exact(got, gpu_canonical(ref, n), "R=%d step %d" % (R, t + 1))
        for r, (x, z, c) in enumerate(parts):
            if len(c):
                assert np.all(shard.owners(z, n, R) == r)
        assert abs(ev.expect() - ref.expect()) < 1e-10
    assert ev.size() == 426052
    mo, op = oracle_mod.run_layers(n, wl["observable"], wl["layers"], wl["steps"], wl["delta"])
    assert_bit_exact(shards_union(ev, n)[1], oracle_canonical(op, n), "R=%d vs oracle" % R)
    assert abs(ev.expect() - mo[-1]) < 1e-10
    sizes = np.array(ev.sizes())
    assert sizes.max() / sizes.mean() < 1.05


def test_split_and_append_limits(orqa):
    """A send buffer too small for the strings that leave, and an append
    beyond the capacity, return ORQA_ECAPACITY with the operator unchanged."""
    import torch
    from paper_2506_13241_gb300 import shard
    n = 40
    rng = np.random.default_rng(12)
    terms = [("".join(rng.choice(list("IXYZ"), n)), float(rng.uniform(-1, 1))) for _ in range(500)]
    ctx = orqa.Context(n, 1024)
    ctx.set_labels(terms)
    before = gpu_canonical(ctx, n)
    small = shard.GpuShard(ctx, send_capacity=10)
    with pytest.raises(orqa.OrqaError) as ei:
        small.split(4, 1)
    assert ei.value.status == orqa.ORQA_ECAPACITY
    assert_bit_exact(gpu_canonical(ctx, n), before, "after failed split")
    big = shard.GpuShard(ctx)
    send, counts = big.split(4, 1)
    assert counts[1] == 0 and sum(counts) == send.shape[0] and len(ctx) == len(before[1]) - sum(counts)
    # the records carry the strings: putting them back restores the operator
    kept = len(ctx)
    recv = send.clone()
    big.append(recv)
    assert len(ctx) == kept + recv.shape[0]
    assert_bit_exact(gpu_canonical(ctx, n), before, "split then append")
    too_many = torch.zeros((1024, shard.record_words(n)), dtype=torch.int64, device="cuda")
    with pytest.raises(orqa.OrqaError) as ei:
        big.append(too_many)
    assert ei.value.status == orqa.ORQA_ECAPACITY
    assert_bit_exact(gpu_canonical(ctx, n), before, "after failed append")


def test_sharded_fp32_and_one_word_planes(orqa):
    """FP32 coefficients (records carry float bits) and W = 1 planes: the
    sharded run equals the unsharded one bit for bit."""
    from paper_2506_13241_gb300 import shard
    wl = W.workload("chain12")
    n = wl["n"]
    for fp32 in (False, True):
        ev = shard.LocalShards([shard.GpuShard(orqa.Context(n, 1 << 18, fp32=fp32)) for _ in range(2)])
        ev.set_terms(wl["observable"])
        ref = orqa.Context(n, 1 << 18, fp32=fp32)
        ref.set_labels(wl["observable"])
        for _ in range(wl["steps"]):
            for layer in wl["layers"]:
                ev.apply_layer(layer, 1e-6)
                ref.apply_layer(layer, 1e-6)
        assert_bit_exact(shards_union(ev, n)[1], gpu_canonical(ref, n), "fp32=%s" % fp32)
        assert abs(ev.expect() - ref.expect()) < 1e-12
