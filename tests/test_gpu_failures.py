"""Failure paths of the CUDA path, made to fire from the host through the
test hooks of orqa_debug_set: every device-side wait and loop is bounded, so
each condition ends the kernels with an error bit and the call returns its
status with the operator held before the call unchanged.  Nothing here
faults, traps or hangs the GPU: a poisoned merge table makes each insertion
wait out its (short) spin limit; a small table, pass limit or bucket count
makes a bounded loop or a capacity check give up."""
import math

import numpy as np
import pytest

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


def snapshot(ctx):
    x, z, c = ctx.export()
    key = np.concatenate([x, z], axis=1)
    order = np.lexsort(key.T[::-1])
    return key[order], c[order].view(np.uint64)


def same(a, b):
    return a[0].shape == b[0].shape and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def heavyhex_state(orqa, steps, delta=1e-4, capacity=1 << 20):
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, math.pi / 4)
    ctx = orqa.Context(n, capacity)
    ctx.set_labels([(W.z_label(n, [62]), 1.0)])
    for _ in range(steps):
        for layer in layers:
            ctx.apply_layer(layer, delta)
    return ctx, layers


def random_terms(n, k, seed):
    rng = np.random.default_rng(seed)
    labels = {"".join(rng.choice(list("IXYZ"), n)) for _ in range(k)}
    return [(lab, float(rng.uniform(0.5, 1.0))) for lab in sorted(labels)]


def test_merge_wait_times_out_and_keeps_operator(orqa):
    """Every merge-table slot marked busy: each insertion's bounded wait runs
    out, the call returns ORQA_ETIMEOUT, and the operator is unchanged."""
    n = 20
    ctx = orqa.Context(n, 1 << 12)
    ctx.set_labels(random_terms(n, 200, 1))
    before = snapshot(ctx)
    ctx.debug_set(orqa.ORQA_DEBUG_SPIN_LIMIT, 256)
    ctx.debug_set(orqa.ORQA_DEBUG_POISON_MERGE_TABLE, 1)
    with pytest.raises(orqa.OrqaError) as ei:
        ctx.merge_truncate(0.0)
    assert ei.value.status == orqa.ORQA_ETIMEOUT
    assert same(snapshot(ctx), before)
    with pytest.raises(orqa.OrqaError) as ei:
        ctx.set_labels(random_terms(n, 50, 2))
    assert ei.value.status == orqa.ORQA_ETIMEOUT
    assert same(snapshot(ctx), before)
    # the hooks off again: the same calls succeed
    ctx.debug_set(orqa.ORQA_DEBUG_POISON_MERGE_TABLE, 0)
    ctx.debug_set(orqa.ORQA_DEBUG_SPIN_LIMIT, 0)
    assert ctx.merge_truncate(0.0) == len(before[1])
    assert same(snapshot(ctx), before)


def test_merge_table_full_keeps_operator(orqa):
    """More distinct strings than merge-table slots: the probe loop gives up
    with ORQA_ECAPACITY and the operator is unchanged."""
    n = 20
    ctx = orqa.Context(n, 1 << 12)
    ctx.set_labels(random_terms(n, 40, 3))
    before = snapshot(ctx)
    ctx.debug_set(orqa.ORQA_DEBUG_MERGE_TABLE_SLOTS, 16)
    with pytest.raises(orqa.OrqaError) as ei:
        ctx.set_labels(random_terms(n, 100, 4))
    assert ei.value.status == orqa.ORQA_ECAPACITY
    assert "table full" in str(ei.value)
    assert same(snapshot(ctx), before)
    ctx.debug_set(orqa.ORQA_DEBUG_MERGE_TABLE_SLOTS, 0)
    ctx.set_labels(random_terms(n, 100, 4))
    assert len(ctx) == 100


def test_pass_limit_keeps_operator(orqa, oracle_mod):
    """An X layer that needs two chunk passes under a one-pass limit returns
    ORQA_ETIMEOUT with the operator unchanged; without the limit the same
    layer gives the oracle's operator bit for bit."""
    import paritylib
    ctx, layers = heavyhex_state(orqa, 3)
    ctx.apply_layer(layers[0], 1e-4)
    before = snapshot(ctx)
    ctx.debug_set(orqa.ORQA_DEBUG_PASS_LIMIT, 1)
    with pytest.raises(orqa.OrqaError) as ei:
        ctx.apply_layer(layers[1], 1e-4)
    assert ei.value.status == orqa.ORQA_ETIMEOUT
    assert "pass limit" in str(ei.value)
    assert same(snapshot(ctx), before)
    ctx.debug_set(orqa.ORQA_DEBUG_PASS_LIMIT, 0)
    ctx.apply_layer(layers[1], 1e-4)
    n = ctx.n_qubits
    mo, op = oracle_mod.run_layers(n, [(W.z_label(n, [62]), 1.0)], layers, 4, 1e-4)
    paritylib.assert_bit_exact(paritylib.gpu_canonical(ctx, n), paritylib.oracle_canonical(op, n), "after limit")
    assert abs(ctx.expect() - mo[-1]) < 1e-10


def test_pass_limit_in_captured_program(orqa):
    """Inside a captured program the pass limit stops the graph: the call
    returns ORQA_ETIMEOUT and the context holds the operator of the last
    completed layer (here the ZZ layer before it)."""
    ctx, layers = heavyhex_state(orqa, 3)
    ref, _ = heavyhex_state(orqa, 3)
    ref.apply_layer(layers[0], 1e-4)
    prog = ctx.program([(layers[0], False, None), (layers[1], True, None)])
    ctx.debug_set(orqa.ORQA_DEBUG_PASS_LIMIT, 1)
    with pytest.raises(orqa.OrqaError) as ei:
        ctx.run_program(prog, 1, 1e-4)
    assert ei.value.status == orqa.ORQA_ETIMEOUT
    assert same(snapshot(ctx), snapshot(ref))


def test_bucket_overflow_keeps_operator(orqa):
    """All strings forced into two fine buckets: a bucket above the
    shared-memory range size ends the unit kernel with ORQA_ECAPACITY and
    the operator is unchanged."""
    ctx, layers = heavyhex_state(orqa, 4)
    ctx.apply_layer(layers[0], 1e-4)
    before = snapshot(ctx)
    assert len(before[1]) == 2582  # more than two 512-string ranges
    ctx.debug_set(orqa.ORQA_DEBUG_BUCKET_SHIFT, 63)
    with pytest.raises(orqa.OrqaError) as ei:
        ctx.apply_layer(layers[1], 1e-4)
    assert ei.value.status == orqa.ORQA_ECAPACITY
    assert same(snapshot(ctx), before)
    ctx.debug_set(orqa.ORQA_DEBUG_BUCKET_SHIFT, 0)
    ctx.apply_layer(layers[1], 1e-4)


def test_debug_knobs_validated(orqa):
    ctx = orqa.Context(8, 64)
    for knob, value in ((orqa.ORQA_DEBUG_SPIN_LIMIT, -1), (orqa.ORQA_DEBUG_POISON_MERGE_TABLE, 2),
                        (orqa.ORQA_DEBUG_MERGE_TABLE_SLOTS, 24), (orqa.ORQA_DEBUG_PASS_LIMIT, 33),
                        (orqa.ORQA_DEBUG_BUCKET_SHIFT, 64), (99, 0)):
        with pytest.raises(orqa.OrqaError) as ei:
            ctx.debug_set(knob, value)
        assert ei.value.status == orqa.ORQA_EINVAL
