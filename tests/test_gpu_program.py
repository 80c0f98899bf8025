"""Captured programs (orqa_run_program: a layer sequence as one CUDA graph
with device-side pass loops) against the same layers applied one call at a
time, and against the CPU oracle.  Results are bit-exact; expectations agree
to 1e-10 (summation order)."""
import math

import numpy as np
import pytest

from paritylib import assert_bit_exact, canonical, gpu_canonical, oracle_canonical, planes_to_codes
from paper_2506_13241_gb300 import workloads as W

pytestmark = pytest.mark.gpu

M_TOL = 1e-10


@pytest.fixture(scope="module")
def orqa():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2506_13241_gb300 import build, orqa as binding
    build.build()
    return binding


def batch_sets(ctx, n, P):
    x, z, c, p = ctx.export_batch()
    codes = planes_to_codes(x, z, n)
    return [canonical(codes[p == k], c[p == k]) for k in range(P)]


def kicked_program(orqa, ctx, layers):
    zz, xx = layers
    return ctx.program([(zz, False, None), (xx, True, None)])


@pytest.mark.parametrize("fp32", [False, True])
def test_program_matches_layer_calls(orqa, oracle_mod, fp32):
    """heavy-hex, theta = pi/4, Z_62, 5 steps, delta = 1e-4 as one graph
    launch: the same operator as five pairs of apply_layer calls, and the
    oracle's magnetization; a second run replays the cached graph."""
    wl = W.workload("heavyhex")
    n, delta = wl["n"], wl["delta"]
    ref = orqa.Context(n, 1 << 21, fp32=fp32)
    ref.set_labels(wl["observable"])
    mr = []
    for _ in range(5):
        for layer in wl["layers"]:
            ref.apply_layer(layer, delta)
        mr.append(ref.expect())
    ctx = orqa.Context(n, 1 << 21, fp32=fp32)
    prog = kicked_program(orqa, ctx, wl["layers"])
    for run in range(2):
        ctx.set_labels(wl["observable"])
        m = ctx.run_program(prog, 5, delta)[:, 0]
        assert np.max(np.abs(m - np.array(mr))) < M_TOL, run
        assert_bit_exact(gpu_canonical(ctx, n), gpu_canonical(ref, n), "run %d" % run)
    st = ctx.stats()
    assert st["n_strings"] == len(ref)
    assert st["string_gate_updates"] > 0 and st["chunk_passes"] >= 5
    if not fp32:
        mo, _ = oracle_mod.run_layers(n, wl["observable"], wl["layers"], 5, delta)
        assert np.max(np.abs(m - np.array(mo))) < M_TOL


def test_program_updates_match_layer_calls(orqa):
    """The program's string-gate update count equals the sum of the per-layer
    counts of the same layers applied one call at a time."""
    wl = W.workload("heavyhex_t=3")
    n, delta = wl["n"], wl["delta"]
    ref = orqa.Context(n, 1 << 21)
    ref.set_labels(wl["observable"])
    total = 0
    for _ in range(3):
        for layer in wl["layers"]:
            ref.apply_layer(layer, delta)
            total += ref.stats()["string_gate_updates"]
    ctx = orqa.Context(n, 1 << 21)
    ctx.set_labels(wl["observable"])
    ctx.run_program(kicked_program(orqa, ctx, wl["layers"]), 3, delta)
    assert ctx.stats()["string_gate_updates"] == total


def test_update_counts_match_oracle(orqa, oracle_mod):
    """The string-gate update count of a layer is the sum over its gates of
    |O| before the gate: taken from the oracle gate by gate (heavy-hex,
    theta = pi/4, 4 steps, delta = 1e-4, so strings branch, merge and drop
    inside the layers), it equals the CUDA path's count for every layer
    applied by a call, and their total equals a captured program's count."""
    wl = W.workload("heavyhex")
    n, delta = wl["n"], 1e-4
    op = oracle_mod.Oracle(n)
    for lab, c in wl["observable"]:
        op.add_label(lab, c)
    ctx = orqa.Context(n, 1 << 20)
    ctx.set_labels(wl["observable"])
    total = 0
    for t in range(4):
        for layer in wl["layers"]:
            expected = 0
            for g in layer:
                expected += len(op)
                op.apply(g, delta)
            ctx.apply_layer(layer, delta)
            got = ctx.counters()["string_gate_updates"]
            assert got == expected, (t, layer[0][0], got, expected)
            total += expected
    prog_ctx = orqa.Context(n, 1 << 20)
    prog_ctx.set_labels(wl["observable"])
    prog_ctx.run_program(kicked_program(orqa, prog_ctx, wl["layers"]), 4, delta)
    assert prog_ctx.counters()["string_gate_updates"] == total


def test_batched_program(orqa, oracle_mod):
    """theta x observable sweep (4 angles x weights 1, 3, 5; 3 steps;
    delta = 1e-4) as one graph: bit-exact per problem against the oracle."""
    wl = W.sweep_workload(4, 3, 1e-4, (1, 3, 5))
    n, P = wl["n"], len(wl["problems"])
    zz, xx = wl["layers"]
    theta = np.array([[wl["theta"][p]] * len(xx) for p in range(P)])
    ctx = orqa.Context(n, 1 << 22, problems=P)
    prog = ctx.program([(zz, False, None), (xx, True, theta)])
    ctx.set_labels_batch(wl["problems"])
    mags = ctx.run_program(prog, 3, 1e-4)
    assert mags.shape == (3, P)
    sets = batch_sets(ctx, n, P)
    for p in range(P):
        layers = W.kicked_ising_layers(n, wl["edges"], wl["theta"][p])
        mo, op = oracle_mod.run_layers(n, wl["problems"][p], layers, 3, 1e-4)
        assert np.max(np.abs(mags[:, p] - np.array(mo))) < M_TOL, p
        assert_bit_exact(sets[p], oracle_canonical(op, n), "problem %d" % p)


def test_tuning_does_not_change_results(orqa):
    """Every tuning gives the same operator, bit for bit."""
    wl = W.workload("heavyhex")
    n, delta = wl["n"], wl["delta"]
    ctx = orqa.Context(n, 1 << 21)
    prog = kicked_program(orqa, ctx, wl["layers"])
    ref = None
    for tune in [dict(), dict(range_target=128, sub_max=256, bucket_density=8, grid_per_sm=1),
                 dict(range_target=1024, sub_max=256, bucket_density=64, grid_per_sm=32),
                 dict(range_target=448, sub_max=256, bucket_density=85, grid_per_sm=24),
                 dict(range_target=320, sub_max=128, bucket_density=32, grid_per_sm=16)]:
        if tune:
            ctx.set_tuning(**tune)
        ctx.set_labels(wl["observable"])
        m = ctx.run_program(prog, 5, delta)[:, 0]
        got = gpu_canonical(ctx, n)
        if ref is None:
            ref, mref = got, m
        else:
            assert_bit_exact(got, ref, str(tune))
            assert np.max(np.abs(m - mref)) < M_TOL
    for bad in [dict(range_target=64), dict(sub_max=1024), dict(bucket_density=7), dict(bucket_density=129),
                dict(grid_per_sm=0),
                dict(sub_max=128, bucket_density=48)]:  # a bucket must fit a sub-range with a factor 3 of margin
        with pytest.raises(orqa.OrqaError) as e:
            ctx.set_tuning(**bad)
        assert e.value.status == orqa.ORQA_EINVAL


def test_autotune_restores_operator(orqa):
    wl = W.workload("heavyhex_t=3")
    n, delta = wl["n"], wl["delta"]
    ctx = orqa.Context(n, 1 << 21)
    prog = kicked_program(orqa, ctx, wl["layers"])
    ctx.set_labels(wl["observable"])
    before = gpu_canonical(ctx, n)
    best, ms = ctx.autotune(prog, 3, delta, trials=1)
    assert ms > 0
    assert best == ctx.tuning()
    assert_bit_exact(gpu_canonical(ctx, n), before, "operator after autotune")


def test_program_capacity_error_keeps_last_layer(orqa):
    """A program that overflows the capacity stops on the device: the call
    returns ORQA_ECAPACITY, the context holds the operator after the last
    completed layer (equal to the layer-call path stopped at the same
    point)."""
    wl = W.workload("heavyhex")
    n, delta, cap = wl["n"], wl["delta"], 10000
    ref = orqa.Context(n, cap)
    ref.set_labels(wl["observable"])
    mr, failed = [], False
    for _ in range(5):
        for layer in wl["layers"]:
            try:
                ref.apply_layer(layer, delta)
            except orqa.OrqaError as e:
                assert e.status == orqa.ORQA_ECAPACITY
                failed = True
                break
        if failed:
            break
        mr.append(ref.expect())
    assert failed
    ctx = orqa.Context(n, cap)
    prog = kicked_program(orqa, ctx, wl["layers"])
    ctx.set_labels(wl["observable"])
    with pytest.raises(orqa.OrqaError) as e:
        ctx.run_program(prog, 5, delta)
    assert e.value.status == orqa.ORQA_ECAPACITY
    assert_bit_exact(gpu_canonical(ctx, n), gpu_canonical(ref, n), "state after the failing layer")
    assert abs(ctx.expect() - ref.expect()) < M_TOL


@pytest.mark.parametrize("fp32", [False, True])
def test_batched_program_one_word_planes(orqa, oracle_mod, fp32):
    """A batched program on 40 qubits (one 64-bit word per plane): random
    edges with a Clifford ZZ layer and X layers with per-problem angles;
    FP64 bit-exact per problem, FP32 within 1e-6 of the oracle."""
    import random
    rng = random.Random(4040)
    n = 40
    edges = set()
    while len(edges) < 45:
        a, b = rng.sample(range(n), 2)
        edges.add((min(a, b), max(a, b)))
    edges = sorted(edges)
    thetas = [0.0, 0.4, math.pi / 4, 1.1, math.pi / 2]
    obs = [W.z_label(n, [7]), W.z_label(n, [3, 20, 33])]
    problems = [[(lab, 1.0)] for th in thetas for lab in obs]
    theta_p = [th for th in thetas for _ in obs]
    P = len(problems)
    zz = [("rzz", a, b, -math.pi / 2) for a, b in edges]
    xx = [("rx", q, None, 0.3) for q in range(n)]
    theta = np.array([[theta_p[p]] * n for p in range(P)])
    ctx = orqa.Context(n, 1 << 22, problems=P, fp32=fp32)
    prog = ctx.program([(zz, False, None), (xx, True, theta)])
    ctx.set_labels_batch(problems)
    mags = ctx.run_program(prog, 3, 1e-4)
    sets = batch_sets(ctx, n, P)
    for p in range(P):
        layers = [zz, [("rx", q, None, theta_p[p]) for q in range(n)]]
        mo, op = oracle_mod.run_layers(n, problems[p], layers, 3, 1e-4)
        if fp32:
            assert np.max(np.abs(mags[:, p] - np.array(mo))) < 1e-6, p
        else:
            assert np.max(np.abs(mags[:, p] - np.array(mo))) < M_TOL, p
            assert_bit_exact(sets[p], oracle_canonical(op, n), "problem %d" % p)
