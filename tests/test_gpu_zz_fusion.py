"""The held-back ZZ layer: a ZZ layer of Clifford angles is applied inside
the entry split of the X layer that follows it (the closed form of the ZZ
layer, string by string, before the split routes the string), instead of by
a pass of its own.  Every other call that reads or changes the operator
applies a held-back layer first.  Results must not depend on it: each test
runs the same calls on a context with the fusion (the default) and on one
with ORQA_DEBUG_NO_ZZ_FUSION, and compares the exported operators (canonical
order) bit for bit, and the oracle where it is cheap."""
import math

import numpy as np
import pytest

from paritylib import assert_bit_exact, gpu_canonical, oracle_canonical
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


def pair(orqa, n, terms, capacity=1 << 20, **kw):
    """Two contexts holding the same operator: fused (default), unfused."""
    a = orqa.Context(n, capacity, **kw)
    b = orqa.Context(n, capacity, **kw)
    b.debug_set(orqa.ORQA_DEBUG_NO_ZZ_FUSION, 1)
    for ctx in (a, b):
        ctx.set_labels(terms)
    return a, b


def same(a, b, what):
    xa, za, ca = a.export()
    xb, zb, cb = b.export()
    assert xa.shape == xb.shape, "%s: %d vs %d strings" % (what, len(ca), len(cb))
    assert np.array_equal(xa, xb) and np.array_equal(za, zb), what
    assert np.array_equal(ca.view(np.uint64), cb.view(np.uint64)), what


def heavyhex(orqa, steps, delta=1e-4, **kw):
    wl = W.workload("heavyhex")
    a, b = pair(orqa, wl["n"], wl["observable"], **kw)
    for _ in range(steps):
        for layer in wl["layers"]:
            a.apply_layer(layer, delta)
            b.apply_layer(layer, delta)
    return wl, a, b


@pytest.mark.parametrize("fp32", [False, True])
def test_fused_evolution_matches_unfused_and_oracle(orqa, oracle_mod, fp32):
    """Heavy-hex, theta = pi/4, Z_62, 5 steps at delta = 1e-4: equal after
    every step (the export applies nothing: each step ends on an X layer),
    and (FP64) equal to the oracle's operator."""
    wl = W.workload("heavyhex")
    n = wl["n"]
    a, b = pair(orqa, n, wl["observable"], fp32=fp32)
    for t in range(wl["steps"]):
        for layer in wl["layers"]:
            a.apply_layer(layer, wl["delta"])
            b.apply_layer(layer, wl["delta"])
        same(a, b, "step %d" % (t + 1))
        # the sum runs in buffer order, which the outputs' atomic
        # reservations decide: equal up to rounding
        assert abs(a.expect() - b.expect()) < 1e-12
    if not fp32:
        mo, op = oracle_mod.run_layers(n, wl["observable"], wl["layers"], wl["steps"], wl["delta"])
        assert_bit_exact(gpu_canonical(a, n), oracle_canonical(op, n), "fused vs oracle")
        assert abs(a.expect() - mo[-1]) < 1e-10


def test_one_word_planes_and_all_clifford_modes(orqa, oracle_mod):
    """W = 1 (40 qubits), ZZ layers at -pi/2, +pi/2 and pi mixed in one
    layer (one launch of several sets), random X angles and operators."""
    rng = np.random.default_rng(8)
    n = 40
    terms = [("".join(rng.choice(list("IXYZ"), n)), float(rng.uniform(-1, 1))) for _ in range(300)]
    terms = list(dict(terms).items())
    a, b = pair(orqa, n, terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    for step in range(3):
        edges = set()
        while len(edges) < 30:
            i, j = sorted(rng.choice(n, 2, replace=False))
            edges.add((int(i), int(j)))
        zz = [("rzz", i, j, float(rng.choice([-math.pi / 2, math.pi / 2, math.pi]))) for i, j in sorted(edges)]
        xx = [("rx", int(q), None, float(rng.uniform(-1, 1))) for q in sorted(rng.choice(n, 8, replace=False))]
        for layer in (zz, xx):
            a.apply_layer(layer, 1e-3)
            b.apply_layer(layer, 1e-3)
            for g in layer:
                op.apply(g, 1e-3)
        same(a, b, "step %d" % step)
        assert_bit_exact(gpu_canonical(a, n), oracle_canonical(op, n), "W=1 step %d" % step)


@pytest.mark.parametrize("follow", ["export", "expect", "histogram", "merge_truncate", "pauli", "zz_again",
                                    "stats", "set_operator", "no_fusion_knob"])
def test_every_other_call_applies_the_held_layer(orqa, follow):
    """After a ZZ layer (held back on the fused context) each other kind of
    call sees the layer applied: same outputs, same operator afterwards."""
    wl, a, b = heavyhex(orqa, 3)
    zz, xx = wl["layers"]
    a.apply_layer(zz, 1e-4)
    b.apply_layer(zz, 1e-4)
    if follow == "export":
        pass
    elif follow == "expect":
        assert abs(a.expect() - b.expect()) < 1e-12
    elif follow == "histogram":
        ha, ma = a.histogram(32, -12.0)
        hb, mb = b.histogram(32, -12.0)
        assert np.array_equal(ha, hb) and ma == mb
    elif follow == "merge_truncate":
        assert a.merge_truncate(3e-4) == b.merge_truncate(3e-4)
    elif follow == "pauli":
        lab = "".join("X" if q in (3, 4) else ("Z" if q == 5 else "I") for q in range(wl["n"]))
        assert a.apply_pauli_rotation(lab, 0.3, 1e-4) == b.apply_pauli_rotation(lab, 0.3, 1e-4)
    elif follow == "zz_again":
        a.apply_layer(zz, 1e-4)
        b.apply_layer(zz, 1e-4)
    elif follow == "stats":
        sa, sb = a.stats(), b.stats()
        assert abs(sa["sum_sq"] - sb["sum_sq"]) < 1e-12 and sa["max_abs"] == sb["max_abs"]
    elif follow == "set_operator":
        for ctx in (a, b):
            ctx.set_labels(wl["observable"])
    elif follow == "no_fusion_knob":
        a.debug_set(orqa.ORQA_DEBUG_NO_ZZ_FUSION, 1)
        a.debug_set(orqa.ORQA_DEBUG_NO_ZZ_FUSION, 0)
    same(a, b, follow)
    # and the next X layer still agrees
    a.apply_layer(xx, 1e-4)
    b.apply_layer(xx, 1e-4)
    same(a, b, follow + " then X")


def test_failed_x_layer_keeps_the_held_layer(orqa):
    """An X layer that fails (pass limit) after a held-back ZZ layer leaves
    the operator after the ZZ layer; a ZZ layer after a failed call is
    applied (error bits of the failed call do not make it skip)."""
    wl, a, b = heavyhex(orqa, 3)
    zz, xx = wl["layers"]
    for ctx in (a, b):
        ctx.apply_layer(zz, 1e-4)
        ctx.debug_set(orqa.ORQA_DEBUG_PASS_LIMIT, 1)
        with pytest.raises(orqa.OrqaError) as ei:
            ctx.apply_layer(xx, 1e-4)
        assert ei.value.status == orqa.ORQA_ETIMEOUT
    same(a, b, "after the failed layer")
    for ctx in (a, b):
        ctx.debug_set(orqa.ORQA_DEBUG_PASS_LIMIT, 1)
        with pytest.raises(orqa.OrqaError):
            ctx.apply_layer(xx, 1e-4)
        ctx.apply_layer(zz, 1e-4)  # right after a failure, on both
        ctx.debug_set(orqa.ORQA_DEBUG_PASS_LIMIT, 0)
        ctx.apply_layer(xx, 1e-4)
    ref = orqa.Context(wl["n"], 1 << 20)
    ref.debug_set(orqa.ORQA_DEBUG_NO_ZZ_FUSION, 1)
    ref.set_labels(wl["observable"])
    for _ in range(3):
        for layer in wl["layers"]:
            ref.apply_layer(layer, 1e-4)
    for layer in (zz, zz, xx):
        ref.apply_layer(layer, 1e-4)
    same(a, ref, "fused after failures")
    same(b, ref, "unfused after failures")


def test_programs_fuse_between_layers(orqa):
    """A captured program of 4 steps, with and without fusion, and with an
    expectation after the ZZ layer (which keeps that layer unfused): the
    same expectations and the same operator bit for bit."""
    wl = W.workload("heavyhex")
    zz, xx = wl["layers"]
    out = []
    for fuse, mark_zz in ((True, False), (False, False), (True, True)):
        ctx = orqa.Context(wl["n"], 1 << 20)
        if not fuse:
            ctx.debug_set(orqa.ORQA_DEBUG_NO_ZZ_FUSION, 1)
        ctx.set_labels(wl["observable"])
        prog = ctx.program([(zz, mark_zz, None), (xx, True, None)])
        m = ctx.run_program(prog, 4, 1e-4)
        m = m[1::2] if mark_zz else m
        out.append((m, ctx.export()))
    for m, (x, z, c) in out[1:]:
        assert np.max(np.abs(m - out[0][0])) < 1e-12
        assert np.array_equal(x, out[0][1][0]) and np.array_equal(z, out[0][1][1])
        assert np.array_equal(c.view(np.uint64), out[0][1][2].view(np.uint64))


def test_sharded_evolution_with_held_layers(orqa):
    """The sharded driver splits after each ZZ layer, which applies the held
    layer first: two shards equal one unfused context."""
    from paper_2506_13241_gb300 import shard
    wl = W.workload("heavyhex")
    n = wl["n"]
    ev = shard.LocalShards([shard.GpuShard(orqa.Context(n, 1 << 19)) for _ in range(2)])
    ev.set_terms(wl["observable"])
    ref = orqa.Context(n, 1 << 20)
    ref.debug_set(orqa.ORQA_DEBUG_NO_ZZ_FUSION, 1)
    ref.set_labels(wl["observable"])
    for _ in range(4):
        for layer in wl["layers"]:
            ev.apply_layer(layer, 1e-4)
            ref.apply_layer(layer, 1e-4)
    assert abs(ev.expect() - ref.expect()) < 1e-12
    assert ev.size() == len(ref)
