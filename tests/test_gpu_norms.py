"""Norm bookkeeping of the CUDA path (orqa_stats: sum c^2, max |c|, and the
sum of c^2 that each truncation removed) against the oracle and against the
unitarity of the rotations: Eq. (update_rule) maps every pair (c_Z, c_Y) by
an orthogonal 2x2 matrix, so sum c^2 is unchanged by a gate and falls only
by what the truncation of Eq. (truncation1) removes."""
import math

import numpy as np
import pytest

from paper_2506_13241_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# fixed-order FP64 sums over <= 1e6 terms: a few 1e-15 relative; the
# rotations add a few ulps per update
REL_TOL = 1e-12


@pytest.fixture(scope="module")
def orqa():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2506_13241_gb300 import build, orqa as binding
    build.build()
    return binding


def test_norms_match_oracle_and_balance_per_layer(orqa, oracle_mod):
    """Heavy-hex, theta = pi/4, Z_62, 5 steps, delta = 1e-4: sum c^2 and max|c|
    equal the oracle's after every layer, and sum c^2 before a layer minus
    sum c^2 after it equals the dropped sum of c^2 the kernels report."""
    wl = W.workload("heavyhex")
    n = wl["n"]
    ctx = orqa.Context(n, 1 << 20)
    ctx.set_labels(wl["observable"])
    ctx.set_norm_tracking(True)
    op = oracle_mod.Oracle(n)
    for lab, c in wl["observable"]:
        op.add_label(lab, c)
    before = ctx.stats()["sum_sq"]
    assert before == 1.0
    worst = 0.0
    for t in range(wl["steps"]):
        for layer in wl["layers"]:
            ctx.apply_layer(layer, wl["delta"])
            for g in layer:
                op.apply(g, wl["delta"])
            s = ctx.stats()
            assert abs(s["sum_sq"] - op.norm2()) <= REL_TOL * op.norm2()
            assert s["max_abs"] == op.max_abs()
            gap = abs(before - s["sum_sq"] - s["dropped_sum_sq"]) / before
            worst = max(worst, gap)
            assert gap <= REL_TOL, (t, layer[0][0], before, s["sum_sq"], s["dropped_sum_sq"])
            before = s["sum_sq"]
    assert before < 1.0  # truncation did remove weight
    assert worst <= REL_TOL


def test_norm_conserved_without_truncation(orqa):
    """12-qubit chain, theta = pi/4, Z_6, 5 steps at delta = 0: sum c^2 stays 1 and
    nothing is dropped."""
    wl = W.workload("chain12")
    ctx = orqa.Context(wl["n"], 1 << 20)
    ctx.set_labels(wl["observable"])
    ctx.set_norm_tracking(True)
    for _ in range(wl["steps"]):
        for layer in wl["layers"]:
            ctx.apply_layer(layer, 0.0)
            s = ctx.stats()
            assert abs(s["sum_sq"] - 1.0) < 1e-13
            assert s["dropped_sum_sq"] == 0.0


def test_dropped_norm_untracked_is_nan_and_results_unchanged(orqa):
    """Without tracking the X layer reports NaN for the dropped sum of c^2,
    and the operator is the same bit for bit as with tracking."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, math.pi / 4)
    out = []
    for track in (False, True):
        ctx = orqa.Context(n, 1 << 20)
        ctx.set_labels([(W.z_label(n, [62]), 1.0)])
        ctx.set_norm_tracking(track)
        for _ in range(4):
            for layer in layers:
                ctx.apply_layer(layer, 1e-4)
        s = ctx.stats()
        assert math.isnan(s["dropped_sum_sq"]) != track
        x, z, c = ctx.export()
        order = np.lexsort(np.concatenate([x, z], axis=1).T[::-1])
        out.append((x[order], z[order], c[order].view(np.uint64)))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_norms_of_merge_truncate(orqa, oracle_mod):
    """merge_truncate reports the sum of c^2 of the merged entries it drops."""
    n = 16
    rng = np.random.default_rng(5)
    labels = ["".join(rng.choice(list("IXYZ"), n)) for _ in range(300)]
    coefs = rng.uniform(-1, 1, size=300) * 10.0 ** rng.uniform(-5, 0, size=300)
    terms = list(zip(labels, coefs))
    ctx = orqa.Context(n, 1 << 12)
    ctx.set_labels(terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    before = ctx.stats()["sum_sq"]
    assert abs(before - op.norm2()) <= REL_TOL * op.norm2()
    ctx.merge_truncate(1e-2)
    op.truncate(1e-2)
    s = ctx.stats()
    assert abs(s["sum_sq"] - op.norm2()) <= REL_TOL * before
    assert abs(before - s["sum_sq"] - s["dropped_sum_sq"]) <= REL_TOL * before
    assert s["max_abs"] == op.max_abs()
