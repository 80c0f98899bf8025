"""CUDA path against the CPU oracle, element by element, through the C ABI.

String sets and coefficients must be bit-exact (Clifford signs and the
FP64 per-gate update are evaluated in the same order on both sides);
magnetizations agree to 1e-10 absolute (only the order of the final sum
differs)."""
import math
import random

import numpy as np
import pytest

from paritylib import assert_bit_exact, gpu_canonical, oracle_canonical
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


def run_both(orqa, oracle_mod, n, layers, observable, steps, delta, capacity=1 << 20,
             check_sets=True):
    ctx = orqa.Context(n, capacity)
    ctx.set_labels(observable)
    op = oracle_mod.Oracle(n)
    for lab, c in observable:
        op.add_label(lab, c)
    mg, mo = [], []
    for t in range(steps):
        for layer in layers:
            ctx.apply_layer(layer, delta)
            for g in layer:
                op.apply(g, delta)
            if check_sets:
                assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n),
                                 "step %d layer %s" % (t + 1, layer[0][0]))
        mg.append(ctx.expect())
        mo.append(op.expect_zero())
    assert np.max(np.abs(np.array(mg) - np.array(mo))) < M_TOL
    return mg, mo, ctx, op


def test_chain12_config(orqa, oracle_mod):
    """12-qubit open chain, theta_h = pi/4, Z_6, 5 steps, delta = 0."""
    wl = W.workload("chain12")
    run_both(orqa, oracle_mod, wl["n"], wl["layers"], wl["observable"], wl["steps"], wl["delta"])


def test_heavyhex_config(orqa, oracle_mod):
    """127-qubit heavy-hex, theta_h = pi/4, Z_62, 5 steps, delta = 1e-4."""
    wl = W.workload("heavyhex")
    mg, _, ctx, _ = run_both(orqa, oracle_mod, wl["n"], wl["layers"], wl["observable"],
                             wl["steps"], wl["delta"])
    assert len(ctx) == 426052


def test_table_app_e_exact(orqa, oracle_mod):
    """App. E Table workload (theta_x = 0.9 pi, delta = 0) through t = 4,
    bit-exact, and the printed eps0 = 0 column."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, 0.9 * math.pi)
    mg, _, _, _ = run_both(orqa, oracle_mod, n, layers, [(W.z_label(n, [62]), 1.0)], 4, 0.0)
    table = [-0.95105651629515, 0.90450849718747, -0.9423841865631, 0.97436799430396]
    assert np.max(np.abs(np.array(mg) - np.array(table))) < 1e-13


@pytest.mark.parametrize("steps", [5])
def test_relative_truncation_table_column(orqa, oracle_mod, steps):
    """Relative truncation (Eq. truncation1, ORQA_FLAG_RELATIVE): the App. E
    Table workload at eps0 = 1e-5, bit-exact against the oracle after every
    layer, and the printed eps0 = 1e-5 column."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, 0.9 * math.pi)
    ctx = orqa.Context(n, 1 << 18, relative=True)
    ctx.set_labels([(W.z_label(n, [62]), 1.0)])
    op = oracle_mod.Oracle(n)
    op.add_label(W.z_label(n, [62]), 1.0)
    mg = []
    for t in range(steps):
        for layer in layers:
            ctx.apply_layer(layer, 1e-5)
            for g in layer:
                op.apply_rel(g, 1e-5)
            assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n), "rel step %d" % (t + 1))
        mg.append(ctx.expect())
    table = [-0.95105651629515, 0.90450849718747, -0.9423841865631, 0.97438562148434, -0.95311531321393]
    assert np.max(np.abs(np.array(mg) - np.array(table[:steps]))) < 1e-13


def test_relative_truncation_random(orqa, oracle_mod):
    """Relative truncation on a random 40-qubit operator and layers."""
    n = 40
    rng = random.Random(77)
    labels = _random_labels(rng, n, 80)
    terms = [(lab, rng.uniform(-1, 1)) for lab in labels]
    ctx = orqa.Context(n, 1 << 20, relative=True)
    ctx.set_labels(terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    for step in range(3):
        edges = set()
        while len(edges) < 50:
            a, b = rng.sample(range(n), 2)
            edges.add((a, b))
        zz = [("rzz", a, b, -math.pi / 2) for a, b in edges]
        qs = sorted(rng.sample(range(n), 6))
        xx = [("rx", q, None, rng.choice([0.3, 0.9, 2.0])) for q in qs]
        for layer in (zz, xx):
            ctx.apply_layer(layer, 1e-3)
            for g in layer:
                op.apply_rel(g, 1e-3)
            assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n), "rel random %d" % step)
    ctx.merge_truncate(0.05)
    keys_before = len(op)
    # relative merge_truncate: drop |c| <= 0.05 max|c| of the merged set
    mx = op.max_abs()
    op.truncate(0.0)
    ref = oracle_mod.Oracle(n)
    for k, v in op.as_dict().items():
        if abs(v) > 0.05 * mx:
            ref.add(k, v)
    assert 0 < len(ref) < keys_before
    assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(ref, n), "relative merge_truncate")


@pytest.mark.parametrize("delta", [1e-4, 1e-5])
def test_fp32_precision_form(orqa, oracle_mod, delta):
    """ORQA_FLAG_FP32 on the 127-qubit heavy hex (Z_62, theta = pi/4, 5
    steps): coefficients in FP32, two-member pair updates by the compensated
    Dot2 scheme, cos and sin as float pairs hi + lo, FP64 expectation sum.
    The magnetization must stay within 1e-6 of the FP64 oracle: each
    coefficient sees a few hundred FP32 roundings (2^-24 relative) through
    5 steps."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, math.pi / 4)
    ctx = orqa.Context(n, 1 << 23, fp32=True)
    ctx.set_labels([(W.z_label(n, [62]), 1.0)])
    mg = []
    for _ in range(5):
        for layer in layers:
            ctx.apply_layer(layer, delta)
        mg.append(ctx.expect())
    mo, op = oracle_mod.run_layers(n, [(W.z_label(n, [62]), 1.0)], layers, 5, delta)
    err = np.max(np.abs(np.array(mg) - np.array(mo)))
    assert err < 1e-6, err
    # the string set may differ only where a coefficient sits at the threshold
    assert abs(len(ctx) - len(op)) <= 1e-4 * len(op)


def test_table_app_e_t5(orqa):
    """t = 5 of the Table (2.1e6 strings): GPU alone against the printed
    eps0 = 0 value and the state vector value."""
    n, edges = W.heavy_hex_eagle()
    ctx = orqa.Context(n, 1 << 23)
    ctx.set_labels([(W.z_label(n, [62]), 1.0)])
    for _ in range(5):
        for layer in W.kicked_ising_layers(n, edges, 0.9 * math.pi):
            ctx.apply_layer(layer, 0.0)
    m = ctx.expect()
    assert abs(m - (-0.95315824248965)) < 1e-13
    assert abs(m - (-0.95315824248959)) < 1e-12
    assert len(ctx) == 2146564


@pytest.mark.parametrize("theta", [0.0, math.pi / 2])
def test_clifford_points(orqa, theta):
    n, edges = W.heavy_hex_eagle()
    ctx = orqa.Context(n, 1024)
    ctx.set_labels([(W.z_label(n, [62]), 1.0)])
    for t in range(5):
        for layer in W.kicked_ising_layers(n, edges, theta):
            ctx.apply_layer(layer, 0.0)
        assert len(ctx) == 1
        _, _, c = ctx.export()
        assert abs(c[0]) == 1.0
        m = ctx.expect()
        assert m == (1.0 if theta == 0.0 else m) and m in (-1.0, 0.0, 1.0)


def _random_labels(rng, n, k, alphabet="IXYZ"):
    return list({"".join(rng.choice(alphabet) for _ in range(n)) for _ in range(k)})


@pytest.mark.parametrize("n,seed", [(10, 1), (40, 2), (70, 3), (127, 4)])
def test_random_operators_and_layers(orqa, oracle_mod, n, seed):
    """Random Pauli sums, random edge sets with all four Clifford ZZ angles,
    X layers on random ascending qubit subsets with per-gate angles,
    thresholds including 0; sizes span several warps and a ragged tail."""
    rng = random.Random(0x2506 + seed)
    labels = _random_labels(rng, n, 60 + seed)
    terms = [(lab, rng.uniform(-1, 1)) for lab in labels]
    ctx = orqa.Context(n, 1 << 22)
    ctx.set_labels(terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n), "set")
    for step in range(3):
        edges = set()
        while len(edges) < min(2 * n, 60):
            a, b = rng.sample(range(n), 2)
            edges.add((a, b))
        zz = [("rzz", a, b, rng.choice([-math.pi / 2, math.pi / 2, math.pi, 0.0])) for a, b in edges]
        qs = sorted(rng.sample(range(n), rng.randint(1, min(n, 7))))
        xx = [("rx", q, None, rng.choice([0.3, -0.7, math.pi / 4, math.pi / 2, 2.2])) for q in qs]
        delta = [0.0, 1e-4, 1e-3][step]
        for layer in (zz, xx):
            ctx.apply_layer(layer, delta)
            for g in layer:
                op.apply(g, delta)
            assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n),
                             "n=%d step %d %s" % (n, step, layer[0][0]))
        assert abs(ctx.expect() - op.expect_zero()) < M_TOL


def test_small_coefficients_entering_a_layer(orqa, oracle_mod):
    """Strings below delta before an X layer: the truncation after the
    layer's first gate removes them unless that gate acts on them first."""
    n = 6
    terms = [("ZIIIII", 1e-5), ("IZIIII", 1e-5), ("YZIIII", 0.5), ("ZZIIII", 0.5), ("IIZIII", 0.9)]
    ctx = orqa.Context(n, 4096)
    ctx.set_labels(terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    layer = [("rx", q, None, 0.4) for q in range(n)]
    ctx.apply_layer(layer, 1e-3)
    for g in layer:
        op.apply(g, 1e-3)
    assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n), "small")


def test_merge_truncate_and_duplicates(orqa, oracle_mod):
    n = 20
    rng = random.Random(11)
    labels = _random_labels(rng, n, 500)
    # dyadic values of small exponent range: every sum is exact in any order
    terms = [(rng.choice(labels), rng.choice([0.25, -0.5, 1.0, 2.0 ** -13])) for _ in range(1500)]
    ctx = orqa.Context(n, 1 << 16)
    ctx.set_labels(terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    op.truncate(0.0)
    assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n), "merge")
    ctx.merge_truncate(1e-3)
    op.truncate(1e-3)
    assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n), "truncate")
    # the merged operator is the committed one for the device-side counts of
    # the next layers and of the expectation
    assert abs(ctx.expect() - op.expect_zero()) < M_TOL
    for layer in ([("rzz", 3, 7, -math.pi / 2), ("rzz", 1, 12, -math.pi / 2)],
                  [("rx", q, None, 0.7) for q in (2, 5, 9, 13)]):
        ctx.apply_layer(layer, 1e-3)
        for g in layer:
            op.apply(g, 1e-3)
        assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n), "layer after merge")
    assert abs(ctx.expect() - op.expect_zero()) < M_TOL


def test_empty_operator(orqa):
    n, edges = W.heavy_hex_eagle()
    ctx = orqa.Context(n, 64)
    ctx.set_operator(np.zeros((0, 2), np.uint64), np.zeros((0, 2), np.uint64), np.zeros(0))
    for layer in W.kicked_ising_layers(n, edges, 0.3):
        assert ctx.apply_layer(layer, 1e-4) == 0
    assert ctx.expect() == 0.0
    assert ctx.merge_truncate(0.1) == 0


def test_capacity_error_keeps_operator(orqa):
    """The X layer of step 5 grows 2582 strings to 426052; with capacity
    10000 it must fail with ECAPACITY and leave the operator untouched."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, math.pi / 4)
    ctx = orqa.Context(n, 10000)
    ctx.set_labels([(W.z_label(n, [62]), 1.0)])
    for _ in range(4):
        for layer in layers:
            ctx.apply_layer(layer, 1e-4)
    ctx.apply_layer(layers[0], 1e-4)
    mid = gpu_canonical(ctx, n)
    assert len(mid[1]) == 2582
    with pytest.raises(orqa.OrqaError) as ei:
        ctx.apply_layer(layers[1], 1e-4)
    assert ei.value.status == orqa.ORQA_ECAPACITY
    assert_bit_exact(gpu_canonical(ctx, n), mid, "after failed layer")


def test_invalid_layers_rejected(orqa):
    ctx = orqa.Context(8, 64)
    ctx.set_labels([("ZIIIIIII", 1.0)])
    with pytest.raises(orqa.OrqaError) as ei:
        ctx.apply_layer([("rx", 3, None, 0.1), ("rx", 2, None, 0.1)], 0.0)
    assert ei.value.status == orqa.ORQA_EINVAL
    with pytest.raises(orqa.OrqaError) as ei:
        ctx.apply_layer([("rzz", 0, 1, 0.3)], 0.0)
    assert ei.value.status == orqa.ORQA_EINVAL
    with pytest.raises(orqa.OrqaError):
        ctx.apply_layer([("rx", 9, None, 0.1)], 0.0)
    with pytest.raises(orqa.OrqaError):
        ctx.apply_layer([("rzz", 0, 1, -math.pi / 2), ("rx", 2, None, 0.1)], 0.0)
    assert len(ctx) == 1
