"""orqa_export's canonical order (ascending 256-bit key: x words from the
highest to the lowest, then z words likewise; problem index first in
batched contexts), made on the device.  The expected rows are the oracle's
operator re-coded to x/z planes and sorted by numpy; coefficients must be
bit-exact in that order."""
import math

import numpy as np
import pytest

from paritylib import canonical_key_order, codes_to_planes, index_words_to_codes
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


def oracle_rows(op, n):
    keys, c = op.export()
    x, z = codes_to_planes(index_words_to_codes(keys, n), 1 if n <= 64 else 2)
    order = canonical_key_order(x, z)
    return x[order], z[order], c[order]


def assert_rows_equal(got, want):
    gx, gz, gc = got
    wx, wz, wc = want
    assert gx.shape == wx.shape
    assert np.array_equal(gx, wx) and np.array_equal(gz, wz)
    assert np.array_equal(gc.view(np.uint64), wc.view(np.uint64))


def assert_strictly_ascending(x, z):
    if len(x) < 2:
        return
    order = canonical_key_order(x, z)
    assert np.array_equal(order, np.arange(len(x)))
    key = np.concatenate([x[:, ::-1], z[:, ::-1]], axis=1)
    assert not np.any(np.all(key[1:] == key[:-1], axis=1))  # no duplicates


def test_export_order_heavyhex(orqa, oracle_mod):
    """Heavy-hex, theta = pi/4, 5 steps, delta = 1e-4 (426,052 strings over
    two-word planes): the export equals the oracle's set in canonical order."""
    wl = W.workload("heavyhex")
    n = wl["n"]
    ctx = orqa.Context(n, 1 << 20)
    ctx.set_labels(wl["observable"])
    mo, op = oracle_mod.run_layers(n, wl["observable"], wl["layers"], wl["steps"], wl["delta"])
    for _ in range(wl["steps"]):
        for layer in wl["layers"]:
            ctx.apply_layer(layer, wl["delta"])
    got = ctx.export()
    assert len(got[2]) == 426052
    assert_strictly_ascending(got[0], got[1])
    assert_rows_equal(got, oracle_rows(op, n))
    # the export does not disturb the operator
    assert abs(ctx.expect() - mo[-1]) < 1e-10
    assert_rows_equal(ctx.export(), got)


@pytest.mark.parametrize("n,seed", [(12, 1), (64, 2), (65, 3), (128, 4)])
def test_export_order_random(orqa, oracle_mod, n, seed):
    """Random Pauli sums (top qubits included) on one- and two-word planes."""
    rng = np.random.default_rng(seed)
    labels = {"".join(rng.choice(list("IXYZ"), n)) for _ in range(3000)}
    # strings that differ only in the highest qubit and only in z
    labels |= {"I" * (n - 1) + ch for ch in "XYZ"} | {"Z" + "I" * (n - 1)}
    terms = [(lab, float(rng.uniform(-1, 1))) for lab in sorted(labels)]
    ctx = orqa.Context(n, 1 << 14)
    ctx.set_labels(terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    got = ctx.export()
    assert_strictly_ascending(got[0], got[1])
    assert_rows_equal(got, oracle_rows(op, n))


def test_export_edge_cases(orqa):
    n = 127
    ctx = orqa.Context(n, 64)
    ctx.set_operator(np.zeros((0, 2), np.uint64), np.zeros((0, 2), np.uint64), np.zeros(0))
    assert len(ctx.export()[2]) == 0
    ctx.set_labels([("I" * 126 + "Y", -0.5)])
    x, z, c = ctx.export()
    assert c.tolist() == [-0.5] and x[0, 1] == 1 << 62 and z[0, 1] == 1 << 62
    # equal x, z differs only in one low bit: one varying digit
    ctx.set_labels([("ZI", 1.0), ("II", 2.0), ("XI", 3.0), ("YI", 4.0)])
    x, z, c = ctx.export()
    assert c.tolist() == [2.0, 1.0, 3.0, 4.0]


def test_export_batch_and_fp32(orqa):
    """Batched context: problem index first, then the key; FP32 coefficients
    widened to FP64 in the same order."""
    n = 40
    rng = np.random.default_rng(9)
    per = [[("".join(rng.choice(list("IXYZ"), n)), float(rng.uniform(-1, 1))) for _ in range(200)]
           for _ in range(3)]
    ctx = orqa.Context(n, 1 << 12, problems=3)
    ctx.set_labels_batch(per)
    x, z, c, p = ctx.export_batch()
    order = canonical_key_order(x, z, p)
    assert np.array_equal(order, np.arange(len(c)))
    assert np.array_equal(np.bincount(p, minlength=3), [len({lab for lab, _ in t}) for t in per])
    f = orqa.Context(n, 1 << 12, fp32=True)
    f.set_labels(per[0])
    xf, zf, cf = f.export()
    assert_strictly_ascending(xf, zf)
    want = {lab: np.float32(c) for lab, c in per[0]}
    assert len(cf) == len(want)
