"""Rotations about general Pauli strings (orqa_apply_pauli_rotation: Eq.
update_rule for any sigma_J) against the CPU oracle, element by element;
and the X-layer path against the same gates applied as general rotations."""
import math
import random

import numpy as np
import pytest

from oracle import index_from_label
from paritylib import assert_bit_exact, canonical, gpu_canonical, oracle_canonical, planes_to_codes
from paper_2506_13241_gb300 import workloads as W

pytestmark = pytest.mark.gpu

M_TOL = 1e-10
ANGLES = [0.3, -0.7, math.pi / 4, math.pi / 2, -math.pi / 2, math.pi, 2.2, 0.0]


@pytest.fixture(scope="module")
def orqa():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2506_13241_gb300 import build, orqa as binding
    build.build()
    return binding


def random_label(rng, n, support):
    s = ["I"] * n
    for q in rng.sample(range(n), support):
        s[q] = rng.choice("XYZ")
    return "".join(s)


@pytest.mark.parametrize("n,seed", [(5, 0), (10, 1), (64, 2), (70, 3), (127, 4)])
def test_general_rotations_match_oracle(orqa, oracle_mod, n, seed):
    """Random Pauli sums through random generators of weight 1..6 (X, Y, Z
    on random qubits) at generic and Clifford angles, with and without
    truncation: bit-exact after every gate."""
    rng = random.Random(0x5eed + seed)
    terms = [(random_label(rng, n, rng.randint(1, min(n, 8))), rng.uniform(-1, 1)) for _ in range(40 + seed)]
    ctx = orqa.Context(n, 1 << 20)
    ctx.set_labels(terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    for k in range(10):
        J = random_label(rng, n, rng.randint(1, min(n, 6)))
        theta = rng.choice(ANGLES)
        delta = [0.0, 1e-3][k % 2]
        ctx.apply_pauli_rotation(J, theta, delta)
        op.apply(("pauli", index_from_label(J), None, theta), delta)
        assert_bit_exact(gpu_canonical(ctx, n), oracle_canonical(op, n), "gate %d J=%s theta=%g" % (k, J, theta))
        assert abs(ctx.expect() - op.expect_zero()) < M_TOL


def test_x_layer_equals_general_rotations(orqa):
    """The kicked-Ising X layer (chunk passes) and the same X gates applied
    one by one as general rotations give the same operator, bit for bit
    (heavy-hex, Z_62, theta = pi/4, 2 steps, delta = 1e-4)."""
    wl = W.workload("heavyhex_t=2")
    n, delta = wl["n"], wl["delta"]
    zz, xx = wl["layers"]
    a = orqa.Context(n, 1 << 20)
    b = orqa.Context(n, 1 << 20)
    a.set_labels(wl["observable"])
    b.set_labels(wl["observable"])
    for _ in range(2):
        a.apply_layer(zz, delta)
        b.apply_layer(zz, delta)
        a.apply_layer(xx, delta)
        for _, q, _, th in xx:
            lab = ["I"] * n
            lab[q] = "X"
            b.apply_pauli_rotation("".join(lab), th, delta)
        assert_bit_exact(gpu_canonical(a, n), gpu_canonical(b, n))


def test_general_rotation_fp32(orqa, oracle_mod):
    n = 40
    rng = random.Random(77)
    terms = [(random_label(rng, n, rng.randint(1, 6)), rng.uniform(-1, 1)) for _ in range(50)]
    ctx = orqa.Context(n, 1 << 20, fp32=True)
    ctx.set_labels(terms)
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    for k in range(12):
        J = random_label(rng, n, rng.randint(1, 4))
        theta = rng.choice([0.3, -0.7, 1.1])
        ctx.apply_pauli_rotation(J, theta, 1e-4)
        op.apply(("pauli", index_from_label(J), None, theta), 1e-4)
        assert abs(ctx.expect() - op.expect_zero()) < 1e-6


def test_general_rotation_batched_and_relative(orqa, oracle_mod):
    """A batched context rotates every problem; a relative-truncation
    context truncates after the gate with eps0 * max|c|."""
    n = 12
    rng = random.Random(5)
    probs = [[(random_label(rng, n, rng.randint(1, 5)), rng.uniform(-1, 1)) for _ in range(6)] for _ in range(3)]
    ctx = orqa.Context(n, 1 << 16, problems=3)
    ctx.set_labels_batch(probs)
    ops = []
    for terms in probs:
        op = oracle_mod.Oracle(n)
        for lab, c in terms:
            op.add_label(lab, c)
        ops.append(op)
    rel = orqa.Context(n, 1 << 16, relative=True)
    rel.set_labels(probs[0])
    opr = oracle_mod.Oracle(n)
    for lab, c in probs[0]:
        opr.add_label(lab, c)
    for k in range(8):
        J = random_label(rng, n, rng.randint(1, 4))
        theta = rng.choice([0.3, -0.7, math.pi / 2])
        ctx.apply_pauli_rotation(J, theta, 1e-3)
        rel.apply_pauli_rotation(J, theta, 1e-2)
        for op in ops:
            op.apply(("pauli", index_from_label(J), None, theta), 1e-3)
        opr.apply_rel(("pauli", index_from_label(J), None, theta), 1e-2)
        x, z, c, p = ctx.export_batch()
        codes = planes_to_codes(x, z, n)
        for k2, op in enumerate(ops):
            assert_bit_exact(canonical(codes[p == k2], c[p == k2]), oracle_canonical(op, n), "problem %d" % k2)
        assert_bit_exact(gpu_canonical(rel, n), oracle_canonical(opr, n), "relative")


def test_general_rotation_errors(orqa):
    n = 70
    ctx = orqa.Context(n, 1 << 12)
    ctx.set_labels([("Z" + "I" * (n - 1), 1.0)])
    with pytest.raises(orqa.OrqaError) as e:
        ctx.apply_pauli_rotation("I" * n, 0.3)
    assert e.value.status == orqa.ORQA_EINVAL
    xj = np.zeros(2, dtype=np.uint64)
    zj = np.array([0, 1 << 10], dtype=np.uint64)  # qubit 74 >= n
    with pytest.raises(orqa.OrqaError) as e:
        orqa.orqa_apply_pauli_rotation(ctx.ctx, xj, zj, 0.3, 0.0)
    assert e.value.status == orqa.ORQA_EINVAL
    assert len(ctx) == 1
