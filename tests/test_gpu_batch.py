"""Batched contexts (several independent operators in one context) against
the CPU oracle run problem by problem, and against plain one-operator
contexts.  Per problem, string sets and FP64 coefficients are bit-exact;
expectations agree to 1e-10 (only the summation order differs)."""
import math

import numpy as np
import pytest

from paritylib import assert_bit_exact, canonical, oracle_canonical, planes_to_codes
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


def problem_sets(ctx, n, P):
    """Canonical (codes, coefficients) of every problem of a batched context."""
    x, z, c, p = ctx.export_batch()
    codes = planes_to_codes(x, z, n)
    return [canonical(codes[p == k], c[p == k]) for k in range(P)]


def run_batch(orqa, wl, steps, delta, fp32=False, capacity=1 << 22):
    n, P = wl["n"], len(wl["problems"])
    zz, xx = wl["layers"]
    theta = np.array([[wl["theta"][p]] * len(xx) for p in range(P)])
    ctx = orqa.Context(n, capacity, fp32=fp32, problems=P)
    ctx.set_labels_batch(wl["problems"])
    mags = []
    for _ in range(steps):
        ctx.apply_layer(zz, delta)
        ctx.apply_layer_batch(xx, theta, delta)
        mags.append(ctx.expect_batch())
    return ctx, np.array(mags)


def oracle_problem(oracle_mod, wl, p, steps, delta):
    n = wl["n"]
    layers = W.kicked_ising_layers(n, wl["edges"], wl["theta"][p])
    return oracle_mod.run_layers(n, wl["problems"][p], layers, steps, delta)


@pytest.mark.parametrize("steps,weights,n_theta", [(3, (1, 3, 5), 4), (1, (17,), 3)])
def test_batch_matches_oracle(orqa, oracle_mod, steps, weights, n_theta):
    """theta sweep over [0, pi/2] (Clifford ends included) x Z-strings around
    qubit 62, delta = 1e-4: each problem equals its own oracle run."""
    wl = W.sweep_workload(n_theta, steps, 1e-4, weights)
    ctx, mags = run_batch(orqa, wl, steps, 1e-4)
    P = len(wl["problems"])
    sets = problem_sets(ctx, wl["n"], P)
    sizes = ctx.problem_sizes()
    for p in range(P):
        mo, op = oracle_problem(oracle_mod, wl, p, steps, 1e-4)
        assert np.max(np.abs(mags[:, p] - np.array(mo))) < M_TOL, p
        assert_bit_exact(sets[p], oracle_canonical(op, wl["n"]), "problem %d" % p)
        assert sizes[p] == len(op)
    assert sizes.sum() == len(ctx)


def test_batch_equals_plain_contexts(orqa):
    """The theta x observable sweep's problem mix at reduced size (8 angles x weights 1, 3, 17,
    2 steps, delta = 1e-3): every problem of the batch equals the same
    problem run alone in a plain context."""
    wl = W.sweep_workload(8, 2, 1e-3)
    n, P = wl["n"], len(wl["problems"])
    ctx, mags = run_batch(orqa, wl, 2, 1e-3)
    sets = problem_sets(ctx, n, P)
    for p in range(P):
        solo = orqa.Context(n, 1 << 21)
        solo.set_labels(wl["problems"][p])
        layers = W.kicked_ising_layers(n, wl["edges"], wl["theta"][p])
        ms = []
        for _ in range(2):
            for layer in layers:
                solo.apply_layer(layer, 1e-3)
            ms.append(solo.expect())
        x, z, c = solo.export()
        assert_bit_exact(sets[p], canonical(planes_to_codes(x, z, n), c), "problem %d" % p)
        assert np.max(np.abs(mags[:, p] - np.array(ms))) < M_TOL


def test_batch_fp32(orqa, oracle_mod):
    """FP32 precision form of a batched sweep: |Delta M_t| < 1e-6 per problem
    against the FP64 oracle."""
    wl = W.sweep_workload(4, 3, 1e-4, (1, 3, 5))
    _, mags = run_batch(orqa, wl, 3, 1e-4, fp32=True)
    for p in range(len(wl["problems"])):
        mo, _ = oracle_problem(oracle_mod, wl, p, 3, 1e-4)
        assert np.max(np.abs(mags[:, p] - np.array(mo))) < 1e-6, p


def test_batch_problems_never_merge(orqa):
    """Equal strings of different problems stay separate; duplicates inside
    a problem are summed (dyadic values: exact)."""
    n = 127
    lab = W.z_label(n, [62])
    ctx = orqa.Context(n, 1 << 12, problems=3)
    x, z = orqa.strings_from_labels([lab, lab, lab, lab], n)
    ctx.set_operator_batch(x, z, np.array([1.0, 0.5, 0.25, -0.5]), np.array([0, 1, 0, 1]))
    assert list(ctx.problem_sizes()) == [1, 0, 0]
    assert list(ctx.expect_batch()) == [1.25, 0.0, 0.0]
    ctx.set_operator_batch(x, z, np.array([1.0, 0.5, 0.25, 0.125]), np.array([0, 1, 2, 1]))
    assert list(ctx.problem_sizes()) == [1, 1, 1]
    assert list(ctx.expect_batch()) == [1.0, 0.625, 0.25]


def test_batch_call_errors(orqa):
    n = 127
    ctx = orqa.Context(n, 1 << 12, problems=4)
    x, z = orqa.strings_from_labels([W.z_label(n, [62])], n)
    with pytest.raises(orqa.OrqaError) as e:
        ctx.set_operator(x, z, np.array([1.0]))
    assert e.value.status == orqa.ORQA_EINVAL
    with pytest.raises(orqa.OrqaError) as e:
        ctx.set_operator_batch(x, z, np.array([1.0]), np.array([4]))
    assert e.value.status == orqa.ORQA_EINVAL
    ctx.set_operator_batch(x, z, np.array([1.0]), np.array([3]))
    with pytest.raises(orqa.OrqaError) as e:
        ctx.expect()
    assert e.value.status == orqa.ORQA_ESTATE
    _, edges = W.heavy_hex_eagle()
    zz = [("rzz", a, b, -math.pi / 2) for a, b in edges[:4]]
    with pytest.raises(orqa.OrqaError) as e:
        ctx.apply_layer_batch(zz, np.zeros((4, 4)), 0.0)
    assert e.value.status == orqa.ORQA_EINVAL
    with pytest.raises(ValueError):
        ctx.apply_layer_batch([("rx", 62, None, 0.3)], np.zeros((4, 2)), 0.0)
    assert list(ctx.problem_sizes()) == [0, 0, 0, 1]
