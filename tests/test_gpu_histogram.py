"""Pauli-string density D_t(x) (App. D, orqa_histogram) against the oracle's
histogram of its own operator: identical counts (the FP64 coefficients are
bit-exact, and both sides form the bin edges by the same formula)."""
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


def test_histogram_heavyhex(orqa, oracle_mod):
    wl = W.workload("heavyhex")
    n = wl["n"]
    ctx = orqa.Context(n, 1 << 21)
    ctx.set_labels(wl["observable"])
    mo, op = oracle_mod.run_layers(n, wl["observable"], wl["layers"], 5, wl["delta"])
    for _ in range(5):
        for layer in wl["layers"]:
            ctx.apply_layer(layer, wl["delta"])
    _, c = op.export()
    for n_bins, lo in [(40, -8.0), (7, -3.5), (1, -1.0), (256, -12.0)]:
        got, m = ctx.histogram(n_bins, lo)
        want, mw = oracle_mod.histogram(c, n_bins, lo)
        assert m == mw
        assert (got == want).all(), (n_bins, lo)
        assert got.sum() == len(ctx)


def test_histogram_relative_truncation_cutoff(orqa, oracle_mod):
    """Fig. 5 setting at reduced size (theta_x = 0.1 pi, relative
    truncation eps0 = 1e-4, 3 steps): no string below eps0 * max, and the
    counts equal the oracle's."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, 0.1 * math.pi)
    obs = [(W.z_label(n, [62]), 1.0)]
    ctx = orqa.Context(n, 1 << 21, relative=True)
    ctx.set_labels(obs)
    for _ in range(3):
        for layer in layers:
            ctx.apply_layer(layer, 1e-4)
    _, op = oracle_mod.run_layers(n, obs, layers, 3, 1e-4, mode="rel")
    _, c = op.export()
    got, m = ctx.histogram(24, -6.0)
    want, _ = oracle_mod.histogram(c, 24, -6.0)
    assert (got == want).all()
    # bins entirely below eps0 = 1e-4 (edges 1e-6 .. 1e-4: bins 0..7) are empty
    assert got[:, :8].sum() == 0 and got[:, 24].sum() == 0


def test_histogram_empty_and_bad_args(orqa):
    ctx = orqa.Context(12, 1024)
    counts, m = ctx.histogram(4, -2.0)
    assert counts.sum() == 0 and m == 0.0
    for bad in [(0, -2.0), (300, -2.0), (4, 0.0), (4, 1.0)]:
        with pytest.raises(orqa.OrqaError) as e:
            ctx.histogram(*bad)
        assert e.value.status == orqa.ORQA_EINVAL
