"""The restructured X layer, as the CUDA path organises it, checked on the CPU
against the oracle's gate-by-gate run of Algorithm 1.

An X-rotation layer never changes z, and a gate on qubit q acts only on the
strings with z_q = 1, pairing P (sigma_z at q) with P xor X_q (sigma_y at q).
The layer is therefore applied in chunk passes: pass p takes, for every
string, the set bits of F = z & M of rank [5p, 5p + 5) (M: the layer's
qubits), groups the strings into units of equal z and equal x outside
those bits, and applies the chunk's gates level by level inside each unit
(slot = the chunk bits of x), truncating every result.  A string below
delta that the layer's first gate does not touch is removed by the
truncation after that gate (Algorithm 1 truncates the whole operator after
every gate).  Written here in plain Python (FP64, every product and sum
rounded once), this model must give the oracle's operator bit for bit: the
claim that the GPU's pass structure changes no arithmetic."""
import math
import random

import pytest

from paper_2506_13241_gb300 import workloads as W

CHUNK = 5


def _chunk_pass_layer(strings, gates, delta, cos_sin, planted=False, counts=None):
    """strings: {(x, z): c}; gates: [(q, theta)] on ascending qubits.
    planted: the sin terms of a two-member pair enter with swapped signs
    (the source-indexed sign of Algorithm 1 as printed).
    counts (a dict, optional) receives the pieces of the CUDA path's
    string-gate update count: the strings entering, the strings the entry
    split drops, and the sum over units and gates of the unit's population
    change at the gate times the number of the layer's gates above it."""
    M = 0
    rot = {}
    for q, theta in gates:
        M |= 1 << q
        rot[q] = cos_sin(theta)
    q1 = gates[0][0]
    above = {q: sum(1 for g, _ in gates if g > q) for q, _ in gates}
    kept = lambda v: v != 0.0 and abs(v) >= delta
    done, active = {}, {}
    split_dropped, upd_w = 0, 0
    for (x, z), c in strings.items():
        f = z & M
        if not (z >> q1) & 1 and not kept(c):
            split_dropped += 1
            continue                      # truncated after the first gate
        if f == 0:
            done[(x, z)] = c
        else:
            active[(x, z)] = c
    p = 0
    while active:
        units = {}
        for (x, z), c in active.items():
            bits = [q for q in range(z.bit_length()) if (z & M) >> q & 1]
            chunk = bits[CHUNK * p:CHUNK * p + CHUNK]
            idx, xb = 0, x
            for j, q in enumerate(chunk):
                if x >> q & 1:
                    idx |= 1 << j
                    xb &= ~(1 << q)
            unit = units.setdefault((z, xb), (chunk, len(bits) > CHUNK * (p + 1), {}))
            unit[2][idx] = c
        nxt = {}
        for (z, xb), (chunk, more, slots) in units.items():
            for j, q in enumerate(chunk):
                co, si = rot[q]
                bit = 1 << j
                new = {}
                for l in sorted({s & ~bit for s in slots}):
                    a, b = slots.get(l), slots.get(l | bit)   # sigma_z at q, sigma_y at q
                    if a is not None and b is not None and planted:
                        na, nb = co * a + si * b, co * b - si * a
                    elif a is not None and b is not None:
                        na, nb = co * a - si * b, co * b + si * a
                    elif a is not None:
                        na, nb = co * a, si * a
                    else:
                        na, nb = -(si * b), co * b
                    if kept(na):
                        new[l] = na
                    if kept(nb):
                        new[l | bit] = nb
                upd_w += (len(new) - len(slots)) * above[q]
                slots = new
            for l, v in slots.items():
                x = xb
                for j, q in enumerate(chunk):
                    if l >> j & 1:
                        x |= 1 << q
                (nxt if more else done)[(x, z)] = v
        active = nxt
        p += 1
    if counts is not None:
        counts.update(n_in=len(strings), split_dropped=split_dropped, upd_w=upd_w)
    return done


def _planes(oracle_mod, key, n):
    x = z = 0
    for q, a in enumerate(oracle_mod.codes_from_index(key, n)):
        if a in (1, 2):
            x |= 1 << q
        if a in (2, 3):
            z |= 1 << q
    return x, z


def _as_planes(oracle_mod, op, n):
    return {_planes(oracle_mod, k, n): c for k, c in op.as_dict().items()}


def _run(oracle_mod, n, terms, layers, delta, planted=False):
    """Applies the layers to the oracle (gate by gate) and to the model (ZZ
    layers through the oracle, X layers by chunk passes); compares after
    every X layer."""
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    for layer in layers:
        before = _as_planes(oracle_mod, op, n)
        for g in layer:
            op.apply(g, delta)
        if layer[0][0] != "rx":
            continue
        got = _chunk_pass_layer(before, [(g[1], g[3]) for g in layer], delta, oracle_mod.rotation_cos_sin,
                                planted)
        assert got == _as_planes(oracle_mod, op, n)
    return len(op)


def test_heavy_hex_layers_match_algorithm_1(oracle_mod):
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, math.pi / 4)
    size = _run(oracle_mod, n, [(W.z_label(n, [62]), 1.0)], layers * 4, 1e-4)
    assert size > 1000


@pytest.mark.parametrize("seed", range(6))
def test_random_operators_and_x_subsets(oracle_mod, seed):
    """Random Pauli sums (some terms below delta), random ascending X subsets
    with per-gate angles including Clifford ones, delta = 0 and 1e-3."""
    rng = random.Random(0x250613241 + seed)
    n = rng.choice([6, 12, 20])
    terms = []
    for _ in range(60):
        lab = "".join(rng.choice("IXYZ") for _ in range(n))
        terms.append((lab, rng.choice([rng.uniform(-1, 1), rng.uniform(-1e-3, 1e-3)])))
    angles = [0.3, -0.8, math.pi / 4, math.pi / 2, -math.pi / 2, math.pi, 2.2]
    layers = []
    for _ in range(4):
        qs = sorted(rng.sample(range(n), rng.randint(1, n)))
        layers.append([("rx", q, None, rng.choice(angles)) for q in qs])
    _run(oracle_mod, n, terms, layers, [0.0, 1e-3][seed % 2])


def test_small_strings_entering_a_layer(oracle_mod):
    """Strings below delta that the layer's first gate (qubit 1) does not
    touch are gone before any later gate: one with no qubit of the layer in
    F, one whose first layer qubit is 3 and whose sigma_y partner there is
    large (Algorithm 1 meets the partner alone at gate 3), and one with x
    bits only."""
    n = 6
    terms = [("ZIIIII", 1e-5), ("IIIZIZ", 1e-5), ("IIIYIZ", 0.5), ("XIIIIX", -2e-5),
             ("IZIIII", 1e-5), ("IZIZII", 0.9), ("IYIIZI", -0.3)]
    layer = [("rx", q, None, th) for q, th in ((1, 0.4), (3, -1.1), (4, math.pi / 4))]
    assert _run(oracle_mod, n, terms, [layer, layer], 1e-3) > 4


@pytest.mark.parametrize("seed", range(4))
def test_update_count_formula(oracle_mod, seed):
    """The string-gate update count of an X layer -- the sum over its gates
    of |O| before the gate, read off the oracle gate by gate -- equals
    n_g n_in - (strings the entry split drops) (n_g - 1) + the weighted sum
    of the units' population changes that the unit kernel accumulates."""
    rng = random.Random(0x13241 + seed)
    n = rng.choice([8, 12, 20])
    terms = [("".join(rng.choice("IXYZ") for _ in range(n)), rng.choice([rng.uniform(-1, 1), rng.uniform(-1e-3, 1e-3)]))
             for _ in range(80)]
    op = oracle_mod.Oracle(n)
    for lab, c in terms:
        op.add_label(lab, c)
    delta = [0.0, 1e-3][seed % 2]
    for _ in range(3):
        qs = sorted(rng.sample(range(n), rng.randint(2, n)))
        layer = [("rx", q, None, rng.choice([0.3, -0.8, math.pi / 4, 1.3])) for q in qs]
        before = _as_planes(oracle_mod, op, n)
        expected = 0
        for g in layer:
            expected += len(op)
            op.apply(g, delta)
        counts = {}
        got = _chunk_pass_layer(before, [(g[1], g[3]) for g in layer], delta, oracle_mod.rotation_cos_sin,
                                counts=counts)
        assert got == _as_planes(oracle_mod, op, n)
        ng = len(layer)
        formula = ng * counts["n_in"] - counts["split_dropped"] * (ng - 1) + counts["upd_w"]
        assert formula == expected, (formula, expected, counts)


def test_planted_sign_is_caught(oracle_mod):
    """The same comparison sees the two-member update with swapped signs."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, math.pi / 4)
    with pytest.raises(AssertionError):
        _run(oracle_mod, n, [(W.z_label(n, [62]), 1.0)], layers * 4, 1e-4, planted=True)
