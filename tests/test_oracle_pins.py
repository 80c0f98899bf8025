"""Pins of the CPU oracle against facts fixed outside it: Pauli matrix
products, dense-matrix Heisenberg evolution, dense state vectors, closed
forms, the paper's printed Table (App. E), Clifford points and invariants.
A last group plants plausible mistakes in the oracle and checks that some
pin catches each one."""
import math
import os
import random

import numpy as np
import pytest

import bruteforce as bf
from paper_2506_13241_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table_app_e.txt")


def labels_dict(op, n):
    """Oracle contents as {label: coefficient}."""
    import oracle
    out = {}
    for key, c in op.as_dict().items():
        codes = oracle.codes_from_index(key, n)
        out["".join("IXYZ"[a] for a in codes)] = c
    return out


def random_label(rng, n, allow_identity=True):
    while True:
        lab = "".join(rng.choice("IXYZ") for _ in range(n))
        if allow_identity or set(lab) != {"I"}:
            return lab


# --------------------------------------------------------------------------
# Pauli algebra: sigma_I sigma_J = i^B(I,J) sigma_{I xor J}  (Eq. orqaproduct)
# --------------------------------------------------------------------------

def test_phase_exponent_single_site(oracle_mod):
    for a in "IXYZ":
        for b in "IXYZ":
            I = oracle_mod.index_from_label(a)
            J = oracle_mod.index_from_label(b)
            B = oracle_mod.phase_exponent(I, J, 1)
            K = tuple(x ^ y for x, y in zip(I, J))
            lab = "IXYZ"[oracle_mod.codes_from_index(K, 1)[0]]
            lhs = bf.PAULI[a] @ bf.PAULI[b]
            rhs = (1j ** B) * bf.PAULI[lab]
            assert np.allclose(lhs, rhs), (a, b, B)


def test_phase_exponent_multi_site(oracle_mod):
    rng = random.Random(0x250613241)
    n = 4
    for _ in range(60):
        a = random_label(rng, n)
        b = random_label(rng, n)
        I = oracle_mod.index_from_label(a)
        J = oracle_mod.index_from_label(b)
        B = oracle_mod.phase_exponent(I, J, n)
        K = tuple(x ^ y for x, y in zip(I, J))
        lab = "".join("IXYZ"[c] for c in oracle_mod.codes_from_index(K, n))
        assert np.allclose(bf.pauli_matrix(a) @ bf.pauli_matrix(b),
                           (1j ** B) * bf.pauli_matrix(lab))


# --------------------------------------------------------------------------
# One gate: Eq. (update_rule) against U^dagger O U with dense matrices
# --------------------------------------------------------------------------

def _single_gate_case(oracle_mod, n, terms, J_label, theta, lib_path=None):
    op = oracle_mod.Oracle(n, lib_path)
    dense = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    for lab, c in terms:
        op.add_label(lab, c)
        dense += c * bf.pauli_matrix(lab)
    gate = ("pauli", oracle_mod.index_from_label(J_label), None, theta)
    op.rotate_only(gate)
    got = labels_dict(op, n)
    ref = bf.pauli_decompose(bf.heisenberg(dense, [("label", J_label, None, theta)], n), n, 1e-14)
    return got, ref


def _assert_same_pauli_sum(got, ref, tol=1e-13):
    keys = set(got) | set(ref)
    for k in keys:
        g = got.get(k, 0.0)
        r = ref.get(k, 0.0)
        assert abs(np.imag(r)) < tol, (k, r)
        assert abs(g - np.real(r)) < tol, (k, g, r)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_single_gate_matches_dense(oracle_mod, n):
    rng = random.Random(1000 + n)
    thetas = [0.0, math.pi / 2, -math.pi / 2, math.pi, 0.3, -1.1, 2.5, 0.9 * math.pi]
    for trial in range(40):
        terms = [(random_label(rng, n), rng.uniform(-1, 1)) for _ in range(rng.randint(1, 5))]
        J = random_label(rng, n, allow_identity=False)
        theta = thetas[trial % len(thetas)] if trial < 16 else rng.uniform(-math.pi, math.pi)
        got, ref = _single_gate_case(oracle_mod, n, terms, J, theta)
        _assert_same_pauli_sum(got, ref)


def test_rx_rule_closed_form(oracle_mod):
    """U^dagger Z U = cos Z + sin Y and U^dagger Y U = cos Y - sin Z for
    U = exp(-i theta X / 2); X is left unchanged."""
    th = 0.41
    for src, expect in (("Z", {"Z": math.cos(th), "Y": math.sin(th)}),
                        ("Y", {"Y": math.cos(th), "Z": -math.sin(th)}),
                        ("X", {"X": 1.0})):
        op = oracle_mod.Oracle(1)
        op.add_label(src, 1.0)
        op.rotate_only(("rx", 0, None, th))
        got = labels_dict(op, 1)
        assert set(got) == set(expect)
        for k in expect:
            assert got[k] == pytest.approx(expect[k], abs=1e-15)


def test_rzz_clifford_rule(oracle_mod):
    """exp(-i theta/2 ZZ) with theta = -pi/2: X_1 -> Y_1 Z_2, Y_1 -> -X_1 Z_2,
    and the image is a single string (exact Clifford angle)."""
    for src, (dst, sign) in (("XI", ("YZ", 1.0)), ("YI", ("XZ", -1.0)),
                             ("IX", ("ZY", 1.0)), ("ZI", ("ZI", 1.0))):
        op = oracle_mod.Oracle(2)
        op.add_label(src, 1.0)
        op.apply(("rzz", 0, 1, -math.pi / 2), 0.0)
        assert labels_dict(op, 2) == {dst: sign}


# --------------------------------------------------------------------------
# Whole circuits against dense Heisenberg evolution and state vectors
# --------------------------------------------------------------------------

def test_kicked_ising_chain5_dense_heisenberg(oracle_mod):
    n = 5
    edges = W.chain_edges(n)
    layers = W.kicked_ising_layers(n, edges, 0.37)
    obs = W.z_label(n, [2])
    m, op = oracle_mod.run_layers(n, [(obs, 1.0)], layers, 3, 0.0)
    gates = [g for _ in range(3) for layer in layers for g in layer]
    dense = bf.heisenberg(bf.pauli_matrix(obs), gates, n)
    ref = bf.pauli_decompose(dense, n, 1e-14)
    _assert_same_pauli_sum(labels_dict(op, n), ref, 1e-12)


@pytest.mark.parametrize("theta", [math.pi / 4, 0.3])
def test_chain12_statevector(oracle_mod, theta):
    n = 12
    edges = W.chain_edges(n)
    layers = W.kicked_ising_layers(n, edges, theta)
    m, _ = oracle_mod.run_layers(n, [(W.z_label(n, [6]), 1.0)], layers, 5, 0.0)
    sv = bf.statevector_magnetization(n, layers, 5, 6)
    assert np.max(np.abs(np.array(m) - np.array(sv))) < 1e-12


def test_closed_forms(oracle_mod):
    """Single-Z observable: M_1 = cos(theta).  Odd-degree site (heavy-hex
    qubit 62, degree 3): M_2 = cos^2(theta).  Interior chain site (degree
    2): M_2 = cos^2(theta) (1 + sin^2(theta))."""
    n, edges = W.heavy_hex_eagle()
    for th in (0.3, 0.9 * math.pi, math.pi / 4):
        m, _ = oracle_mod.run_layers(n, [(W.z_label(n, [62]), 1.0)],
                                     W.kicked_ising_layers(n, edges, th), 2, 0.0)
        assert m[0] == pytest.approx(math.cos(th), abs=1e-14)
        assert m[1] == pytest.approx(math.cos(th) ** 2, abs=1e-14)
    nc = 12
    for th in (0.3, math.pi / 4):
        m, _ = oracle_mod.run_layers(nc, [(W.z_label(nc, [6]), 1.0)],
                                     W.kicked_ising_layers(nc, W.chain_edges(nc), th), 2, 0.0)
        assert m[1] == pytest.approx(math.cos(th) ** 2 * (1 + math.sin(th) ** 2), abs=1e-14)


def _table():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t, sv, e0, e5 = line.split()
                rows.append((int(t), float(sv), float(e0), float(e5)))
    return rows


@pytest.mark.slow
def test_table_app_e_exact_column(oracle_mod):
    """eps0 = 0 column of the App. E Table (t = 1..5), heavy-hex, theta_x =
    0.9 pi, sigma_z^62.  Printed to 13-14 decimals; the paper's own spread
    against the state vector is 6e-14."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, 0.9 * math.pi)
    m, _ = oracle_mod.run_layers(n, [(W.z_label(n, [62]), 1.0)], layers, 5, 0.0)
    for (t, sv, e0, _), got in zip(_table(), m):
        assert abs(got - e0) < 1e-13, (t, got, e0)
        assert abs(got - sv) < 1e-12, (t, got, sv)


def test_table_app_e_relative_truncation_column(oracle_mod):
    """eps0 = 1e-5 column of the App. E Table: relative truncation
    |O_I| <= eps0 max|O| (Eq. truncation1) after every gate, max taken over
    the operator after that gate's updates."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, 0.9 * math.pi)
    m, _ = oracle_mod.run_layers(n, [(W.z_label(n, [62]), 1.0)], layers, 5, 1e-5, mode="rel")
    for (t, _, _, e5), got in zip(_table(), m):
        assert abs(got - e5) < 1e-13, (t, got, e5)


# --------------------------------------------------------------------------
# Clifford points and invariants
# --------------------------------------------------------------------------

def test_clifford_points(oracle_mod):
    """theta_x = 0: O stays sigma_z^62, M_t = 1.  theta_x = pi/2 (dual
    unitary): O stays one string with coefficient +-1."""
    n, edges = W.heavy_hex_eagle()
    for th in (0.0, math.pi / 2):
        sizes, coefs = [], []

        def cb(t, op):
            sizes.append(len(op))
            coefs.append(list(op.as_dict().values()))
        m, _ = oracle_mod.run_layers(n, [(W.z_label(n, [62]), 1.0)],
                                     W.kicked_ising_layers(n, edges, th), 5, 0.0, on_step=cb)
        assert sizes == [1] * 5
        assert all(abs(abs(c[0]) - 1.0) == 0.0 for c in coefs)
        if th == 0.0:
            assert m == [1.0] * 5
        else:
            assert all(v in (-1.0, 0.0, 1.0) for v in m)


def test_norm_conserved_without_truncation(oracle_mod):
    n = 12
    norms = []
    oracle_mod.run_layers(n, [(W.z_label(n, [6]), 1.0)],
                          W.kicked_ising_layers(n, W.chain_edges(n), math.pi / 4), 5, 0.0,
                          on_step=lambda t, op: norms.append(op.norm2()))
    assert np.max(np.abs(np.array(norms) - 1.0)) < 1e-12


def test_truncation_drops_exactly_small_terms(oracle_mod):
    """Gate by gate: truncation removes exactly the entries with c == 0 or
    |c| < delta, and the norm decrease equals the squares of those entries."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, math.pi / 4)
    delta = 1e-3
    op = oracle_mod.Oracle(n)
    op.add_label(W.z_label(n, [62]), 1.0)
    for _ in range(4):
        for layer in layers:
            for g in layer:
                op.rotate_only(g)
                before = op.as_dict()
                op.truncate(delta)
                after = op.as_dict()
                dropped = {k: v for k, v in before.items() if k not in after}
                assert all(v == 0.0 or abs(v) < delta for v in dropped.values())
                assert all(v != 0.0 and abs(v) >= delta for v in after.values())
                assert all(after[k] == before[k] for k in after)
                lost = sum(v * v for v in before.values()) - sum(v * v for v in after.values())
                assert lost == pytest.approx(sum(v * v for v in dropped.values()), abs=1e-15)


def _relative_hand_cases(oracle_mod, lib_path=None):
    """Hand examples of the relative rule of Eq. (truncation1): after a gate,
    drop c == 0 and |c| <= eps0 * max|c|, the max taken over the operator
    after that gate's updates.  Returns the three resulting operators as
    {label: coefficient}."""
    theta = math.atan2(0.8, 0.6)  # cos = 0.6, sin = 0.8 (to rounding)
    rx = ("rx", 0, None, theta)
    # (a) Z + 0.09 X under Rx: the max falls from 1 to 0.8, so with eps0 = 0.1
    # the threshold is 0.08 after the gate (X kept) but 0.1 before it
    a = oracle_mod.Oracle(1, lib_path)
    a.add_label("Z", 1.0)
    a.add_label("X", 0.09)
    a.apply_rel(rx, 0.1)
    # (b) a tie: Z + 0.5 I under a gate that commutes with both; eps0 = 0.5
    # puts the threshold exactly at 0.5, and |c| <= threshold is dropped
    b = oracle_mod.Oracle(1, lib_path)
    b.add_label("Z", 1.0)
    b.add_label("I", 0.5)
    b.apply_rel(("pauli", oracle_mod.index_from_label("Z"), None, 0.7), 0.5)
    # (c) Rx(pi/2) on Z: cos = 0 exactly, so Z is left with an exact zero
    # (removed) and Y carries the whole coefficient
    c = oracle_mod.Oracle(1, lib_path)
    c.add_label("Z", 1.0)
    c.apply_rel(("rx", 0, None, math.pi / 2), 1e-3)
    return [labels_dict(op, 1) for op in (a, b, c)]


def test_relative_truncation_hand_examples(oracle_mod):
    a, b, c = _relative_hand_cases(oracle_mod)
    assert set(a) == {"Z", "Y", "X"}
    assert a["X"] == 0.09
    assert abs(a["Z"] - 0.6) < 1e-15 and abs(abs(a["Y"]) - 0.8) < 1e-15
    assert b == {"Z": 1.0}
    assert set(c) == {"Y"} and abs(c["Y"]) == 1.0


def test_support_stays_in_light_cone(oracle_mod):
    n, edges = W.heavy_hex_eagle()
    _, dist = W.bfs_order(n, edges, 62)

    def cb(t, op):
        for key in op.as_dict():
            codes = oracle_mod.codes_from_index(key, n)
            assert max(dist[q] for q, a in enumerate(codes) if a) <= t - 1

    oracle_mod.run_layers(n, [(W.z_label(n, [62]), 1.0)],
                          W.kicked_ising_layers(n, edges, math.pi / 4), 4, 1e-4, on_step=cb)


def test_rzz_layer_order_independent(oracle_mod):
    """All ZZ rotations commute, so the edge order of U_zz does not change
    the result (bit for bit: each Clifford gate maps a string to one
    string with an exact sign)."""
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, 0.3)
    base = None
    for seed in range(3):
        zz = list(layers[0])
        random.Random(seed).shuffle(zz)
        _, op = oracle_mod.run_layers(n, [(W.z_label(n, [62]), 1.0)], [zz, layers[1]], 3, 1e-6)
        d = op.as_dict()
        if base is None:
            base = d
        assert d == base


def test_colouring_and_lattice():
    n, edges = W.heavy_hex_eagle()
    assert n == 127 and len(edges) == 144
    adj = W.adjacency(n, edges)
    assert max(len(a) for a in adj) == 3 and adj[62] == [61, 63, 72]
    classes = W.edge_colouring(n, edges)
    assert sorted(len(c) for c in classes) and sum(len(c) for c in classes) == 144
    for cls in classes:
        touched = [q for e in cls for q in e]
        assert len(touched) == len(set(touched))
    _, dist = W.bfs_order(n, edges, 62)
    # the causal cone of qubit 62 holds 31 qubits at radius 5 (App. E)
    assert sum(1 for d in dist if 0 <= d <= 5) == 31


# --------------------------------------------------------------------------
# Planted mistakes: each one must make some pin above fail.
# --------------------------------------------------------------------------

def _pin_phase(oracle_mod, path):
    """sigma_a sigma_b = i^B sigma_{a xor b} on one site."""
    for a in "XYZ":
        for b in "XYZ":
            I = oracle_mod.index_from_label(a)
            J = oracle_mod.index_from_label(b)
            B = oracle_mod.phase_exponent(I, J, 1, lib_path=path)
            K = tuple(x ^ y for x, y in zip(I, J))
            lab = "IXYZ"[oracle_mod.codes_from_index(K, 1)[0]]
            if not np.allclose(bf.PAULI[a] @ bf.PAULI[b], (1j ** B) * bf.PAULI[lab]):
                return False
    return True


def _pin_dense(oracle_mod, path):
    """One gate against dense matrices, generic and Clifford angles."""
    rng = random.Random(7)
    for trial in range(24):
        terms = [(random_label(rng, 2), rng.uniform(-1, 1)) for _ in range(3)]
        J = random_label(rng, 2, allow_identity=False)
        theta = [0.3 + trial, math.pi / 2, -math.pi / 2, math.pi][trial % 4]
        got, ref = _single_gate_case(oracle_mod, 2, terms, J, theta, path)
        try:
            _assert_same_pauli_sum(got, ref)
        except AssertionError:
            return False
    return True


def _pin_statevector(oracle_mod, path):
    """The 12-qubit chain against the state vector."""
    n = 12
    layers = W.kicked_ising_layers(n, W.chain_edges(n), math.pi / 4)
    m, _ = oracle_mod.run_layers(n, [(W.z_label(n, [6]), 1.0)], layers, 3, 0.0, lib_path=path)
    return np.max(np.abs(np.array(m) - np.array(bf.statevector_magnetization(n, layers, 3, 6)))) <= 1e-12


def _pin_clifford(oracle_mod, path):
    """theta = pi/2 on the heavy hex keeps one string."""
    nh, edges = W.heavy_hex_eagle()
    _, op = oracle_mod.run_layers(nh, [(W.z_label(nh, [62]), 1.0)],
                                  W.kicked_ising_layers(nh, edges, math.pi / 2), 3, 0.0,
                                  lib_path=path)
    return len(op) == 1


def _pin_table_relative(oracle_mod, path):
    """The Table's eps0 = 1e-5 column (relative truncation), t = 1..5."""
    nh, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(nh, edges, 0.9 * math.pi)
    m, _ = oracle_mod.run_layers(nh, [(W.z_label(nh, [62]), 1.0)], layers, 5, 1e-5, mode="rel",
                                 lib_path=path)
    return all(abs(got - e5) < 1e-13 for (_, _, _, e5), got in zip(_table(), m))


def _pin_relative_hand(oracle_mod, path):
    """The hand examples of the relative rule."""
    try:
        a, b, _ = _relative_hand_cases(oracle_mod, path)
    except Exception:
        return False
    return "X" in a and b == {"Z": 1.0}


# Cheapest first: a mistake that blows the operator up is caught by the
# small pins before the heavy-hex runs meet it.
PINS = [("phase", _pin_phase), ("dense", _pin_dense), ("relative_hand", _pin_relative_hand),
        ("statevector", _pin_statevector), ("clifford", _pin_clifford),
        ("table_relative", _pin_table_relative)]


def _first_failing_pin(oracle_mod, path):
    """The pins above, re-run in order on the oracle built at ``path``; the
    name of the first that fails, or None."""
    for name, pin in PINS:
        if not pin(oracle_mod, path):
            return name
    return None


# Each planted mistake (see the list at the top of orqa_oracle.cpp) and the
# first pin, in the order above, that catches it.
MUTATIONS = {
    1: "dense",            # Algorithm 1's source-indexed sign
    2: "dense",            # sin term taken from the updated value
    3: "clifford",         # no exact Clifford angles: ghost strings
    4: "statevector",      # sigma_y counted as diagonal in <0|O|0>
    5: "clifford",         # exact zeros kept
    6: "phase",            # Levi-Civita orientation reversed
    7: "dense",            # commuting strings rotated too
    8: "relative_hand",    # relative threshold from the max before the gate
    9: "dense",            # a branch overwrites the term already at its destination
    10: "dense",           # sin sign reversed at the Clifford angles
}


def test_default_oracle_passes_every_pin(oracle_mod):
    assert _first_failing_pin(oracle_mod, oracle_mod.build()) is None


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(oracle_mod, tmp_path, mutation):
    path = oracle_mod.build(out=str(tmp_path / ("mut%d.so" % mutation)),
                            defines=["ORACLE_MUTATION=%d" % mutation])
    assert _first_failing_pin(oracle_mod, path) == MUTATIONS[mutation]


def test_histogram_hand_example(oracle_mod):
    """D_t(x) counts on a hand-checked example: n_bins = 2 over
    log10|x| in [-4, 0] gives edges 1e-4 and 1e-2 times max|c| = 1."""
    counts, m = oracle_mod.histogram([1.0, -0.5, 0.01, -1e-7, 0.3, 2e-3, -5e-5], 2, -4.0)
    assert m == 1.0
    assert counts.tolist() == [[0 + 1, 3, 0], [0, 1, 2]]


def test_histogram_invariants(oracle_mod):
    """Every string lands in exactly one bin; the largest is in the top
    bin; scaling all coefficients by a power of two changes nothing."""
    import numpy as np
    rng = np.random.default_rng(3)
    c = rng.standard_normal(5000) * 10.0 ** rng.uniform(-8, 0, 5000)
    counts, m = oracle_mod.histogram(c, 16, -8.0)
    assert counts.sum() == c.size
    top = 0 if c[np.argmax(np.abs(c))] > 0 else 1
    assert counts[top, 15] >= 1
    scaled, m2 = oracle_mod.histogram(c * 0.25, 16, -8.0)
    assert m2 == m * 0.25 and (scaled == counts).all()
