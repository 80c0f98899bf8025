"""The closed form the ZZ-layer kernel applies, checked on the CPU against
the oracle's gate-by-gate rule (Eq. update_rule at the Clifford angles).

All ZZ gates of a layer commute, so the kernel applies a whole edge set at
once.  With n_s the number of anticommuting edges at site s (neighbours t
with x_t != x_s) and C0, C1 the planes of the low two bits of n_s:
    z' = z xor C0                                  (theta = +-pi/2)
    sign flips iff parity(x & ((z & C0) xor C1))   (theta = -pi/2)
    sign flips iff parity(x & ((z & C0) xor C1 xor C0))   (theta = +pi/2)
    sign flips iff parity(x & C0), z unchanged     (theta = pi)
C0 and C1 are counted per offset group d (the edges (i, i + d)) with a
two-bit carry-save counter, as in the kernel.  Here both sides act on one
string with coefficient 1; the oracle returns its image and sign."""
import math
import random

import pytest


def _label(x, z, n):
    code = {(0, 0): "I", (1, 0): "X", (1, 1): "Y", (0, 1): "Z"}
    return "".join(code[((x >> q) & 1, (z >> q) & 1)] for q in range(n))


def _planes(codes):
    x = z = 0
    for q, a in enumerate(codes):
        if a in (1, 2):
            x |= 1 << q
        if a in (2, 3):
            z |= 1 << q
    return x, z


def _closed_form(x, z, edges, theta, n, planted=False):
    """(z', sign flip) of one string under all edges at a Clifford angle.
    planted: the sign rules of -pi/2 and +pi/2 swapped (a plausible slip)."""
    groups = {}
    for i, j in edges:
        a, b = min(i, j), max(i, j)
        groups[b - a] = groups.get(b - a, 0) | (1 << a)
    full = (1 << n) - 1
    c0 = c1 = 0
    for d, mask in sorted(groups.items()):
        a = (x ^ (x >> d)) & mask          # anticommuting edges (i, i + d), counted at i
        c1 ^= c0 & a
        c0 ^= a
        b = (a << d) & full                # ... and at i + d
        c1 ^= c0 & b
        c0 ^= b
    parity = lambda v: bin(v).count("1") & 1
    if abs(theta - math.pi) < 1e-12:
        return z, parity(x & c0)
    if (theta < 0) != planted:
        return z ^ c0, parity(x & ((z & c0) ^ c1))
    return z ^ c0, parity(x & ((z & c0) ^ c1 ^ c0))


def _random_case(rng):
    n = rng.choice([5, 12, 70, 127])
    m = rng.randint(1, min(60, n * (n - 1) // 2))
    edges = set()
    while len(edges) < m:
        a, b = rng.sample(range(n), 2)
        edges.add((min(a, b), max(a, b)))
    edges = sorted(edges)
    rng.shuffle(edges)
    x, z = rng.getrandbits(n), rng.getrandbits(n)
    if x == 0 and z == 0:
        z = 1
    return n, edges, x, z


def _oracle_image(oracle_mod, n, edges, x, z, theta):
    op = oracle_mod.Oracle(n)
    op.add_label(_label(x, z, n), 1.0)
    for i, j in edges:
        op.apply(("rzz", i, j, theta), 0.0)
    (key, c), = op.as_dict().items()
    xo, zo = _planes(oracle_mod.codes_from_index(key, n))
    return xo, zo, c


@pytest.mark.parametrize("theta", [-math.pi / 2, math.pi / 2, math.pi])
def test_closed_form_equals_gate_by_gate_rule(oracle_mod, theta):
    rng = random.Random(0x250613241 + int(theta * 1000))
    for trial in range(120):
        n, edges, x, z = _random_case(rng)
        xo, zo, c = _oracle_image(oracle_mod, n, edges, x, z, theta)
        z_cf, flip = _closed_form(x, z, edges, theta, n)
        assert xo == x, (trial, n)
        assert zo == z_cf, (trial, n)
        assert c == (-1.0 if flip else 1.0), (trial, n, c, flip)


def test_planted_sign_rule_is_caught(oracle_mod):
    """The same comparison sees the -pi/2 and +pi/2 sign rules swapped."""
    rng = random.Random(7)
    theta = -math.pi / 2
    caught = 0
    for _ in range(40):
        n, edges, x, z = _random_case(rng)
        _, _, c = _oracle_image(oracle_mod, n, edges, x, z, theta)
        _, flip = _closed_form(x, z, edges, theta, n, planted=True)
        caught += c != (-1.0 if flip else 1.0)
    assert caught > 0
