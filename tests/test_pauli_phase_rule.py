"""The bit-plane rule of the general-rotation kernel, checked on the CPU
against the oracle's gate (Eq. update_rule for any sigma_J).

For U = exp(-i theta J / 2), U^dagger P U = P when P commutes with J, else
cos(theta) P + i sin(theta) J P, with J P = i^B(J,P) sigma_{J xor P} and B odd:
the child's factor is i^(1 + B), -1 for B = 1 and +1 for B = 3 (mod 4).
The kernel works on x/z planes: P anticommutes with J iff
popcount((x & z_J) ^ (z & x_J)) is odd, and B(J, P) mod 4 is the number of
sites where (J, P) is (X, Y), (Y, Z) or (Z, X) minus the number where it is
(X, Z), (Y, X) or (Z, Y).  Here that rule, written on Python integers as
the kernel writes it on 64-bit words, must give the string, sign and
magnitude the oracle gives for one string under one gate."""
import math
import random

import pytest

CODE = {(0, 0): "I", (1, 0): "X", (1, 1): "Y", (0, 1): "Z"}


def _label(x, z, n):
    return "".join(CODE[((x >> q) & 1, (z >> q) & 1)] for q in range(n))


def _planes(codes):
    x = z = 0
    for q, a in enumerate(codes):
        if a in (1, 2):
            x |= 1 << q
        if a in (2, 3):
            z |= 1 << q
    return x, z


def _kernel_rule(jx_, jz_, x, z, n, planted=False):
    """(anticommutes, child factor) by the kernel's plane arithmetic.
    planted: B counted as B(P, J) instead of B(J, P) (operands swapped)."""
    full = (1 << n) - 1
    anti = bin((x & jz_) ^ (z & jx_)).count("1") & 1
    jx, jy, jz = jx_ & ~jz_ & full, jx_ & jz_, ~jx_ & jz_ & full
    px, py, pz = x & ~z & full, x & z, ~x & z & full
    if planted:
        (jx, jy, jz), (px, py, pz) = (px, py, pz), (jx, jy, jz)
    plus = bin((jx & py) | (jy & pz) | (jz & px)).count("1")
    minus = bin((jx & pz) | (jy & px) | (jz & py)).count("1")
    B = (plus - minus) & 3
    return anti == 1, (-1.0 if B == 1 else 1.0)


@pytest.mark.parametrize("n", [1, 3, 64, 70, 128])
def test_plane_rule_matches_oracle(oracle_mod, n):
    rng = random.Random(0x250613241 + n)
    theta = 0.7
    c, s = oracle_mod.rotation_cos_sin(theta)
    for trial in range(300):
        x, z = rng.getrandbits(n), rng.getrandbits(n)
        jx, jz = rng.getrandbits(n), rng.getrandbits(n)
        if jx == 0 and jz == 0:
            jz = 1
        op = oracle_mod.Oracle(n)
        op.add_label(_label(x, z, n), 1.0)
        op.rotate_only(("pauli", oracle_mod.index_from_label(_label(jx, jz, n)), None, theta))
        got = {_planes(oracle_mod.codes_from_index(k, n)): v for k, v in op.as_dict().items()}
        anti, factor = _kernel_rule(jx, jz, x, z, n)
        if not anti:
            assert got == {(x, z): 1.0}, trial
        else:
            assert got == {(x, z): c, (x ^ jx, z ^ jz): factor * s}, trial


def test_planted_operand_order_is_caught(oracle_mod):
    """The same comparison sees B(P, J) used in place of B(J, P)."""
    rng = random.Random(3)
    n, theta = 4, 0.7
    c, s = oracle_mod.rotation_cos_sin(theta)
    caught = 0
    for _ in range(60):
        x, z, jx, jz = (rng.getrandbits(n) for _ in range(4))
        anti, factor = _kernel_rule(jx, jz, x, z, n, planted=True)
        if not anti:
            continue
        op = oracle_mod.Oracle(n)
        op.add_label(_label(x, z, n), 1.0)
        op.rotate_only(("pauli", oracle_mod.index_from_label(_label(jx, jz, n)), None, theta))
        got = {_planes(oracle_mod.codes_from_index(k, n)): v for k, v in op.as_dict().items()}
        caught += got.get((x ^ jx, z ^ jz)) != factor * s
    assert caught > 0
