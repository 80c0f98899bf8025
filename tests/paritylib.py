"""Helpers shared by the parity tests: canonical forms of the CUDA path's
export (x/z planes) and of the oracle's export (paper multi-index), so the
two can be compared element by element."""
from __future__ import annotations

import numpy as np


def planes_to_codes(x: np.ndarray, z: np.ndarray, n: int) -> np.ndarray:
    """Per-site local codes (0 id, 1 x, 2 y, 3 z) [N, n] from x/z planes:
    the paper's code has high bit z and low bit x xor z."""
    N = x.shape[0]
    codes = np.zeros((N, n), dtype=np.uint8)
    for q in range(n):
        w, b = divmod(q, 64)
        xb = ((x[:, w] >> np.uint64(b)) & np.uint64(1)).astype(np.uint8)
        zb = ((z[:, w] >> np.uint64(b)) & np.uint64(1)).astype(np.uint8)
        codes[:, q] = (zb << 1) | (xb ^ zb)
    return codes


def index_words_to_codes(keys: np.ndarray, n: int) -> np.ndarray:
    """Per-site codes [N, n] from oracle multi-index words [N, 4]."""
    N = keys.shape[0]
    codes = np.zeros((N, n), dtype=np.uint8)
    for q in range(n):
        bit = 2 * q
        w, b = divmod(bit, 64)
        codes[:, q] = ((keys[:, w] >> np.uint64(b)) & np.uint64(3)).astype(np.uint8)
    return codes


def canonical(codes: np.ndarray, coef: np.ndarray):
    """Rows sorted lexicographically by code string."""
    if codes.shape[0] == 0:
        return codes, coef
    order = np.lexsort(codes.T[::-1])
    return codes[order], coef[order]


def gpu_canonical(ctx, n: int):
    x, z, c = ctx.export()
    return canonical(planes_to_codes(x, z, n), c)


def oracle_canonical(op, n: int):
    keys, c = op.export()
    return canonical(index_words_to_codes(keys, n), c)


def assert_bit_exact(gpu, ora, what=""):
    gc, gv = gpu
    oc, ov = ora
    assert gc.shape == oc.shape, "%s: |O| gpu %d vs oracle %d" % (what, gc.shape[0], oc.shape[0])
    if gc.shape[0]:
        same_keys = np.all(gc == oc, axis=1)
        assert same_keys.all(), "%s: first differing string at row %d" % (what, int(np.argmin(same_keys)))
        bad = np.nonzero(gv.view(np.uint64) != ov.view(np.uint64))[0]
        assert bad.size == 0, "%s: %d coefficients differ, first row %d: %r vs %r" % (
            what, bad.size, bad[0], gv[bad[0]], ov[bad[0]])




def codes_to_planes(codes: np.ndarray, W: int):
    """x/z planes [N, W] from per-site codes [N, n] (z = high bit, x = high
    xor low of the paper's code)."""
    N, n = codes.shape
    x = np.zeros((N, W), dtype=np.uint64)
    z = np.zeros((N, W), dtype=np.uint64)
    for q in range(n):
        w, b = divmod(q, 64)
        hi = (codes[:, q] >> 1) & 1
        lo = codes[:, q] & 1
        x[:, w] |= (hi ^ lo).astype(np.uint64) << np.uint64(b)
        z[:, w] |= hi.astype(np.uint64) << np.uint64(b)
    return x, z


def canonical_key_order(x: np.ndarray, z: np.ndarray, problem=None):
    """Row order of the canonical export: ascending by x words from the
    highest to the lowest, then z words likewise (problem index first)."""
    W = x.shape[1]
    keys = [z[:, w] for w in range(W)] + [x[:, w] for w in range(W)]
    if problem is not None:
        keys.append(np.asarray(problem))
    return np.lexsort(keys)


def planes_to_index_words(x: np.ndarray, z: np.ndarray, n: int) -> np.ndarray:
    """Oracle multi-index words [N, 4] (two bits per site, the paper's code)
    from x/z planes."""
    codes = planes_to_codes(x, z, n)
    keys = np.zeros((x.shape[0], 4), dtype=np.uint64)
    for q in range(n):
        w, b = divmod(2 * q, 64)
        keys[:, w] |= codes[:, q].astype(np.uint64) << np.uint64(b)
    return keys
