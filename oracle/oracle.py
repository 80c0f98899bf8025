"""ORQA oracle -- TEST INFRASTRUCTURE ONLY.

ctypes front end of the plain CPU oracle in ``orqa_oracle.cpp`` (a
``std::map`` run of Algorithm 1 of arXiv 2506.13241 with the sign of
Eq. (update_rule)).  Only the tests, the smoke check and the benchmark's CPU
baseline leg use this module; the CUDA library never imports it.

Strings cross this boundary in the paper's own encoding: the 2n-bit
multi-index with two bits per site (00 = id, 01 = x, 10 = y, 11 = z), site q
at bits 2q and 2q+1, stored as four little-endian uint64 words.

Gates are given as ``(kind, q0, q1, theta)`` tuples with kind ``"rx"``
(generator sigma_x on q0) or ``"rzz"`` (generator sigma_z sigma_z on q0, q1),
or as ``("pauli", J_words, None, theta)`` with an explicit multi-index J.
Each gate is exp(-i theta/2 sigma_J) (App. A).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orqa_oracle.cpp")
_LIB = os.path.join(_HERE, "liborqa_oracle.so")
_lock = threading.Lock()
_libs = {}

CODE = {"I": 0, "X": 1, "Y": 2, "Z": 3}


def build(force: bool = False, out: str | None = None, defines=()) -> str:
    """Compile the oracle with g++ (no FMA contraction: products and sums
    are rounded one at a time, in the order the paper's update states).
    ``defines`` plants a deliberate mistake (ORACLE_MUTATION=k) for the tests
    that show the pins catch it; the default build has none."""
    out = out or _LIB
    if force or defines or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".tmp.%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", tmp, _SRC]
        cmd[1:1] = ["-D" + d for d in defines]
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


def _load(path: str | None = None):
    with _lock:
        key = path or _LIB
        if key not in _libs:
            lib = ctypes.CDLL(path if path else build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_new.restype = ctypes.c_void_p
            lib.oracle_new.argtypes = [ctypes.c_int]
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            lib.oracle_add_term.argtypes = [ctypes.c_void_p, u64p, ctypes.c_double]
            lib.oracle_size.restype = ctypes.c_int64
            lib.oracle_size.argtypes = [ctypes.c_void_p]
            for name in ("oracle_apply_gate", "oracle_apply_gate_rel"):
                getattr(lib, name).argtypes = [ctypes.c_void_p, u64p, ctypes.c_double, ctypes.c_double]
            lib.oracle_rotate_only.argtypes = [ctypes.c_void_p, u64p, ctypes.c_double]
            lib.oracle_truncate.argtypes = [ctypes.c_void_p, ctypes.c_double]
            lib.oracle_max_abs.restype = ctypes.c_double
            lib.oracle_max_abs.argtypes = [ctypes.c_void_p]
            lib.oracle_expect_zero.restype = ctypes.c_double
            lib.oracle_expect_zero.argtypes = [ctypes.c_void_p]
            lib.oracle_norm2.restype = ctypes.c_double
            lib.oracle_norm2.argtypes = [ctypes.c_void_p]
            lib.oracle_export.restype = ctypes.c_int64
            lib.oracle_export.argtypes = [ctypes.c_void_p, ctypes.c_int64, u64p, dp]
            lib.oracle_phase_exponent.restype = ctypes.c_int
            lib.oracle_phase_exponent.argtypes = [u64p, u64p, ctypes.c_int]
            lib.oracle_rotation_cos_sin.argtypes = [ctypes.c_double, dp, dp]
            _libs[key] = lib
    return _libs[key]


def _words(key) -> ctypes.Array:
    arr = (ctypes.c_uint64 * 4)(*[int(w) & 0xFFFFFFFFFFFFFFFF for w in key])
    return arr


def index_from_codes(codes) -> tuple:
    """Multi-index words from a per-site list of local codes (0..3)."""
    v = 0
    for q, a in enumerate(codes):
        v |= (int(a) & 3) << (2 * q)
    return tuple((v >> (64 * w)) & 0xFFFFFFFFFFFFFFFF for w in range(4))


def index_from_label(label: str) -> tuple:
    """Multi-index of a label such as "XIZY" (character q is site q)."""
    return index_from_codes([CODE[ch] for ch in label])


def codes_from_index(key, n: int) -> list:
    v = 0
    for w in range(4):
        v |= int(key[w]) << (64 * w)
    return [(v >> (2 * q)) & 3 for q in range(n)]


def gate_index(gate, n: int) -> tuple:
    kind, q0, q1, _theta = gate
    codes = [0] * n
    if kind == "rx":
        codes[q0] = CODE["X"]
    elif kind == "rzz":
        codes[q0] = CODE["Z"]
        codes[q1] = CODE["Z"]
    elif kind == "pauli":
        return tuple(q0)
    else:
        raise ValueError("unknown gate kind %r" % (kind,))
    return index_from_codes(codes)


def phase_exponent(I, J, n: int, lib_path: str | None = None) -> int:
    """B(I, J) of Eq. (orqaproduct): sigma_I sigma_J = i^B sigma_{I xor J}."""
    return _load(lib_path).oracle_phase_exponent(_words(I), _words(J), n)


def rotation_cos_sin(theta: float):
    c = ctypes.c_double()
    s = ctypes.c_double()
    _load().oracle_rotation_cos_sin(theta, ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def histogram(coefs, n_bins: int, log10_lo: float):
    """Pauli-string density D_t(x) of App. D as counts: x = c / max|c|, bins
    uniform in log10|x| over [log10_lo, 0].  Reading (the paper gives no
    binning): edge k is t_k = max|c| * 10**(log10_lo + k * w) with
    w = -log10_lo / n_bins; bin k holds t_k <= |c| < t_{k+1}, the last bin
    also |c| = max|c|; column n_bins counts |c| < t_0; row 0 is c > 0 and
    row 1 is c < 0.  Returns (counts [2, n_bins + 1], max|c|)."""
    c = np.asarray(coefs, dtype=np.float64)
    counts = np.zeros((2, n_bins + 1), dtype=np.int64)
    if c.size == 0:
        return counts, 0.0
    a = np.abs(c)
    m = float(a.max())
    w = -log10_lo / n_bins
    edges = np.array([m * 10.0 ** (log10_lo + k * w) for k in range(n_bins)])
    k = np.searchsorted(edges, a, side="right") - 1   # largest k with edges[k] <= |c|
    k = np.where(k < 0, n_bins, np.minimum(k, n_bins - 1))
    row = np.where(c > 0, 0, 1)
    np.add.at(counts, (row, k), 1)
    return counts, m


class Oracle:
    """A Pauli-sum operator O = sum_I O_I sigma_I held by the C++ oracle."""

    def __init__(self, n_qubits: int, lib_path: str | None = None):
        self.n = n_qubits
        self._lib = _load(lib_path)
        self._h = self._lib.oracle_new(n_qubits)
        if not self._h:
            raise ValueError("n_qubits must be in 1..128")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_free(h)
            self._h = None

    def add(self, key, c: float):
        self._lib.oracle_add_term(self._h, _words(key), float(c))

    def add_label(self, label: str, c: float):
        self.add(index_from_label(label), c)

    def __len__(self):
        return int(self._lib.oracle_size(self._h))

    def apply(self, gate, delta: float = 0.0):
        """One gate of Algorithm 1 followed by |c| < delta / c == 0 truncation."""
        J = gate_index(gate, self.n)
        self._lib.oracle_apply_gate(self._h, _words(J), float(gate[3]), float(delta))

    def apply_rel(self, gate, eps0: float):
        J = gate_index(gate, self.n)
        self._lib.oracle_apply_gate_rel(self._h, _words(J), float(gate[3]), float(eps0))

    def rotate_only(self, gate):
        J = gate_index(gate, self.n)
        self._lib.oracle_rotate_only(self._h, _words(J), float(gate[3]))

    def truncate(self, delta: float):
        self._lib.oracle_truncate(self._h, float(delta))

    def expect_zero(self) -> float:
        return float(self._lib.oracle_expect_zero(self._h))

    def norm2(self) -> float:
        return float(self._lib.oracle_norm2(self._h))

    def max_abs(self) -> float:
        return float(self._lib.oracle_max_abs(self._h))

    def export(self):
        """(keys uint64[N,4], coefficients float64[N]) in key order."""
        n = len(self)
        keys = np.zeros((max(n, 1), 4), dtype=np.uint64)
        coef = np.zeros(max(n, 1), dtype=np.float64)
        got = self._lib.oracle_export(
            self._h, n,
            keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
            coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert got == n
        return keys[:n], coef[:n]

    def as_dict(self) -> dict:
        keys, coef = self.export()
        return {tuple(int(w) for w in k): float(c) for k, c in zip(keys, coef)}


def run_layers(n: int, observable, layers, steps: int, delta: float = 0.0,
               mode: str = "abs", on_step=None, lib_path: str | None = None):
    """Evolve ``observable`` (a list of (label-or-key, coefficient)) through
    ``steps`` repetitions of ``layers`` (a list of gate lists applied in
    order, one gate at a time, each followed by truncation).  Returns the
    list of <0|O_t|0> after each step and the final Oracle."""
    op = Oracle(n, lib_path)
    for key, c in observable:
        if isinstance(key, str):
            op.add_label(key, c)
        else:
            op.add(key, c)
    m = []
    for t in range(steps):
        for layer in layers:
            for g in layer:
                if mode == "abs":
                    op.apply(g, delta)
                else:
                    op.apply_rel(g, delta)
        m.append(op.expect_zero())
        if on_step is not None:
            on_step(t + 1, op)
    return m, op
