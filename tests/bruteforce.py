"""Dense brute-force references used to pin the oracle (test helpers only).

Everything here works with explicit 2^n x 2^n complex matrices or 2^n state
vectors, so it shares no representation with the oracle's multi-index code.
Qubit q is bit q of a basis-state index (kron factor ``n-1-q``).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

PAULI = {
    "I": np.array([[1, 0], [0, 1]], dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def pauli_matrix(label: str) -> np.ndarray:
    """Matrix of a label whose character q acts on qubit q."""
    m = np.array([[1.0 + 0j]])
    for ch in reversed(label):  # qubit n-1 is the leftmost kron factor
        m = np.kron(m, PAULI[ch])
    return m


def gate_label(gate, n: int) -> str:
    kind, q0, q1, _ = gate
    s = ["I"] * n
    if kind == "rx":
        s[q0] = "X"
    elif kind == "rzz":
        s[q0] = "Z"
        s[q1] = "Z"
    elif kind == "label":
        return q0
    else:
        raise ValueError(kind)
    return "".join(s)


def gate_unitary(gate, n: int) -> np.ndarray:
    """exp(-i theta/2 sigma_J) by the matrix exponential (scipy)."""
    theta = gate[3]
    return scipy.linalg.expm(-0.5j * theta * pauli_matrix(gate_label(gate, n)))


def heisenberg(op: np.ndarray, gates, n: int) -> np.ndarray:
    """U^dagger O U for U = G_1 G_2 ... applied gate by gate: the gate list
    is in Heisenberg order (first list entry conjugates first)."""
    for g in gates:
        U = gate_unitary(g, n)
        op = U.conj().T @ op @ U
    return op


def all_labels(n: int):
    labels = [""]
    for _ in range(n):
        labels = [l + c for l in labels for c in "IXYZ"]
    return labels


def pauli_decompose(op: np.ndarray, n: int, tol: float = 0.0) -> dict:
    """Coefficients c_Q = Tr(sigma_Q op) / 2^n of every Pauli string Q."""
    out = {}
    dim = 2 ** n
    for lab in all_labels(n):
        c = np.trace(pauli_matrix(lab) @ op) / dim
        if abs(c) > tol:
            out[lab] = c
    return out


def statevector_magnetization(n: int, layers, steps: int, site: int):
    """<psi_t| Z_site |psi_t> with |psi_t> = U^t |0>, U = U_zz U_x: each
    step applies U_x to the state first, then U_zz.  ``layers`` is in
    Heisenberg order [U_zz gates, U_x gates]; the state sees them reversed."""
    dim = 2 ** n
    psi = np.zeros(dim, dtype=np.complex128)
    psi[0] = 1.0
    idx = np.arange(dim)
    zsign = np.where((idx >> site) & 1, -1.0, 1.0)
    out = []
    for _ in range(steps):
        for layer in reversed(layers):
            for g in layer:
                psi = _apply_gate_to_state(psi, g, n)
        out.append(float(np.real(np.vdot(psi, zsign * psi))))
    return out


def _apply_gate_to_state(psi, gate, n):
    kind, q0, q1, theta = gate
    c = np.cos(theta / 2)
    s = np.sin(theta / 2)
    idx = np.arange(psi.size)
    if kind == "rx":
        flipped = psi[idx ^ (1 << q0)]
        return c * psi - 1j * s * flipped
    if kind == "rzz":
        parity = ((idx >> q0) ^ (idx >> q1)) & 1
        zz = np.where(parity, -1.0, 1.0)
        return (c - 1j * s * zz) * psi
    raise ValueError(kind)
