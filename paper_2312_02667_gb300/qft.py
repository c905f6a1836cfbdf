"""The quantum Fourier transformation (QFT) compiled onto a line of qubits
(the additional benchmark of the paper's App. B), as sparse brickwork layers
of fused two-qubit gates for ``ptebd_apply_bonds``.

The paper compiles its QFT circuits with Qiskit to a linear layout (CX and
one-qubit gates).  No Qiskit is used here: the QFT is compiled by a SWAP
network of our own that needs no gates beyond nearest neighbours.

Textbook QFT on qubits 0..N-1 (qubit 0 the most significant bit, as everywhere
in this repository): for j = 0..N-1, a Hadamard on j, then for every k > j a
controlled phase CP(pi / 2^(k - j)) between j and k; the output bits come out
in reverse order.  The network moves logical qubit j, right after its
Hadamard, from the left end of the line to the right through all later
qubits: at each step it meets logical qubit k = j + m + 1 on bond (m, m+1) and
the two share one fused gate SWAP . CP(pi / 2^(m+1)).  Logical qubit j starts
two steps after j - 1, so the gate of (j, m) runs at step t = 2 j + m: every
step gates bonds of one parity, and the whole QFT is 2N - 3 steps of
N(N-1)/2 gates.  Since all controlled phases are diagonal they commute, and
each qubit meets its Hadamard before its first (j as mover) and after its last
(j as partner) phase gate; the last qubit's Hadamard is folded into the last
gate.  At the end position p holds logical qubit N-1-p: the reversal that the
textbook circuit needs is done by the network itself, so the state on the
line is QFT|psi> in natural order.

Gates use the library layout U[(2 s0' + s1'), (2 s0 + s1)], s0 the left site.
"""
from __future__ import annotations

import numpy as np

__all__ = ["qft_line_layers", "qft_gate_count", "qft_depth"]

_H = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=complex) / np.sqrt(2.0)
_I2 = np.eye(2, dtype=complex)
_SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)


def _cp(phi: float) -> np.ndarray:
    return np.diag([1.0, 1.0, 1.0, np.exp(1j * phi)]).astype(complex)


def qft_depth(n: int) -> int:
    """Number of compiled layers (steps) of the line network: 2N - 3."""
    return max(0, 2 * n - 3)


def qft_gate_count(n: int) -> int:
    """Number of fused two-qubit gates: N(N-1)/2."""
    return n * (n - 1) // 2


def qft_line_layers(n: int):
    """[(bonds int32 array, gates (n_bonds, 4, 4) complex128)] for N >= 2 qubits."""
    if n < 2:
        raise ValueError("the line network needs at least two qubits")
    hl = np.kron(_H, _I2)  # Hadamard on the left site of a bond
    layers = []
    for t in range(qft_depth(n)):
        bonds, gates = [], []
        for m in range(t % 2, n - 1, 2):
            j = (t - m) // 2
            if j < 0 or m > n - 2 - j:
                continue
            u = _SWAP @ _cp(np.pi / 2.0 ** (m + 1))
            if m == 0:
                u = u @ hl  # logical j starts its sweep: its Hadamard first
            if m == 0 and j == n - 2:
                u = hl @ u  # logical N-1 has met every other qubit: its Hadamard last
            bonds.append(m)
            gates.append(u)
        layers.append((np.asarray(bonds, dtype=np.int32), np.stack(gates)))
    return layers
