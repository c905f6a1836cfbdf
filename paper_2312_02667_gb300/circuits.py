"""The circuit families of the paper's benchmarks (App. A) as layers of
two-qubit gates on the MPS path.

Input preparation only: this module builds gate lists; it holds no step of
pTEBD itself.

* RQC-1D: N odd, D even physical layers.  Layer l = 1..D applies a random
  one-qubit gate U = exp[-i theta (sin(alpha) cos(phi) X + sin(alpha) sin(phi) Y
  + cos(alpha) Z)] to every qubit, then CZ on the pairs (0,1), (2,3), ... for
  odd l and (1,2), (3,4), ... for even l.
* PQC-1D (Hamiltonian variational ansatz of the Heisenberg chain): N and D
  even.  A first layer turns |0...0> into singlet dimers on (0,1), (2,3), ...;
  then D layers of eSWAP(theta) = exp(-i theta P / 2) (P = SWAP) on the pairs
  (1,2), (3,4), ... for odd l and (0,1), (2,3), ... for even l.
* RQC-2D / PQC-2D: the same gates in the A B C D pattern of a square lattice
  (``circuits2d``); for PQC-2D the first A layer makes the singlet dimers.

A one-qubit gate is folded into the two-qubit gate that next acts on its qubit
(applied first, as U_pair (V (x) W)); a qubit left without a partner in a layer
carries its one-qubit gates to its next pair; gates still carried after the
last layer are folded, applied after, into the last pair gate on their qubit.
The compiled circuit is therefore the same unitary as the physical one (pinned
by statevector simulation).

Readings of points the paper leaves open: alpha uniform in [0, pi), theta and
phi uniform in [0, 2 pi) for the one-qubit gates; the eSWAP angle uniform in
[0, 2 pi); the singlet dimers are made by CNOT (H (x) 1)(X (x) X), which maps
|00> to (|01> - |10>) / sqrt 2; the dimer layer of PQC-1D comes before the D
eSWAP layers (it is not one of them), so that the first eSWAP layer couples
the dimers.
"""
from __future__ import annotations

import numpy as np

from .circuits2d import SWAP, _pairs
from .inputs import _rng, layer_bonds

__all__ = [
    "CZ", "SINGLET_PREP", "one_qubit_gate", "eswap",
    "rqc1d_physical", "pqc1d_physical", "fuse_1d", "rqc1d_circuit", "pqc1d_circuit",
    "rqc2d_physical", "pqc2d_physical", "fuse_2d",
]

I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
_CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)

CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
SINGLET_PREP = _CNOT @ np.kron(_H, I2) @ np.kron(_X, _X)


def one_qubit_gate(rng: np.random.Generator) -> np.ndarray:
    """exp[-i theta n.sigma] with n = (sin a cos p, sin a sin p, cos a): since
    (n.sigma)^2 = 1 this is cos(theta) 1 - i sin(theta) n.sigma."""
    alpha = rng.uniform(0.0, np.pi)
    theta = rng.uniform(0.0, 2.0 * np.pi)
    phi = rng.uniform(0.0, 2.0 * np.pi)
    ns = (np.sin(alpha) * np.cos(phi)) * _X + (np.sin(alpha) * np.sin(phi)) * _Y + np.cos(alpha) * _Z
    return np.cos(theta) * I2 - 1j * np.sin(theta) * ns


def eswap(theta: float) -> np.ndarray:
    """exp(-i theta P / 2) = cos(theta / 2) 1 - i sin(theta / 2) P (P^2 = 1)."""
    return np.cos(theta / 2.0) * np.eye(4, dtype=np.complex128) - 1j * np.sin(theta / 2.0) * SWAP


# ------------------------------------------------------------------ 1D ----

def rqc1d_physical(seed: int, n: int, depth: int):
    """Physical layers [(one-qubit gates (n, 2, 2), pairs [(q, q + 1, CZ)])]."""
    if n % 2 == 0 or depth % 2:
        raise ValueError("RQC-1D takes an odd number of qubits and an even depth")
    out = []
    for l in range(1, depth + 1):
        rng = _rng(seed, 0x1D0, n, l)
        ones = np.stack([one_qubit_gate(rng) for _ in range(n)])
        parity = 0 if l % 2 else 1
        out.append((ones, [(int(b), int(b) + 1, CZ) for b in layer_bonds(n, parity)]))
    return out


def pqc1d_physical(seed: int, n: int, depth: int):
    """The dimer layer followed by `depth` eSWAP layers, in the format of
    `rqc1d_physical` (no one-qubit gates)."""
    if n % 2 or depth % 2:
        raise ValueError("PQC-1D takes an even number of qubits and an even depth")
    out = [(None, [(int(b), int(b) + 1, SINGLET_PREP) for b in layer_bonds(n, 0)])]
    for l in range(1, depth + 1):
        rng = _rng(seed, 0x1D1, n, l)
        parity = 1 if l % 2 else 0
        out.append((None, [(int(b), int(b) + 1, eswap(rng.uniform(0.0, 2.0 * np.pi)))
                           for b in layer_bonds(n, parity)]))
    return out


def _fuse(layers, qubits):
    """Fold the one-qubit gates into the pair gates (see the module notes).
    layers: [(ones: dict qubit -> 2x2 or None, [(q1, q2, G)])]; returns
    [[(q1, q2, fused 4x4)]] in the same order."""
    carry = {q: I2 for q in qubits}
    out = []
    last = {}  # qubit -> (layer index, pair index, position 0/1) of its last pair gate
    for li, (ones, pairs) in enumerate(layers):
        if ones is not None:
            for q in qubits:
                carry[q] = ones[q] @ carry[q]
        fused = []
        for pi, (q1, q2, g) in enumerate(pairs):
            fused.append([q1, q2, g @ np.kron(carry[q1], carry[q2])])
            carry[q1] = I2
            carry[q2] = I2
            last[q1] = (li, pi, 0)
            last[q2] = (li, pi, 1)
        out.append(fused)
    for q in qubits:
        if np.array_equal(carry[q], I2):
            continue
        if q not in last:
            raise ValueError(f"qubit {q} never takes part in a two-qubit gate")
        li, pi, side = last[q]
        f = out[li][pi]
        f[2] = (np.kron(carry[q], I2) if side == 0 else np.kron(I2, carry[q])) @ f[2]
    return [[(a, b, g) for a, b, g in layer] for layer in out]


def fuse_1d(physical, n: int):
    """Physical 1D layers -> [(parity, bonds, gates)] with the one-qubit gates
    folded in."""
    layers = [({q: ones[q] for q in range(n)} if ones is not None else None, pairs) for ones, pairs in physical]
    out = []
    for layer in _fuse(layers, list(range(n))):
        bonds = np.array([q1 for q1, _, _ in layer], dtype=np.int32)
        parity = int(bonds[0] % 2) if len(bonds) else 0
        gates = np.stack([g for _, _, g in layer]) if layer else np.zeros((0, 4, 4), complex)
        out.append((parity, bonds, gates))
    return out


def rqc1d_circuit(seed: int, n: int, depth: int):
    """RQC-1D as brickwork layers [(parity, bonds, gates)]."""
    return fuse_1d(rqc1d_physical(seed, n, depth), n)


def pqc1d_circuit(seed: int, n: int, depth: int):
    """PQC-1D as brickwork layers [(parity, bonds, gates)]: depth + 1 layers."""
    return fuse_1d(pqc1d_physical(seed, n, depth), n)


# ------------------------------------------------------------------ 2D ----

def _qubits_2d(lx, ly):
    return [(x, y) for x in range(lx) for y in range(ly)]


def rqc2d_physical(seed: int, lx: int, ly: int, depth: int):
    """[(kind, one-qubit gates {qubit: 2x2}, [(q1, q2, CZ)])] in the ABCD pattern."""
    if depth % 4:
        raise ValueError("the ABCD pattern needs a depth that is a multiple of 4")
    out = []
    for l in range(depth):
        kind = "ABCD"[l % 4]
        rng = _rng(seed, 0x2D0, lx, ly, l)
        ones = {q: one_qubit_gate(rng) for q in _qubits_2d(lx, ly)}
        out.append((kind, ones, [(q1, q2, CZ) for q1, q2 in _pairs(kind, lx, ly)]))
    return out


def pqc2d_physical(seed: int, lx: int, ly: int, depth: int):
    """The first A layer makes singlet dimers, the others are eSWAP layers."""
    if depth % 4:
        raise ValueError("the ABCD pattern needs a depth that is a multiple of 4")
    out = []
    for l in range(depth):
        kind = "ABCD"[l % 4]
        rng = _rng(seed, 0x2D1, lx, ly, l)
        if l == 0:
            pairs = [(q1, q2, SINGLET_PREP) for q1, q2 in _pairs(kind, lx, ly)]
        else:
            pairs = [(q1, q2, eswap(rng.uniform(0.0, 2.0 * np.pi))) for q1, q2 in _pairs(kind, lx, ly)]
        out.append((kind, None, pairs))
    return out


def fuse_2d(physical, lx: int, ly: int):
    """[(kind, [(q1, q2, fused 4x4)])]: the input of ``circuits2d.compile_layers``."""
    fused = _fuse([(ones, pairs) for _, ones, pairs in physical], _qubits_2d(lx, ly))
    return [(kind, layer) for (kind, _, _), layer in zip(physical, fused)]
