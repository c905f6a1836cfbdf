"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module only draws random numbers and arranges them into the inputs of the
method (two-qubit gates, random MPS tensors, one-site operators).  It holds no
step of pTEBD itself: no contraction, SVD, truncation or regauging.

Conventions (used everywhere in this repository):

* sites s = 0..N-1, bond b = 0..N-2 joins sites b and b+1;
* a gate on bond b is a 4x4 complex matrix U[(2*s0' + s1'), (2*s0 + s1)] where
  s0 is the physical index of site b (the most significant one) and s1 that of
  site b+1; a layer of parity p gates every bond b with b % 2 == p;
* the circuits are brickwork circuits of Haar-random U(4) gates: layer l has
  parity l % 2, so the first layer gates the pairs (0,1), (2,3), ... which the
  paper calls the odd physical layer (App. A, RQC-1D).

Random streams are keyed by (seed, circuit, layer) through numpy's SeedSequence,
so that any layer of any circuit can be regenerated on its own.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "haar_u4",
    "layer_bonds",
    "brickwork_layer",
    "brickwork_circuit",
    "random_mps_tensors",
    "random_one_site_op",
    "gates_to_interleaved",
    "saturated_bond",
    "trotter_heisenberg_circuit",
    "random_mps_scaled",
]


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng([int(k) & 0xFFFFFFFF for k in key])


def haar_u4(rng: np.random.Generator) -> np.ndarray:
    """One Haar-random 4x4 unitary: QR of a complex Ginibre matrix with the
    phases of R's diagonal moved into Q (Mezzadri, Notices AMS 54, 592 (2007))."""
    z = (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def layer_bonds(n_sites: int, parity: int) -> np.ndarray:
    """Bonds gated by a brickwork layer of the given parity."""
    return np.arange(parity, n_sites - 1, 2, dtype=np.int32)


def brickwork_layer(seed: int, n_sites: int, layer: int, circuit: int = 0):
    """(parity, bonds, gates[n_bonds,4,4]) of one brickwork layer."""
    parity = layer % 2
    bonds = layer_bonds(n_sites, parity)
    rng = _rng(seed, circuit, layer, 0x6A7E)
    gates = np.stack([haar_u4(rng) for _ in range(len(bonds))]) if len(bonds) else np.zeros((0, 4, 4), complex)
    return parity, bonds, gates


def brickwork_circuit(seed: int, n_sites: int, depth: int, circuit: int = 0):
    """List of `depth` brickwork layers, see `brickwork_layer`."""
    return [brickwork_layer(seed, n_sites, l, circuit) for l in range(depth)]


def random_mps_tensors(seed: int, n_sites: int, chi: int, d: int = 2):
    """Random open-MPS tensors M[s] of shape (d, chi_left, chi_right) with
    entries a + ib, a and b uniform in [-1, 1] (the recipe of Sec. III D used
    for the PtSU experiment).  Bond dimensions are min(chi, d^b, d^(N-b))."""
    rng = _rng(seed, 0x3A5, n_sites, chi)
    dims = [1] + [min(chi, d ** (b + 1), d ** (n_sites - b - 1)) for b in range(n_sites - 1)] + [1]
    out = []
    for s in range(n_sites):
        shape = (d, dims[s], dims[s + 1])
        out.append(rng.uniform(-1.0, 1.0, shape) + 1j * rng.uniform(-1.0, 1.0, shape))
    return out


def random_mps_scaled(seed: int, n_sites: int, chi: int, d: int = 2):
    """The random tensors of random_mps_tensors, each scaled to the Frobenius
    norm sqrt(chi_right) that a canonical (left-orthonormal) tensor has, so that
    the norm of a long random MPS stays within floating-point range (it would
    otherwise grow geometrically with N)."""
    out = []
    for m in random_mps_tensors(seed, n_sites, chi, d):
        out.append(m * (np.sqrt(m.shape[2]) / np.linalg.norm(m)))
    return out


def random_one_site_op(seed: int, hermitian: bool = True) -> np.ndarray:
    """A random 2x2 complex operator (Hermitian by default)."""
    rng = _rng(seed, 0x0B5)
    a = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    return (a + a.conj().T) / 2 if hermitian else a


def gates_to_interleaved(gates: np.ndarray) -> np.ndarray:
    """(n,4,4) complex128 -> contiguous float64 array of n*32 values, each gate
    row-major with (re, im) interleaved: the layout the C ABI takes."""
    g = np.ascontiguousarray(np.asarray(gates, dtype=np.complex128))
    return np.ascontiguousarray(g.view(np.float64).reshape(-1))


def saturated_bond(seed: int, chi: int) -> dict:
    """Synthetic environment of one bond of a state saturated at chi_max = chi:
    three descending, normalised Lambda vectors of length chi, two random
    Gamma tensors (2, chi, chi) and a Haar gate.  Used where only the shape of
    the work matters (timing the oracle on a sample of the bench workload)."""
    rng = _rng(seed, 0x5A7, chi)

    def lam():
        x = np.sort(np.abs(rng.standard_normal(chi)))[::-1] + 1e-3
        return x / np.linalg.norm(x)

    def gam():
        return (rng.standard_normal((2, chi, chi)) + 1j * rng.standard_normal((2, chi, chi))) / np.sqrt(2 * chi)

    return {"lam_l": lam(), "lam_c": lam(), "lam_r": lam(), "gamma_l": gam(), "gamma_r": gam(),
            "gate": haar_u4(rng)}


def _haar_u2(rng: np.random.Generator) -> np.ndarray:
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def trotter_heisenberg_circuit(seed: int, n_sites: int, depth: int, dt: float):
    """Brickwork layers of first-order Trotter steps exp(-i dt h_b) of a Heisenberg
    chain with random fields, h_b = XX + YY + ZZ + f_b Z(x)1 + f'_b 1(x)Z (f, f'
    uniform in [-1, 1], fixed per bond), from |0...0> rotated by one Haar-random
    one-qubit gate per site (folded into the first layer's gates; n_sites even).
    Near-identity gates on a weakly entangled state: the Schmidt spectra fall
    off fast, through the range that complex64 arithmetic cannot resolve.
    Returns the same (parity, bonds, gates) list as brickwork_circuit."""
    assert n_sites % 2 == 0
    rng = _rng(seed, 0x7107, n_sites)
    x = np.array([[0, 1], [1, 0]], complex)
    y = np.array([[0, -1j], [1j, 0]])
    z = np.diag([1.0, -1.0]).astype(complex)
    one = np.eye(2)
    fields = rng.uniform(-1.0, 1.0, (n_sites - 1, 2))
    gates_of = []
    for b in range(n_sites - 1):
        h = np.kron(x, x) + np.kron(y, y) + np.kron(z, z) + fields[b, 0] * np.kron(z, one) \
            + fields[b, 1] * np.kron(one, z)
        w, v = np.linalg.eigh(h)
        gates_of.append((v * np.exp(-1j * dt * w)[None, :]) @ v.conj().T)
    rot = [_haar_u2(rng) for _ in range(n_sites)]
    layers = []
    for l in range(depth):
        parity = l % 2
        bonds = layer_bonds(n_sites, parity)
        gates = []
        for b in bonds:
            u = gates_of[b]
            if l == 0:
                u = u @ np.kron(rot[b], rot[b + 1])
            gates.append(u)
        layers.append((parity, bonds, np.stack(gates) if gates else np.zeros((0, 4, 4), complex)))
    return layers
