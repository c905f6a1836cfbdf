"""Exact statevector simulation for small N (oracle pin; test infrastructure only).

Site 0 is the most significant qubit of the 2^N index.  A two-site gate on bond b
acts on (site b, site b+1) as U[(2 s' + t'), (2 s + t)] (the same layout as the
MPS layer), so this module checks the layer without sharing any of its steps.
"""
from __future__ import annotations

import numpy as np

from .mps import Vidal

__all__ = ["zero_state", "apply_two_qubit", "from_vidal", "schmidt_values", "fidelity"]


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_two_qubit(psi: np.ndarray, n: int, b: int, gate: np.ndarray) -> np.ndarray:
    """Apply a 4x4 gate to qubits (b, b+1)."""
    v = psi.reshape(2 ** b, 4, 2 ** (n - b - 2))
    return np.einsum("ij,ajc->aic", np.asarray(gate, dtype=np.complex128), v).reshape(-1)


def from_vidal(mps: Vidal) -> np.ndarray:
    """Contract Gamma_0 Lambda_0 Gamma_1 ... Gamma_{N-1} into the 2^N amplitudes."""
    acc = np.ones((1, 1), dtype=np.complex128)  # (physical prefix, right bond)
    for s in range(mps.n_sites):
        m = mps.gammas[s] * mps.lam(s)[None, None, :]
        acc = np.einsum("pa,sab->psb", acc, m).reshape(-1, m.shape[2])
    return acc.reshape(-1)


def schmidt_values(psi: np.ndarray, n: int, b: int) -> np.ndarray:
    """Singular values of Psi reshaped to (sites 0..b) x (sites b+1..N-1)
    (Sec. II B: the diagonal of Lambda^{[i]} is this spectrum)."""
    return np.linalg.svd(psi.reshape(2 ** (b + 1), 2 ** (n - b - 1)), compute_uv=False)


def fidelity(a: np.ndarray, b: np.ndarray) -> float:
    """|<a|b>|^2 / (<a|a><b|b>)."""
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))
