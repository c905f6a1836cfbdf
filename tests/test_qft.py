"""The QFT line network (App. B workload) against the discrete Fourier
transform, on the CPU: exact statevector simulation of the compiled layers
equals (F psi)_y = sum_x exp(2 pi i x y / 2^N) psi_x / sqrt(2^N) (qubit 0 the
most significant bit) for random inputs, and the layer structure is what the
pTEBD layer needs (bonds of one parity per layer, no shared site)."""
import numpy as np
import pytest

from oracle import statevector as sv
from paper_2312_02667_gb300 import qft


def dft(n):
    x = np.arange(2 ** n)
    return np.exp(2j * np.pi * np.outer(x, x) / 2 ** n) / np.sqrt(2 ** n)


def run_layers(psi, n, layers):
    for bonds, gates in layers:
        for b, u in zip(bonds, gates):
            psi = sv.apply_two_qubit(psi, n, int(b), u)
    return psi


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_network_is_the_dft(n):
    rng = np.random.default_rng(100 + n)
    psi = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    psi /= np.linalg.norm(psi)
    out = run_layers(psi, n, qft.qft_line_layers(n))
    assert np.abs(out - dft(n) @ psi).max() < 1e-13


def test_counts_and_layer_structure():
    for n in range(2, 40):
        layers = qft.qft_line_layers(n)
        assert len(layers) == qft.qft_depth(n) == max(0, 2 * n - 3)
        assert sum(len(b) for b, _ in layers) == qft.qft_gate_count(n) == n * (n - 1) // 2
        for t, (bonds, gates) in enumerate(layers):
            assert len(bonds) > 0 and np.all(bonds % 2 == t % 2)
            assert np.all(np.diff(bonds) >= 2) and bonds.min() >= 0 and bonds.max() <= n - 2
            assert np.allclose(np.einsum("kij,kil->kjl", gates.conj(), gates), np.eye(4), atol=1e-14)


def test_missing_hadamard_is_caught():
    # a planted mistake (the last qubit's Hadamard left out) must fail the pin
    n = 5
    layers = qft.qft_line_layers(n)
    bonds, gates = layers[-1]
    hl = np.kron(np.array([[1, 1], [1, -1]]) / np.sqrt(2), np.eye(2))
    broken = layers[:-1] + [(bonds, np.stack([hl @ gates[0]]))]  # H H = 1 undoes the fold
    rng = np.random.default_rng(7)
    psi = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    psi /= np.linalg.norm(psi)
    assert np.abs(run_layers(psi, n, broken) - dft(n) @ psi).max() > 1e-2
