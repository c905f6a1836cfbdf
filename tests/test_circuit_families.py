"""The paper's circuit families (App. A): the compiled two-qubit layers
against the physical circuit by exact statevector simulation, and the gate
definitions against matrix exponentials."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle import statevector as sv
from paper_2312_02667_gb300 import circuits, circuits2d

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]])
Z = np.diag([1.0, -1.0]).astype(complex)


def apply_one(psi, n, q, u):
    t = np.moveaxis(psi.reshape([2] * n), q, 0)
    sh = t.shape
    t = (u @ t.reshape(2, -1)).reshape(sh)
    return np.moveaxis(t, 0, q).reshape(-1)


def apply_pair(psi, n, p1, p2, u):
    t = np.moveaxis(psi.reshape([2] * n), (p1, p2), (0, 1))
    sh = t.shape
    t = (u @ t.reshape(4, -1)).reshape(sh)
    return np.moveaxis(t, (0, 1), (p1, p2)).reshape(-1)


def test_one_qubit_gate_is_the_exponential():
    rng = np.random.default_rng(0)
    for _ in range(5):
        state = rng.bit_generator.state
        u = circuits.one_qubit_gate(rng)
        rng2 = np.random.default_rng(0)
        rng2.bit_generator.state = state
        a, t, p = rng2.uniform(0, np.pi), rng2.uniform(0, 2 * np.pi), rng2.uniform(0, 2 * np.pi)
        h = np.sin(a) * np.cos(p) * X + np.sin(a) * np.sin(p) * Y + np.cos(a) * Z
        assert np.abs(u - sla.expm(-1j * t * h)).max() < 1e-13


def test_eswap_and_singlet():
    for th in (0.3, 1.7, 5.0):
        assert np.abs(circuits.eswap(th) - sla.expm(-0.5j * th * circuits2d.SWAP)).max() < 1e-13
    out = circuits.SINGLET_PREP @ np.array([1, 0, 0, 0], dtype=complex)
    assert np.abs(out - np.array([0, 1, -1, 0]) / np.sqrt(2)).max() < 1e-15
    assert np.abs(circuits.SINGLET_PREP.conj().T @ circuits.SINGLET_PREP - np.eye(4)).max() < 1e-15


def run_physical_1d(physical, n):
    psi = sv.zero_state(n)
    for ones, pairs in physical:
        if ones is not None:
            for q in range(n):
                psi = apply_one(psi, n, q, ones[q])
        for q1, q2, g in pairs:
            psi = apply_pair(psi, n, q1, q2, g)
    return psi


def run_compiled_1d(layers, n):
    psi = sv.zero_state(n)
    for parity, bonds, gates in layers:
        assert all(int(b) % 2 == parity for b in bonds)
        for b, u in zip(bonds, gates):
            psi = sv.apply_two_qubit(psi, n, int(b), u)
    return psi


@pytest.mark.parametrize("n,depth", [(5, 4), (7, 6), (9, 2)])
def test_rqc1d_compiled_equals_physical(n, depth):
    phys = circuits.rqc1d_physical(11, n, depth)
    comp = circuits.rqc1d_circuit(11, n, depth)
    assert len(comp) == depth
    assert np.abs(run_physical_1d(phys, n) - run_compiled_1d(comp, n)).max() < 1e-12


@pytest.mark.parametrize("n,depth", [(6, 4), (8, 2)])
def test_pqc1d_compiled_equals_physical(n, depth):
    phys = circuits.pqc1d_physical(12, n, depth)
    comp = circuits.pqc1d_circuit(12, n, depth)
    assert len(comp) == depth + 1
    assert np.abs(run_physical_1d(phys, n) - run_compiled_1d(comp, n)).max() < 1e-12
    # after the first layer: a product of singlets, each bond (2q, 2q+1) maximally entangled
    psi = run_compiled_1d(comp[:1], n)
    singlet = np.array([0, 1, -1, 0]) / np.sqrt(2)
    ref = singlet
    for _ in range(n // 2 - 1):
        ref = np.kron(ref, singlet)
    assert np.abs(psi - ref).max() < 1e-15


def run_physical_2d(physical, lx, ly):
    n = lx * ly
    pos = circuits2d.position(lx, ly)
    psi = sv.zero_state(n)
    for kind, ones, pairs in physical:
        if ones is not None:
            for q, u in ones.items():
                psi = apply_one(psi, n, pos[q], u)
        for q1, q2, g in pairs:
            psi = apply_pair(psi, n, pos[q1], pos[q2], g)
    return psi


@pytest.mark.parametrize("family", ["rqc", "pqc"])
@pytest.mark.parametrize("lx,ly", [(3, 3), (2, 4), (3, 2)])
def test_2d_families_compiled_equal_physical(family, lx, ly):
    n = lx * ly
    make = circuits.rqc2d_physical if family == "rqc" else circuits.pqc2d_physical
    phys = make(13, lx, ly, 8)
    compiled = circuits2d.compile_layers(lx, ly, circuits.fuse_2d(phys, lx, ly))
    psi = sv.zero_state(n)
    for bonds, us in compiled:
        for b, u in zip(bonds, us):
            psi = sv.apply_two_qubit(psi, n, b, u)
    ref = run_physical_2d(phys, lx, ly)
    assert abs(abs(np.vdot(ref, psi)) - 1) < 1e-12
    assert np.abs(ref - psi).max() < 1e-12


def test_oracle_runs_rqc1d_exactly():
    n, depth = 9, 6
    comp = circuits.rqc1d_circuit(14, n, depth)
    mps = oracle.product_state(n)
    for parity, bonds, gates in comp:
        oracle.apply_layer(mps, gates, parity, chi_max=64, cutoff=1e-12)
    assert sv.fidelity(sv.from_vidal(mps), run_compiled_1d(comp, n)) > 1 - 1e-12


@pytest.mark.parametrize("family", ["haar1d", "rqc1d", "pqc1d", "haar2d", "rqc2d", "pqc2d"])
def test_run_cli_builds_valid_layers(family):
    # the command-line runner's circuits: every layer's bonds are in range and
    # pairwise non-adjacent (a layer of the TEBD procedure)
    from paper_2312_02667_gb300 import run
    args = run.main.__globals__["argparse"].Namespace(family=family, n=11 if family != "pqc1d" else 12, lx=3, ly=4,
                                                      depth=8, seed=2)
    n, layers = run.build_layers(args)
    assert layers
    for bonds, gates in layers:
        bonds = [int(b) for b in bonds]
        assert len(bonds) == len(gates)
        assert all(0 <= b <= n - 2 for b in bonds)
        assert all(c - a >= 2 for a, c in zip(sorted(bonds), sorted(bonds)[1:]))
