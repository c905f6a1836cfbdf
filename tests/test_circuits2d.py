"""Compilation of 2D random circuits onto the MPS path (App. A): compiled
depths against the paper's Table I, and the compiled circuit against the
physical one by exact statevector simulation."""
import os

import numpy as np
import pytest

import oracle
from oracle import statevector as sv
from paper_2312_02667_gb300 import circuits2d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table_2d_compiled_depth.txt")


def table_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            rows.append(tuple(int(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("row", table_rows())
def test_compiled_depth_matches_table(row):
    n, lx, ly, phys, compiled = row
    assert n == lx * ly
    # the paper's own count: one compiled layer per A/B layer, 3(Ly - 1) + 2 per C/D pair
    paper_formula = phys // 2 + (phys // 4) * (3 * (ly - 1) + 2)
    ours = circuits2d.compiled_depth(lx, ly, phys)
    assert ours == paper_formula
    if compiled != paper_formula:
        pytest.xfail(f"Table I prints {compiled} for {lx}x{ly}, {phys} layers; the text's "
                     f"3(Ly-1)+2 rule gives {paper_formula}")
    assert ours == compiled


def apply_on_pair(psi, n, p1, p2, u):
    """Apply a 4x4 gate to qubits (p1, p2) (p1 the first factor) of an n-qubit state."""
    t = psi.reshape([2] * n)
    t = np.moveaxis(t, (p1, p2), (0, 1))
    sh = t.shape
    t = (u @ t.reshape(4, -1)).reshape(sh)
    return np.moveaxis(t, (0, 1), (p1, p2)).reshape(-1)


@pytest.mark.parametrize("lx,ly", [(4, 4), (3, 4), (4, 3), (5, 3)])
def test_compiled_circuit_equals_physical(lx, ly):
    n = lx * ly
    layers = circuits2d.physical_layers(3, lx, ly, 8)
    pos = circuits2d.position(lx, ly)
    phys = sv.zero_state(n)
    for kind, gates in layers:
        for q1, q2, u in gates:
            phys = apply_on_pair(phys, n, pos[q1], pos[q2], u)
    comp = sv.zero_state(n)
    compiled = circuits2d.compile_layers(lx, ly, layers)
    for bonds, us in compiled:
        assert all(b2 - b1 >= 2 for b1, b2 in zip(bonds, bonds[1:]))  # one layer = disjoint bonds
        for b, u in zip(bonds, us):
            comp = sv.apply_two_qubit(comp, n, b, u)
    assert len(compiled) == circuits2d.compiled_depth(lx, ly, 8)
    assert abs(np.vdot(phys, comp)) > 1 - 1e-12


def test_oracle_runs_compiled_circuit_exactly():
    lx, ly = 3, 4
    n = lx * ly
    layers = circuits2d.physical_layers(5, lx, ly, 8)
    compiled = circuits2d.compile_layers(lx, ly, layers)
    mps = oracle.product_state(n)
    psi = sv.zero_state(n)
    for bonds, us in compiled:
        oracle.apply_bonds(mps, bonds, us, chi_max=64, cutoff=1e-12)
        for b, u in zip(bonds, us):
            psi = sv.apply_two_qubit(psi, n, b, u)
    assert sv.fidelity(sv.from_vidal(mps), psi) > 1 - 1e-12
