"""The autotuner and the Jacobi block width on the GPU (launch choices of the
library; the paper has no counterpart).  Tuning times candidates on the state's
own next layer and must leave the state exactly as it was; every width must
give the oracle's layer; a given width is bit-identical run to run."""
import numpy as np
import pytest

import oracle
from paper_2312_02667_gb300 import inputs

from gpu_helpers import compare_spectra, fidelity, load_into, to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ptebd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02667_gb300 import ptebd as mod
    return mod


def snapshot(st):
    gam, lam = st.export()
    return [g.copy() for g in gam], [l.copy() for l in lam]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autotune_leaves_the_state_unchanged(ptebd, prec):
    n, chi, depth = 64, 32, 8
    st = ptebd.State(n, chi, prec, cutoff=1e-12, g=1)
    circuit = inputs.brickwork_circuit(41, n, depth + 1)
    for parity, bonds, gates in circuit[:depth]:
        st.apply_layer(gates, parity)
    gam0, lam0 = snapshot(st)
    w0 = st.work_counters()
    _, layers0 = st.svd_sweeps()
    nw, chunks, best_ms, prev_ms, pairs = st.autotune(circuit[depth][2], circuit[depth][0])
    gam1, lam1 = snapshot(st)
    assert all(np.array_equal(a, b) for a, b in zip(gam0, gam1))
    assert all(np.array_equal(a, b) for a, b in zip(lam0, lam1))
    assert st.work_counters() == w0 and st.svd_sweeps()[1] == layers0
    assert nw in ((8, 16) if prec == "mixed" else (8,)) and chunks >= 1 and 0 < best_ms
    assert pairs == 1 or (prec == "mixed" and nw == 16 and pairs == 2)
    assert prev_ms < 0 or best_ms <= prev_ms
    # the tuned handle then runs that layer as the oracle does
    ref = to_oracle(st)
    parity, bonds, gates = circuit[depth]
    st.apply_layer(gates, parity)
    oracle.apply_layer(ref, gates, parity, chi, 1e-12, g=1)
    got = to_oracle(st)
    for b in range(n - 1):
        compare_spectra(got.lambdas[b], ref.lambdas[b], 1e-10 if prec == "fp64" else 1e-5, 1e-12, chi)
    assert fidelity(got, ref) >= 1 - (1e-9 if prec == "fp64" else 1e-6)
    print(f"{prec}: tuned width {nw} x {pairs}, chunks {chunks}: {best_ms:.2f} ms (before: {prev_ms:.2f} ms)")


@pytest.mark.parametrize("nw,pairs", [(8, 1), (16, 1), (16, 2)])
def test_jacobi_width_matches_oracle_and_repeats_bitwise(ptebd, nw, pairs):
    n, chi, depth = 32, 64, 8
    circuit = inputs.brickwork_circuit(43, n, depth)
    ref = oracle.product_state(n)
    st = ptebd.State(n, chi, "mixed", cutoff=1e-12)
    st.set_jacobi_width(nw)
    st.set_jacobi_pairs(pairs)
    for parity, bonds, gates in circuit:
        load_into(st, ref)
        st.apply_layer(gates, parity)
        oracle.apply_layer(ref, gates, parity, chi, 1e-12)
        got = to_oracle(st)
        for b in bonds:
            compare_spectra(got.lambdas[b], ref.lambdas[b], 1e-5, 1e-12, chi)
        assert fidelity(got, ref) >= 1 - 1e-6
    runs = []
    for _ in range(2):
        st.reset()
        for parity, bonds, gates in circuit:
            st.apply_layer(gates, parity)
        runs.append(snapshot(st))
    assert all(np.array_equal(a, b) for a, b in zip(runs[0][0], runs[1][0]))
    assert all(np.array_equal(a, b) for a, b in zip(runs[0][1], runs[1][1]))


@pytest.mark.parametrize("g", [0, 1])
def test_two_columns_per_warp_chi256_matches_oracle(ptebd, g):
    """Two I columns per warp on theta' of 512 x 512 (tSU factors too with g = 1):
    the last two layers of a saturated N = 24, chi = 256 circuit against the
    oracle from the same state, and run-to-run bit identity."""
    n, chi, depth = 24, 256, 10
    circuit = inputs.brickwork_circuit(47, n, depth)
    runs = []
    for _ in range(2):
        st = ptebd.State(n, chi, "mixed", cutoff=1e-12, g=g)
        st.set_jacobi_width(16)
        st.set_jacobi_pairs(2)
        for parity, bonds, gates in circuit[:depth - 2]:
            st.apply_layer(gates, parity)
        ref = to_oracle(st)
        for parity, bonds, gates in circuit[depth - 2:]:
            load_into(st, ref)
            st.apply_layer(gates, parity)
            oracle.apply_layer(ref, gates, parity, chi, 1e-12, g=g)
            got = to_oracle(st)
            for b in range(n - 1):
                compare_spectra(got.lambdas[b], ref.lambdas[b], 1e-5, 1e-12, chi)
            assert fidelity(got, ref) >= 1 - 1e-6
        assert max(len(l) for l in got.lambdas) == chi
        runs.append(snapshot(st))
        st.close()
    assert all(np.array_equal(a, b) for a, b in zip(runs[0][0], runs[1][0]))
    assert all(np.array_equal(a, b) for a, b in zip(runs[0][1], runs[1][1]))


def test_jacobi_pairs_rejects_other_values(ptebd):
    st = ptebd.State(8, 8, "mixed")
    with pytest.raises(ptebd.PtebdError):
        st.set_jacobi_pairs(3)
    st.close()


@pytest.mark.parametrize("mode", [0, 3])
def test_polish_modes_match_oracle(ptebd, mode):
    """Polish sweep off, or on the tSU SVDs only: the layer with its PtSU step
    still matches the oracle to the mixed path's tolerance."""
    n, chi, depth = 32, 64, 8
    circuit = inputs.brickwork_circuit(53, n, depth)
    st = ptebd.State(n, chi, "mixed", cutoff=1e-12, g=1)
    st.set_svd_polish(mode)
    for parity, bonds, gates in circuit[:depth - 1]:
        st.apply_layer(gates, parity)
    ref = to_oracle(st)
    load_into(st, ref)
    parity, bonds, gates = circuit[depth - 1]
    st.apply_layer(gates, parity)
    oracle.apply_layer(ref, gates, parity, chi, 1e-12, g=1)
    got = to_oracle(st)
    for b in range(n - 1):
        compare_spectra(got.lambdas[b], ref.lambdas[b], 1e-5, 1e-12, chi)
    assert fidelity(got, ref) >= 1 - 1e-6
    with pytest.raises(ptebd.PtebdError):
        st.set_svd_polish(4)
    st.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ptsu_shortcut_leaves_the_state_as_the_full_step(ptebd, prec):
    """After a layer on bonds 0, 2, 4, ... the first tSU half-step is the
    identity: with it left out (the default) the state after the layer and its
    PtSU steps matches the oracle, which runs every half-step, and the run with
    it; a parity-1 layer runs every half-step either way (bit-identical)."""
    n, chi, depth = 32, 64, 8
    circuit = inputs.brickwork_circuit(59, n, depth)
    tol, ftol = (1e-10, 1e-9) if prec == "fp64" else (1e-5, 1e-6)
    runs = {}
    for shortcut in (True, False):
        st = ptebd.State(n, chi, prec, cutoff=1e-12, g=2)
        st.set_ptsu_shortcut(shortcut)
        for parity, bonds, gates in circuit[:depth - 2]:
            st.apply_layer(gates, parity)
        ref = to_oracle(st)
        for parity, bonds, gates in circuit[depth - 2:]:
            load_into(st, ref)
            st.apply_layer(gates, parity)
            oracle.apply_layer(ref, gates, parity, chi, 1e-12, g=2)
            got = to_oracle(st)
            for b in range(n - 1):
                compare_spectra(got.lambdas[b], ref.lambdas[b], tol, 1e-12, chi)
            assert fidelity(got, ref) >= 1 - ftol
        runs[shortcut] = to_oracle(st)
        st.close()
    assert fidelity(runs[True], runs[False]) >= 1 - ftol
    # a parity-1 layer: the same launches with or without the shortcut
    start = runs[True]
    parity, bonds, gates = circuit[5]
    assert parity == 1
    snaps = []
    for shortcut in (True, False):
        st = ptebd.State(n, chi, prec, cutoff=1e-12, g=1)
        st.set_ptsu_shortcut(shortcut)
        load_into(st, start)
        st.apply_layer(gates, parity)
        snaps.append(snapshot(st))
        st.close()
    assert all(np.array_equal(a, b) for a, b in zip(snaps[0][0], snaps[1][0]))
    assert all(np.array_equal(a, b) for a, b in zip(snaps[0][1], snaps[1][1]))
