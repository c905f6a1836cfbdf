"""The FP64 resolution of the mixed path against the oracle at the configured cutoff.

A complex64 spectrum cannot tell values below about 1e-7 sigma_1 from exact
zeros.  The mixed path therefore decides a bond's kept count (Sec. III B, the
projector P_i with the cutoff) from its complex64 spectrum only when that count
does not depend on values below resolve * sigma_1 (taken as real or as zero,
with rank(theta') <= rank(gate) chi_b); every other bond is recomputed in FP64
from the stored Gamma.  These tests use circuits whose Schmidt spectra fall off
through the unresolvable range (Trotter steps of a Heisenberg chain, the
near-identity gates of a time evolution), where the resolution has to act,
and compare every layer with the complex128 oracle at cutoff 1e-12: singular
values normwise to 1e-5 sigma_1, fidelity >= 1 - 1e-6, bond dimensions equal
wherever the oracle's values are above 1e-5 sigma_1 (the comparison rule of
compare_spectra).
"""
import numpy as np
import pytest

import oracle
from paper_2312_02667_gb300 import inputs

from gpu_helpers import compare_spectra, fidelity, load_into, to_oracle

pytestmark = pytest.mark.gpu

CUT = 1e-12


@pytest.fixture(scope="module")
def ptebd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02667_gb300 import ptebd as mod
    return mod


@pytest.mark.parametrize("g", [0, 1])
def test_trotter_layers_resolve_in_fp64(ptebd, g):
    n, chi, depth, dt = 20, 32, 16, 0.1
    st = ptebd.State(n, chi, "mixed", cutoff=CUT, g=g)
    ref = oracle.product_state(n)
    worst_dev, worst_f, resolved = 0.0, 0.0, 0
    for layer, (parity, bonds, gates) in enumerate(inputs.trotter_heisenberg_circuit(5, n, depth, dt)):
        load_into(st, ref)
        w0 = st.work_counters()
        st.apply_layer(gates, parity)
        resolved += st.work_counters()[8] - w0[8]
        oracle.apply_layer(ref, gates, parity, chi, CUT, g=g)
        got = to_oracle(st)
        for b in range(n - 1):
            worst_dev = max(worst_dev, compare_spectra(got.lambdas[b], ref.lambdas[b], 1e-5, CUT, chi))
        f = fidelity(got, ref)
        worst_f = max(worst_f, 1 - f)
        assert f >= 1 - 1e-6, (layer, f)
    # the spectra reach below what complex64 resolves: the FP64 pass must have run
    assert resolved > 0
    print(f"g={g}: {resolved} bond updates resolved in FP64, worst normwise dev {worst_dev:.2e}, "
          f"worst 1-F {worst_f:.2e}, final chi {st.chi().tolist()}")


def test_trotter_circuit_cumulative_matches_oracle(ptebd):
    # the whole circuit on both sides from |0...0>: the bond dimensions the
    # cutoff keeps agree exactly, and the states agree to well inside 1e-6 per layer
    n, chi, depth, dt = 20, 32, 16, 0.1
    st = ptebd.State(n, chi, "mixed", cutoff=CUT)
    ref = oracle.product_state(n)
    for parity, bonds, gates in inputs.trotter_heisenberg_circuit(6, n, depth, dt):
        st.apply_layer(gates, parity)
        oracle.apply_layer(ref, gates, parity, chi, CUT)
    got = to_oracle(st)
    diff = [b for b in range(n - 1) if len(got.lambdas[b]) != len(ref.lambdas[b])]
    for b in diff:  # a count may differ only by values the tolerance cannot see
        compare_spectra(got.lambdas[b], ref.lambdas[b], 1e-5, CUT, chi)
    assert fidelity(got, ref) >= 1 - depth * 1e-6
    counts = st.work_counters()
    print(f"bond dims differing from the oracle: {diff}; bonds resolved in FP64: {counts[8]}")


def test_without_resolution_complex64_noise_is_kept(ptebd):
    # the same circuit with the resolution off (resolve <= cutoff): the
    # complex64 spectrum alone decides, and its rounding noise (about 1e-7
    # sigma_1) is kept as singular values above the cutoff 1e-12, so bond
    # dimensions grow past the oracle's.  This is what the resolution prevents.
    # (summed over the layers: once chi_max binds everywhere the difference is gone)
    n, chi, depth, dt = 20, 32, 16, 0.1
    plain = ptebd.State(n, chi, "mixed", cutoff=CUT, resolve=0.0)
    res = ptebd.State(n, chi, "mixed", cutoff=CUT)
    ref = oracle.product_state(n)
    s_ref = s_plain = s_res = 0
    for parity, bonds, gates in inputs.trotter_heisenberg_circuit(6, n, depth, dt):
        plain.apply_layer(gates, parity)
        res.apply_layer(gates, parity)
        oracle.apply_layer(ref, gates, parity, chi, CUT)
        s_ref += sum(len(l) for l in ref.lambdas)
        s_plain += int(np.sum(plain.chi()))
        s_res += int(np.sum(res.chi()))
    print(f"chi summed over bonds and layers: oracle {s_ref}, resolved {s_res}, complex64 alone {s_plain}")
    assert plain.work_counters()[8] == 0
    assert s_plain > s_ref
    assert abs(s_res - s_ref) < abs(s_plain - s_ref)


def test_structural_rank_decides_cz_layers_in_complex64(ptebd):
    # CZ-type gates have operator Schmidt rank 2: theta' has rank <= 2 chi_b, so
    # its other singular values are exact zeros and the complex64 pass decides
    # the bond without FP64 whenever the 2 chi_b nonzero values are resolved
    from paper_2312_02667_gb300 import circuits
    n, chi, depth = 25, 16, 12  # RQC-1D takes an odd number of qubits
    st = ptebd.State(n, chi, "mixed", cutoff=CUT)
    ref = oracle.product_state(n)
    gated = 0
    for parity, bonds, gates in circuits.rqc1d_circuit(3, n, depth):
        load_into(st, ref)
        st.apply_bonds(bonds, gates)
        oracle.apply_bonds(ref, bonds, gates, chi, CUT)
        got = to_oracle(st)
        gated += len(bonds)
        for b in bonds:
            compare_spectra(got.lambdas[b], ref.lambdas[b], 1e-5, CUT, chi)
        assert fidelity(got, ref) >= 1 - 1e-6
    resolved = st.work_counters()[8]
    print(f"RQC-1D (CZ): {resolved} of {gated} gated bond updates resolved in FP64")
    assert resolved < gated // 4


def test_resolution_inside_batch_graphs(ptebd):
    # In the batch graphs the FP64 pass is an IF node switched on by the
    # complex64 truncation; states run there must be bit-identical to the same
    # states run one by one (FP64 pass launched directly), with the same
    # number of bonds recomputed in FP64, which must not be zero here
    n, chi, depth, dt = 20, 32, 12, 0.1
    circuits = [inputs.trotter_heisenberg_circuit(20 + i, n, depth, dt) for i in range(3)]
    solo = [ptebd.State(n, chi, "mixed", cutoff=CUT) for _ in circuits]
    for st, circ in zip(solo, circuits):
        for parity, bonds, gates in circ:
            st.apply_layer(gates, parity)
    batched = [ptebd.State(n, chi, "mixed", cutoff=CUT) for _ in circuits]
    batch = ptebd.Batch(batched)
    for layer in range(depth):
        batch.apply_layer([c[layer][2] for c in circuits], [c[layer][0] for c in circuits])
    batch.close()
    for a, b in zip(solo, batched):
        ga, la = a.export()
        gb, lb = b.export()
        assert all(np.array_equal(x, y) for x, y in zip(ga, gb))
        assert all(np.array_equal(x, y) for x, y in zip(la, lb))
        assert a.work_counters()[8] == b.work_counters()[8] > 0
