"""The QFT workload of App. B on the GPU: a random MPS of bond dimension 10
(the paper's initial state), brought to canonical form by the library's own
PtSU steps, then the QFT line network through ptebd_apply_bonds with g = 0
(the paper's setting).  Untruncated, the result is the exact discrete Fourier
transform of the initial state; truncated, every compiled layer matches the
oracle's layer at the configured cutoff."""
import numpy as np
import pytest

import oracle
from oracle import statevector as sv
from paper_2312_02667_gb300 import inputs, qft

from gpu_helpers import compare_spectra, fidelity, load_into, to_oracle

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
FTOL = {"fp64": 1e-9, "mixed": 1e-6}


@pytest.fixture(scope="module")
def ptebd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02667_gb300 import ptebd as mod
    return mod


def random_vidal(seed, n, chi0):
    """The random MPS of the recipe (entries a + ib, a, b uniform in [-1, 1]) as
    a Vidal object with unit Lambdas: a valid, non-canonical MPS."""
    ms = inputs.random_mps_tensors(seed, n, chi0)
    return oracle.Vidal([np.array(m) for m in ms], [np.ones(m.shape[2]) for m in ms[:-1]])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_qft_of_random_mps_is_the_dft(ptebd, prec):
    n, chi = 12, 64  # chi_max = 2^(N/2): nothing is truncated
    init = random_vidal(21, n, 10)
    psi0 = sv.from_vidal(init)
    x = np.arange(2 ** n)
    target = (np.exp(2j * np.pi * np.outer(x, x) / 2 ** n) / np.sqrt(2 ** n)) @ psi0
    st = ptebd.State(n, chi, prec, cutoff=1e-12)
    load_into(st, init)
    st.canonicalize()
    # PtSU leaves the state and its norm unchanged (Theorem 4's canonical form
    # is reached without truncation here); on this far-from-canonical input
    # (unit Lambdas, random Gamma, norm ~6e4) the complex64 SVDs of the first
    # steps see condition numbers of ~1e3, so the norm is kept to ~1e3 x the
    # FP32 rounding
    canon = sv.from_vidal(to_oracle(st))
    assert sv.fidelity(canon, psi0) >= 1 - FTOL[prec]
    assert abs(np.linalg.norm(canon) / np.linalg.norm(psi0) - 1) < (1e-9 if prec == "fp64" else 1e-4)
    for bonds, gates in qft.qft_line_layers(n):
        st.apply_bonds(bonds, gates)
    got = sv.from_vidal(to_oracle(st))
    f = sv.fidelity(got, target)
    assert f >= 1 - FTOL[prec], f


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_qft_layer_parity_n16_chi16(ptebd, prec):
    # N = 16 (the paper's accuracy test), chi_max = 16: the network truncates;
    # every compiled layer of the GPU path applied to the oracle's state before
    # it, compared with the oracle's layer
    n, chi, cut = 16, 16, 1e-12
    st = ptebd.State(n, chi, prec, cutoff=cut)
    ref = random_vidal(22, n, 10)
    load_into(st, ref)
    st.canonicalize()
    ref = to_oracle(st)
    worst = 0.0
    for t, (bonds, gates) in enumerate(qft.qft_line_layers(n)):
        load_into(st, ref)
        st.apply_bonds(bonds, gates)
        oracle.apply_bonds(ref, bonds, gates, chi, cut)
        got = to_oracle(st)
        for b in bonds:
            compare_spectra(got.lambdas[b], ref.lambdas[b], TOL[prec], cut, chi)
        f = fidelity(got, ref)
        worst = max(worst, 1 - f)
        assert f >= 1 - FTOL[prec], (t, f)
    print(f"{prec}: {qft.qft_depth(n)} compiled layers, worst 1-F {worst:.2e}")
