"""Batched serving: many independent states advanced by one graph launch per
layer must give exactly what the same states give one by one, and match the
oracle."""
import numpy as np
import pytest

import oracle
from paper_2312_02667_gb300 import inputs

from gpu_helpers import compare_spectra, fidelity, to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ptebd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02667_gb300 import ptebd as mod
    return mod


def test_batch_equals_one_by_one(ptebd):
    specs = [(10, 4, "fp64", 0), (23, 8, "mixed", 1), (40, 16, "mixed", 0), (17, 32, "fp64", 1),
             (31, 16, "mixed", 1), (12, 8, "mixed", 0)]
    depth = [6, 9, 7, 8, 5, 9]
    solo = [ptebd.State(n, c, p, g=g) for n, c, p, g in specs]
    grouped = [ptebd.State(n, c, p, g=g, workspace_bytes=1 if i % 2 else None) for i, (n, c, p, g) in enumerate(specs)]
    circuits = [inputs.brickwork_circuit(100 + i, n, depth[i], circuit=i) for i, (n, _, _, _) in enumerate(specs)]
    batch = ptebd.Batch(grouped)
    for layer in range(max(depth)):
        gl, par = [], []
        for i in range(len(specs)):
            if layer < depth[i]:
                parity, bonds, gates = circuits[i][layer]
                solo[i].apply_layer(gates, parity)
                gl.append(gates)
                par.append(parity)
            else:
                gl.append(None)
                par.append(-1)
        batch.apply_layer(gl, par)
    for i, (n, _, _, _) in enumerate(specs):
        for s in range(n):
            assert np.array_equal(solo[i].site(s), grouped[i].site(s)), (i, s)
        for b in range(n - 1):
            assert np.array_equal(solo[i].lam(b), grouped[i].lam(b))
        assert grouped[i].svd_sweeps()[1] == depth[i]
    batch.close()


def test_uneven_circuits_against_oracle(ptebd):
    # a reduced version of the batched-serving workload: uneven N, depth and
    # chi_max, Haar gates, one graph launch per layer; oracle on every circuit
    rng = np.random.default_rng(5)
    k = 8
    ns = rng.integers(20, 61, k)
    ds = rng.integers(4, 11, k)
    chis = rng.choice([8, 16, 32], k)
    states = [ptebd.State(int(ns[i]), int(chis[i]), "mixed") for i in range(k)]
    refs = [oracle.product_state(int(ns[i])) for i in range(k)]
    circuits = [inputs.brickwork_circuit(200 + i, int(ns[i]), int(ds[i]), circuit=i) for i in range(k)]
    batch = ptebd.Batch(states)
    for layer in range(int(ds.max())):
        gl, par = [], []
        for i in range(k):
            if layer < ds[i]:
                parity, bonds, gates = circuits[i][layer]
                oracle.apply_layer(refs[i], gates, parity, int(chis[i]), 1e-12)
                gl.append(gates)
                par.append(parity)
            else:
                gl.append(None)
                par.append(-1)
        batch.apply_layer(gl, par)
    for i in range(k):
        got = to_oracle(states[i])
        for b in range(int(ns[i]) - 1):
            compare_spectra(got.lambdas[b], refs[i].lambdas[b], 1e-5, 1e-12, int(chis[i]))
        assert fidelity(got, refs[i]) >= 1 - int(ds[i]) * 1e-6
    batch.close()


def test_batched_serving_64_circuits_sampled_bonds(ptebd):
    # The batched-serving configuration at full size: 64 independent circuits,
    # N ~ U[50, 500], depth ~ U[8, 24], chi_max in {32, 64, 128, 256}, Haar
    # gates, mixed precision, one graph launch per layer for all of them.  Each
    # circuit's last layer is checked on sampled bonds against the oracle's
    # single-bond update of the same inputs (read back just before that layer).
    from gpu_helpers import mini_vidal
    rng = np.random.default_rng(64)
    k = 64
    ns = rng.integers(50, 501, k)
    ds = rng.integers(8, 25, k)
    chis = rng.choice([32, 64, 128, 256], k)
    states = [ptebd.State(int(ns[i]), int(chis[i]), "mixed") for i in range(k)]
    circuits_ = [inputs.brickwork_circuit(300 + i, int(ns[i]), int(ds[i]), circuit=i) for i in range(k)]
    batch = ptebd.Batch(states)
    checks = {}
    for layer in range(int(ds.max())):
        gl, par = [], []
        for i in range(k):
            if layer < ds[i]:
                parity, bonds, gates = circuits_[i][layer]
                if layer == ds[i] - 1:  # the last layer of circuit i: snapshot sampled bonds first
                    n = int(ns[i])
                    pick = sorted(rng.choice(len(bonds), min(3, len(bonds)), replace=False))
                    snap = []
                    for j in pick:
                        b = int(bonds[j])
                        st = states[i]
                        snap.append((b, gates[j], st.lam(b - 1) if b > 0 else np.ones(1), st.site(b), st.lam(b),
                                     st.site(b + 1), st.lam(b + 1) if b + 1 < n - 1 else np.ones(1)))
                    checks[i] = snap
                gl.append(gates)
                par.append(parity)
            else:
                gl.append(None)
                par.append(-1)
        batch.apply_layer(gl, par)
    assert len(checks) == k
    for i in range(k):
        chi = int(chis[i])
        eps_g, _, _ = states[i].bond_stats()
        for b, u, ll, gb, lb, gb1, lr in checks[i]:
            mini = mini_vidal(ll, gb, lb, gb1, lr)
            r = oracle.update_bond(mini, 1, u, chi, 1e-12)
            compare_spectra(states[i].lam(b), mini.lambdas[1], 1e-5, 1e-12, chi)
            assert abs(eps_g[b] - r.eps) <= 1e-5 * max(r.eps, 1e-3)
    batch.close()


def test_batch_with_chunked_states(ptebd):
    # states large enough to run their layers in concurrent chunks, recorded
    # into the batch graph, against the same states on one stream each
    specs = [(256, 16), (130, 8), (200, 12)]
    grouped = [ptebd.State(n, c, "mixed", g=1) for n, c in specs]
    solo = [ptebd.State(n, c, "mixed", g=1) for n, c in specs]
    for s in solo:
        s.set_chunk_streams(1)
    circuits_ = [inputs.brickwork_circuit(500 + i, n, 6, circuit=i) for i, (n, _) in enumerate(specs)]
    batch = ptebd.Batch(grouped)
    for layer in range(6):
        batch.apply_layer([circuits_[i][layer][2] for i in range(3)], [circuits_[i][layer][0] for i in range(3)])
        for i in range(3):
            solo[i].apply_layer(circuits_[i][layer][2], circuits_[i][layer][0])
    for i, (n, _) in enumerate(specs):
        for s in range(n):
            assert np.array_equal(grouped[i].site(s), solo[i].site(s)), (i, s)
    batch.close()
