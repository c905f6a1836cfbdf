"""GPU parity tests: the CUDA path (through the C ABI) against the oracle.

Tolerances (fixed by the target of this project): singular values normwise
to 1e-10 * lambda_1 on the FP64 path and 1e-5 * lambda_1 on the mixed path;
state fidelity per layer >= 1 - 1e-9 (FP64) and >= 1 - 1e-6 (mixed).
Gauge-dependent tensors are never compared elementwise: only Lambda, chi,
eps, nu and fidelities, which the method fixes uniquely.
"""
import numpy as np
import pytest

import oracle
from oracle import statevector as sv
from paper_2312_02667_gb300 import inputs

from gpu_helpers import compare_spectra, fidelity, load_into, mini_vidal, to_oracle

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


def thr(st_prec, cutoff=1e-12):
    """The oracle's truncation threshold for a state of precision st_prec: the
    configured cutoff on both paths (the mixed path resolves in FP64 every bond
    whose kept count its complex64 spectrum cannot decide)."""
    return cutoff


# ----------------------------------------------------- exact (no truncation)

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_untruncated_circuit_matches_statevector(ptebd, prec):
    n, depth = 12, 10
    st = ptebd.State(n, 64, prec, cutoff=1e-12)
    psi = sv.zero_state(n)
    for parity, bonds, gates in inputs.brickwork_circuit(3, n, depth):
        st.apply_layer(gates, parity)
        for b, u in zip(bonds, gates):
            psi = sv.apply_two_qubit(psi, n, int(b), u)
        mps = to_oracle(st)
        f = sv.fidelity(sv.from_vidal(mps), psi)
        assert f >= 1 - FTOL[prec], f
        for b in range(n - 1):
            ref = sv.schmidt_values(psi, n, b)
            ref = ref[ref > thr(prec) * ref[0]]
            compare_spectra(mps.lambdas[b], ref, TOL[prec], thr(prec), 64)
    eps, lognu = st.trunc_error()
    assert eps < 1e-10 and abs(lognu) < 1e-10


def test_c1_config_n16_depth10_chi256(ptebd):
    # N = 16, depth 10, chi_max = 256: no truncation, complex128, vs the 2^16 statevector
    n, depth = 16, 10
    st = ptebd.State(n, 256, "fp64", cutoff=1e-12)
    psi = sv.zero_state(n)
    for parity, bonds, gates in inputs.brickwork_circuit(0, n, depth):
        st.apply_layer(gates, parity)
        for b, u in zip(bonds, gates):
            psi = sv.apply_two_qubit(psi, n, int(b), u)
    mps = to_oracle(st)
    assert sv.fidelity(sv.from_vidal(mps), psi) >= 1 - 1e-9
    for b in range(n - 1):
        ref = sv.schmidt_values(psi, n, b)
        ref = ref[ref > 1e-12 * ref[0]]
        compare_spectra(mps.lambdas[b], ref, 1e-10, 1e-12, 256)
    assert oracle.distance_to_canonical(mps) < 1e-9


# ------------------------------------------------------- one-layer parity --

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_layer_parity_n128_chi64(ptebd, prec):
    # N = 128, depth 20, chi_max = 64: every layer of the GPU path applied to
    # the oracle's own state before that layer, compared with the oracle's layer.
    n, chi, depth = 128, 64, 20
    cut = thr(prec)
    st = ptebd.State(n, chi, prec, cutoff=1e-12)
    ref = oracle.product_state(n)
    worst_dev, worst_f = 0.0, 0.0
    for layer, (parity, bonds, gates) in enumerate(inputs.brickwork_circuit(1, n, depth)):
        load_into(st, ref)
        st.apply_layer(gates, parity)
        res = oracle.apply_layer(ref, gates, parity, chi, cut)
        got = to_oracle(st)
        eps_g, nu_g, rank_g = st.bond_stats()
        for r in res.bonds:
            b = r.bond
            worst_dev = max(worst_dev, compare_spectra(got.lambdas[b], ref.lambdas[b], TOL[prec], cut, chi))
            # the cutoff 1e-12 keeps the same number of values on both paths
            assert len(got.lambdas[b]) == len(ref.lambdas[b]), (layer, b, len(got.lambdas[b]), len(ref.lambdas[b]))
            assert abs(eps_g[b] - r.eps) <= TOL[prec] * max(1.0, r.eps) + 1e-14
            assert abs(nu_g[b] - r.nu) <= 2 * TOL[prec]
            assert rank_g[b] == r.rank_in
        f = fidelity(got, ref)
        worst_f = max(worst_f, 1 - f)
        assert f >= 1 - FTOL[prec], (layer, f)
    sweeps, layers = st.svd_sweeps()
    assert layers == depth and sweeps.max() < 40
    print(f"{prec}: worst normwise lambda deviation {worst_dev:.2e}, worst 1-F {worst_f:.2e}, "
          f"bonds resolved in FP64 {st.work_counters()[8]}")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cumulative_circuit_n128_chi64(ptebd, prec):
    n, chi, depth = 128, 64, 20
    st = ptebd.State(n, chi, prec, cutoff=1e-12)
    ref = oracle.product_state(n)
    for parity, bonds, gates in inputs.brickwork_circuit(2, n, depth):
        st.apply_layer(gates, parity)
        oracle.apply_layer(ref, gates, parity, chi, thr(prec))
    f = fidelity(to_oracle(st), ref)
    # twenty truncated layers: errors add up but stay far below the truncation error
    assert f >= 1 - 20 * FTOL[prec], f
    e_g, l_g = st.trunc_error()
    assert e_g > 0.0


def test_mixed_against_fp64_on_the_gpu(ptebd):
    n, chi, depth = 64, 32, 14
    a = ptebd.State(n, chi, "fp64")
    b = ptebd.State(n, chi, "mixed")
    for parity, bonds, gates in inputs.brickwork_circuit(4, n, depth):
        a.apply_layer(gates, parity)
        b.apply_layer(gates, parity)
        f = fidelity(to_oracle(a), to_oracle(b))
        assert f >= 1 - 1e-5, f


# --------------------------------------------------------------- regauge --

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ptsu_parity_and_theorem_4(ptebd, prec):
    n = 12
    mps = oracle.canonicalize(inputs.random_mps_tensors(5, n, 16))
    cut = oracle.scale_to_unit_norm(oracle.truncate_all_bonds(mps, 8))
    st = ptebd.State(n, 16, prec, cutoff=1e-14)
    load_into(st, cut)
    ref = cut.copy()
    st.regauge(1)
    oracle.ptsu_step(ref, 16, thr(prec, 1e-14))
    got = to_oracle(st)
    for b in range(n - 1):
        compare_spectra(got.lambdas[b], ref.lambdas[b], TOL[prec], thr(prec, 1e-14), 16)
    assert fidelity(got, cut) >= 1 - FTOL[prec]
    st.regauge(n // 2 - 1)
    c = oracle.distance_to_canonical(to_oracle(st))
    # Theorem 4: C = 0 after N/2 steps in exact arithmetic.  The floor in
    # floating point is set by the SVD's orthogonality threshold: the Jacobi
    # leaves |a^H b| <= k sqrt(m) u |a||b| (k = 8 in FP32, 4 in FP64), so each
    # chi x chi block of sum A^dag A - I has off-diagonal entries of that size
    # and a Frobenius norm of about chi * k sqrt(m) u (m = 2 chi rows).
    floor = 4 * 16 * 8 * np.sqrt(32) * 2.0 ** -24 if prec == "mixed" else 1e-10
    assert c < floor, (c, floor)


def test_fp64_regauge_of_a_mixed_state(ptebd):
    # The PtSU steps of a complex64 state run in FP64 (ptebd_set_regauge_precision):
    # each tSU is the FP64 computation on the stored complex64 Gamma, so one step
    # matches the oracle to FP32-rounding level, and after N/2 steps (Theorem 4)
    # the distance to canonical form is limited only by the complex64 storage of
    # Gamma: |sum A^dag A - I|_F <= about 2 u chi (u = 2^-24), far below the
    # complex64 Jacobi's floor of the test above.
    n, chi = 12, 16
    mps = oracle.canonicalize(inputs.random_mps_tensors(5, n, 16))
    cut = oracle.scale_to_unit_norm(oracle.truncate_all_bonds(mps, 8))
    st = ptebd.State(n, chi, "mixed", cutoff=1e-14)
    st.set_regauge_precision("fp64")
    load_into(st, cut)
    ref = cut.copy()
    w0 = st.work_counters()
    st.regauge(1)
    oracle.ptsu_step(ref, chi, 1e-14)
    got = to_oracle(st)
    assert st.work_counters()[8] - w0[8] == n - 1  # every tSU bond ran in FP64
    for b in range(n - 1):
        compare_spectra(got.lambdas[b], ref.lambdas[b], 1e-6, 1e-14, chi)
    assert fidelity(got, cut) >= 1 - 1e-9
    st.regauge(n // 2 - 1)
    c = oracle.distance_to_canonical(to_oracle(st))
    floor = 4 * chi * 2.0 ** -24
    print(f"C after N/2 FP64 PtSU steps of a complex64 state: {c:.2e} (bound {floor:.2e})")
    assert c < floor, (c, floor)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_layer_with_ptsu_g1(ptebd, prec):
    n, chi = 40, 16
    st = ptebd.State(n, chi, prec, g=1)
    ref = oracle.product_state(n)
    for parity, bonds, gates in inputs.brickwork_circuit(6, n, 10):
        load_into(st, ref)
        st.apply_layer(gates, parity)
        res = oracle.apply_layer(ref, gates, parity, chi, thr(prec), g=1)
        got = to_oracle(st)
        for b in range(n - 1):
            compare_spectra(got.lambdas[b], ref.lambdas[b], TOL[prec], thr(prec), chi)
        assert fidelity(got, ref) >= 1 - FTOL[prec]


@pytest.mark.parametrize("prec,k", [("mixed", 24), ("mixed", -24), ("fp64", 24)])
def test_layer_parity_far_from_unit_norm(ptebd, prec, k):
    # Every Lambda times 2^k: theta' = U Lambda Gamma Lambda Gamma Lambda grows
    # by 2^(3k), past what FP32 squared norms and |a^H b|^2 can hold for k = 24
    # (and below their normal range for k = -24).  The method is homogeneous in
    # this scale (relative truncation, eps and nu unchanged, every Lambda_b of the
    # layer scaled alike), so the layer must match the oracle as at unit scale.
    n, chi = 14, 16
    mps = oracle.canonicalize(inputs.random_mps_tensors(21, n, chi))
    mps.lambdas = [l * 2.0 ** k for l in mps.lambdas]
    st = ptebd.State(n, chi, prec, g=1)
    for parity, bonds, gates in inputs.brickwork_circuit(22, n, 3):
        load_into(st, mps)
        st.apply_layer(gates, parity)
        oracle.apply_layer(mps, gates, parity, chi, thr(prec), g=1)
        got = to_oracle(st)
        for b in range(n - 1):
            compare_spectra(got.lambdas[b], mps.lambdas[b], TOL[prec], thr(prec), chi)
        # the fidelity of the states scaled to unit norm (their own norms are
        # far outside what the FP64 overlap of the helper can square)
        assert fidelity(oracle.scale_to_unit_norm(got), oracle.scale_to_unit_norm(mps)) >= 1 - FTOL[prec]


@pytest.mark.parametrize("mode", ["schmidt", "relative", "absolute"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_eps_readings_match_oracle(ptebd, prec, mode):
    # A Vidal MPS far from the canonical form (random Gammas, graded Lambdas),
    # where the three readings of the stabilisation differ: one layer each.
    n, chi = 12, 8
    ts = [np.asarray(t) for t in inputs.random_mps_tensors(31, n, 8)]
    # (the absolute reading needs eps_b < 1: smaller Lambdas there)
    top = 0.6 if mode == "absolute" else 1.5
    raw = oracle.Vidal(ts, [np.linspace(top, 0.2 * top, ts[b].shape[2]) for b in range(n - 1)])
    parity, bonds, gates = inputs.brickwork_layer(31, n, 0)
    st = ptebd.State(n, chi, prec, eps_mode=mode)
    load_into(st, raw)
    st.apply_layer(gates, parity)
    ref = raw.copy()
    res = oracle.apply_layer(ref, gates, parity, chi, thr(prec), eps_mode=mode)
    got = to_oracle(st)
    eps_g, nu_g, _ = st.bond_stats()
    for r in res.bonds:
        compare_spectra(got.lambdas[r.bond], ref.lambdas[r.bond], TOL[prec], thr(prec), chi)
        assert abs(eps_g[r.bond] - r.eps) <= 10 * TOL[prec] * max(r.eps, 1e-3)
    assert fidelity(got, ref) >= 1 - FTOL[prec]


# ---------------------------------------------------------- measurements --

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_norm_overlap_expect(ptebd, prec):
    n, chi = 20, 16
    st = ptebd.State(n, chi, prec)
    st2 = ptebd.State(n, chi, prec)
    for parity, bonds, gates in inputs.brickwork_circuit(7, n, 10):
        st.apply_layer(gates, parity)
    for parity, bonds, gates in inputs.brickwork_circuit(8, n, 7):
        st2.apply_layer(gates, parity)
    a, b = to_oracle(st), to_oracle(st2)
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert abs(st.norm() - oracle.norm(a)) < tol
    assert abs(st.overlap(st2) - oracle.overlap(a, b)) < tol
    op = inputs.random_one_site_op(2)
    for j in (0, 7, n - 1):
        assert abs(st.expect(j, op) - oracle.expect_one_site(a, j, op)) < tol
    op2 = inputs.haar_u4(np.random.default_rng(1))
    for j in (0, 9, n - 2):
        assert abs(st.expect2(j, op2) - oracle.expect_two_site(a, j, op2)) < tol


def test_norm_tracks_nu_stabilisation(ptebd):
    # n* = n prod nu (Sec. III C): the device's running log prod nu against
    # the state norm after a truncated layer on a canonical state
    n = 12
    mps = oracle.canonicalize(inputs.random_mps_tensors(9, n, 6))
    st = ptebd.State(n, 6, "fp64")
    load_into(st, mps)
    parity, bonds, gates = inputs.brickwork_layer(9, n, 1)
    st.apply_layer(gates, parity)
    eps, lognu = st.trunc_error()
    n_star = st.norm()
    n_plain = n_star * np.exp(-lognu)
    assert eps > 1e-3
    assert 1 - np.sqrt(2 * eps) - 1e-12 <= n_plain <= 1 + 1e-12
    assert (1 - np.sqrt(2 * eps)) * np.exp(lognu) - 1e-12 <= n_star <= np.exp(lognu) + 1e-12


# ------------------------------------------------------- full-size sample --

def test_sampled_bonds_n1024_chi256_mixed(ptebd):
    # The bench workload (N = 1024, chi_max = 256, mixed precision, PtSU after
    # every layer): run to saturation, then compare 16 sampled bonds of one
    # gate layer with the oracle's single-bond update on the same inputs.
    n, chi = 1024, 256
    st = ptebd.State(n, chi, "mixed", cutoff=1e-12, g=0)
    circuit = inputs.brickwork_circuit(0, n, 11)
    for parity, bonds, gates in circuit[:10]:
        st.apply_layer(gates, parity)
        st.regauge(1)
    parity, bonds, gates = circuit[10]
    rng = np.random.default_rng(0)
    pick = sorted(rng.choice(len(bonds), 16, replace=False))
    pick[0] = 0  # the open boundary bond
    before = {}
    for j in pick:
        b = int(bonds[j])
        before[j] = (st.lam(b - 1) if b > 0 else np.ones(1), st.site(b), st.lam(b), st.site(b + 1),
                     st.lam(b + 1) if b + 1 < n - 1 else np.ones(1))
    st.apply_layer(gates, parity)
    eps_g, nu_g, _ = st.bond_stats()
    assert st.chi().max() == chi  # saturated
    for j in pick:
        b = int(bonds[j])
        ll, gb, lb, gb1, lr = before[j]
        mini = mini_vidal(ll, gb, lb, gb1, lr)
        r = oracle.update_bond(mini, 1, gates[j], chi, thr("mixed"))
        lam_g = st.lam(b)
        compare_spectra(lam_g, mini.lambdas[1], TOL["mixed"], thr("mixed"), chi)
        assert abs(eps_g[b] - r.eps) <= 1e-5 * max(r.eps, 1e-3)
        got = mini_vidal(ll, st.site(b), lam_g, st.site(b + 1), lr)
        th_g = oracle.two_site_tensor(got, 1).reshape(-1)
        th_o = oracle.two_site_tensor(mini, 1).reshape(-1)
        f = abs(np.vdot(th_o, th_g)) ** 2 / (np.vdot(th_o, th_o).real * np.vdot(th_g, th_g).real)
        assert f >= 1 - FTOL["mixed"], (b, f)


# ------------------------------------------------------------ edge cases --

def test_edge_cases(ptebd):
    # two sites, one bond; parity 1 has no bonds at all
    st = ptebd.State(2, 4, "fp64")
    u = inputs.haar_u4(np.random.default_rng(3))
    st.apply_layer(u[None], 0)
    st.apply_layer(np.zeros((0, 4, 4), complex), 1)
    ref = oracle.product_state(2)
    oracle.apply_layer(ref, [u], 0, 4, 1e-12)
    compare_spectra(st.lam(0), ref.lambdas[0], 1e-12, 1e-12, 4)
    # chi_max = 1: every gated bond is cut back to a product state
    n = 9
    st = ptebd.State(n, 1, "fp64")
    ref = oracle.product_state(n)
    for parity, bonds, gates in inputs.brickwork_circuit(5, n, 4):
        st.apply_layer(gates, parity)
        oracle.apply_layer(ref, gates, parity, 1, 1e-12)
    assert (st.chi() == 1).all()
    assert fidelity(to_oracle(st), ref) >= 1 - 1e-9
    # overlapping bonds, bad parity, out-of-range bond
    st = ptebd.State(8, 4, "fp64")
    with pytest.raises(ptebd.PtebdError) as e:
        st.apply_bonds([2, 3], np.stack([u, u]))
    assert e.value.code == -5
    with pytest.raises(ptebd.PtebdError) as e:
        ptebd.ptebd_apply_layer(st.handle, np.stack([u] * 4), 2)
    assert e.value.code == -1
    with pytest.raises(ptebd.PtebdError):
        st.apply_bonds([7], u[None])
    # an empty sparse layer is a no-op; reset goes back to |0...0>
    st.apply_bonds([], np.zeros((0, 4, 4), complex))
    st.apply_bonds([1, 4], np.stack([u, u]))
    assert st.chi()[1] > 1
    st.reset()
    assert (st.chi() == 1).all() and abs(st.norm() - 1) < 1e-14


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_chunked_workspace_is_bit_identical(ptebd, prec):
    n, chi = 33, 16
    full = ptebd.State(n, chi, prec)
    small = ptebd.State(n, chi, prec, workspace_bytes=1)  # one bond per chunk
    assert small.workspace_bytes < full.workspace_bytes
    for parity, bonds, gates in inputs.brickwork_circuit(11, n, 9):
        full.apply_layer(gates, parity)
        small.apply_layer(gates, parity)
    for s in range(n):
        assert np.array_equal(full.site(s), small.site(s))
    for b in range(n - 1):
        assert np.array_equal(full.lam(b), small.lam(b))


def test_sparse_bonds_match_oracle(ptebd):
    n, chi = 14, 16
    st = ptebd.State(n, chi, "fp64")
    ref = oracle.product_state(n)
    rng = np.random.default_rng(12)
    for layer in range(12):
        bonds = sorted(rng.choice(np.arange(0, n - 1, 3), 3, replace=False) + (layer % 3))
        bonds = [b for b in bonds if b <= n - 2]
        gates = np.stack([inputs.haar_u4(rng) for _ in bonds])
        st.apply_bonds(bonds, gates)
        oracle.apply_bonds(ref, bonds, gates, chi, 1e-12)
    got = to_oracle(st)
    for b in range(n - 1):
        compare_spectra(got.lambdas[b], ref.lambdas[b], 1e-10, 1e-12, chi)
    assert fidelity(got, ref) >= 1 - 1e-9


def test_device_gates(ptebd):
    import torch
    n, chi = 20, 8
    a = ptebd.State(n, chi, "mixed")
    b = ptebd.State(n, chi, "mixed")
    for parity, bonds, gates in inputs.brickwork_circuit(13, n, 6):
        a.apply_layer(gates, parity)
        b.apply_layer(torch.from_numpy(gates).to("cuda"), parity)
    for s in range(n):
        assert np.array_equal(a.site(s), b.site(s))


# ------------------------------------------------------- 2D routed circuits --

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_routed_2d_circuit_against_oracle(ptebd, prec):
    # a 4x4 lattice, ABCD x 2 with Haar gates, compiled onto the path with
    # SWAP networks (App. A); every compiled layer through ptebd_apply_bonds
    from paper_2312_02667_gb300 import circuits2d
    lx, ly, chi = 4, 4, 16
    compiled = circuits2d.compile_layers(lx, ly, circuits2d.physical_layers(2, lx, ly, 8))
    # every compiled layer from the oracle's state (the layer's own parity),
    # then the whole circuit on the GPU alone against the oracle's trajectory
    st = ptebd.State(lx * ly, chi, prec)
    ref = oracle.product_state(lx * ly)
    for bonds, us in compiled:
        load_into(st, ref)
        st.apply_bonds(bonds, us)
        oracle.apply_bonds(ref, bonds, us, chi, thr(prec))
        got = to_oracle(st)
        for b in range(lx * ly - 1):
            compare_spectra(got.lambdas[b], ref.lambdas[b], TOL[prec], thr(prec), chi)
        assert fidelity(got, ref) >= 1 - FTOL[prec]
    st2 = ptebd.State(lx * ly, chi, prec)
    for bonds, us in compiled:
        st2.apply_bonds(bonds, us)
    assert fidelity(to_oracle(st2), ref) >= 1 - len(compiled) * FTOL[prec]


def test_routed_32x32_depth8_chi128_sampled(ptebd):
    # The 2D configuration: 32x32 lattice (1024 qubits) on the path, depth 8
    # (4 A/B layers + 2 compiled C/D pairs of 3*31 + 2 layers), chi_max = 128,
    # mixed precision; the last gate layer is checked on 16 sampled bonds
    # against the oracle's single-bond update of the same inputs.
    from paper_2312_02667_gb300 import circuits2d
    lx = ly = 32
    chi = 128
    compiled = circuits2d.compile_layers(lx, ly, circuits2d.physical_layers(4, lx, ly, 8))
    assert len(compiled) == 4 + 2 * 95
    st = ptebd.State(lx * ly, chi, "mixed")
    last_gate = max(i for i, (b, u) in enumerate(compiled) if not np.allclose(u[0], circuits2d.SWAP))
    for bonds, us in compiled[:last_gate]:
        st.apply_bonds(bonds, us)
    bonds, us = compiled[last_gate]
    rng = np.random.default_rng(1)
    pick = sorted(rng.choice(len(bonds), min(16, len(bonds)), replace=False))
    n = lx * ly
    before = {}
    for j in pick:
        b = bonds[j]
        before[j] = (st.lam(b - 1) if b > 0 else np.ones(1), st.site(b), st.lam(b), st.site(b + 1),
                     st.lam(b + 1) if b + 1 < n - 1 else np.ones(1))
    st.apply_bonds(bonds, us)
    eps_g, _, _ = st.bond_stats()
    for j in pick:
        b = bonds[j]
        ll, gb, lb, gb1, lr = before[j]
        mini = mini_vidal(ll, gb, lb, gb1, lr)
        r = oracle.update_bond(mini, 1, us[j], chi, thr("mixed"))
        compare_spectra(st.lam(b), mini.lambdas[1], TOL["mixed"], thr("mixed"), chi)
        assert abs(eps_g[b] - r.eps) <= 1e-5 * max(r.eps, 1e-3)


# ----------------------------------------------- end of Algorithm 1 --------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sampling_matches_oracle(ptebd, prec):
    # same state, same uniforms: the GPU sampler and the oracle's take the same
    # decisions (both in FP64 from the same tensors)
    n, chi = 14, 16
    st = ptebd.State(n, chi, prec)
    for parity, bonds, gates in inputs.brickwork_circuit(10, n, 8):
        st.apply_layer(gates, parity)
    mps = to_oracle(st)
    u = np.random.default_rng(3).random((300, n))
    bits_g = st.sample(u)
    bits_o = oracle.sample(mps, u)
    assert np.array_equal(bits_g, bits_o)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_canonicalize_after_truncating_layers(ptebd, prec):
    n, chi = 12, 8
    st = ptebd.State(n, chi, prec)
    for parity, bonds, gates in inputs.brickwork_circuit(12, n, 10):
        st.apply_layer(gates, parity)
    before = to_oracle(st)
    c0 = oracle.distance_to_canonical(oracle.scale_to_unit_norm(before))
    st.canonicalize()
    after = to_oracle(st)
    assert fidelity(before, after) >= 1 - FTOL[prec]
    c1 = oracle.distance_to_canonical(oracle.scale_to_unit_norm(after))
    floor = 4 * chi * 8 * np.sqrt(2 * chi) * 2.0 ** -24 if prec == "mixed" else 1e-10
    assert c0 > 1e-3 and c1 < floor, (c0, c1)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_chunk_streams_bit_identical(ptebd, prec):
    # A layer split into bond chunks on concurrent streams (the default for
    # large N) against the same layers on one stream: every bond runs the same
    # kernels on the same data, so the states are bit-identical.
    n, chi = 256, 24
    conc = ptebd.State(n, chi, prec, g=1)
    one = ptebd.State(n, chi, prec, g=1)
    one.set_chunk_streams(1)
    for parity, bonds, gates in inputs.brickwork_circuit(41, n, 8):
        conc.apply_layer(gates, parity)
        one.apply_layer(gates, parity)
    for s in range(n):
        assert np.array_equal(conc.site(s), one.site(s)), s
    for b in range(n - 1):
        assert np.array_equal(conc.lam(b), one.lam(b)), b
    ea, la = conc.trunc_error()
    eb, lb = one.trunc_error()
    assert abs(ea - eb) <= 1e-12 * max(abs(eb), 1e-300) and abs(la - lb) <= 1e-12 * max(abs(lb), 1e-300)


def test_chunk_streams_sparse_bonds_and_odd_counts(ptebd):
    # explicit ascending bond lists (routed 2D layers) and 3 or 5 chunks
    from paper_2312_02667_gb300 import circuits2d
    lx = ly = 12
    compiled = circuits2d.compile_layers(lx, ly, circuits2d.physical_layers(9, lx, ly, 8))[:40]
    for k in (3, 5):
        a = ptebd.State(lx * ly, 16, "mixed", g=1)
        b = ptebd.State(lx * ly, 16, "mixed", g=1)
        a.set_chunk_streams(k)
        b.set_chunk_streams(1)
        for bonds, us in compiled:
            a.apply_bonds(bonds, us)
            b.apply_bonds(bonds, us)
        for s in range(lx * ly):
            assert np.array_equal(a.site(s), b.site(s)), (k, s)


def test_bounded_wait_runs_out_reports_timeout_and_recovers(ptebd):
    # Failure detection without a GPU fault: one hand-off wait per CTA waits for
    # a round count nothing writes, under a short limit; the CTAs abort cleanly,
    # the next synchronising call reports PTEBD_ERR_TIMEOUT, and after a reset
    # the same state runs a circuit bit-identically to a fresh one.
    import time
    n, chi = 32, 32
    circ = inputs.brickwork_circuit(61, n, 8)
    st = ptebd.State(n, chi, "mixed")
    for parity, bonds, gates in circ[:6]:
        st.apply_layer(gates, parity)
    st.sync()
    ptebd.ptebd_test_wait_timeout(st.handle, 1)
    t0 = time.time()
    st.apply_layer(circ[6][2], circ[6][0])
    with pytest.raises(ptebd.PtebdError) as err:
        st.sync()
    assert err.value.code == -9  # PTEBD_ERR_TIMEOUT
    assert time.time() - t0 < 60
    ptebd.ptebd_test_wait_timeout(st.handle, 0)
    st.sync()  # the error word was cleared when it was reported
    st.reset()
    fresh = ptebd.State(n, chi, "mixed")
    for parity, bonds, gates in circ:
        st.apply_layer(gates, parity)
        fresh.apply_layer(gates, parity)
    for s in range(n):
        assert np.array_equal(st.site(s), fresh.site(s)), s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ptsu_with_dependent_columns_of_x(ptebd, prec):
    # X = Lambda Gamma_b Lambda of the tSU on bond b with two proportional
    # columns: the Gram-Schmidt basis drops one of them; theta = X Y, and so its
    # singular values (the new Lambda_b), must come out as the oracle's SVD of
    # theta gives them.
    n, chi = 10, 8
    mps = oracle.canonicalize(inputs.random_mps_tensors(17, n, chi))
    b = 4
    g = mps.gammas[b].copy()                      # (2, chi_{b-1}, chi_b)
    lam_b = mps.lambdas[b]
    g[:, :, 1] = g[:, :, 0] * (lam_b[0] / lam_b[1]) * 0.5  # column 1 of X = column 0 / 2
    mps.gammas[b] = g
    st = ptebd.State(n, chi, prec, cutoff=1e-14)
    load_into(st, mps)
    ref = mps.copy()
    st.regauge(1)
    oracle.ptsu_step(ref, chi, thr(prec, 1e-14))
    got = to_oracle(st)
    for bb in range(n - 1):
        compare_spectra(got.lambdas[bb], ref.lambdas[bb], TOL[prec], thr(prec, 1e-14), chi)
    assert fidelity(got, mps) >= 1 - FTOL[prec]
