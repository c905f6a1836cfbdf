"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms,
an exact statevector simulation (a different algorithm), the theorems of
Sec. III, or a planted mistake that a pin must catch.
"""
import numpy as np
import pytest

import oracle
from oracle import statevector as sv
from paper_2312_02667_gb300 import inputs

H = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.diag([1.0, -1.0]).astype(complex)
CNOT_LR = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)  # control = left site
CNOT_RL = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]], dtype=complex)  # control = right site


def run_circuit(n, depth, chi_max, seed=0, cutoff=1e-12, g=0):
    mps = oracle.product_state(n)
    psi = sv.zero_state(n)
    for layer in inputs.brickwork_circuit(seed, n, depth):
        parity, bonds, gates = layer
        oracle.apply_layer(mps, gates, parity, chi_max, cutoff, g)
        for b, u in zip(bonds, gates):
            psi = sv.apply_two_qubit(psi, n, int(b), u)
    return mps, psi


# ---------------------------------------------------------------- inputs ---

def test_haar_gates_unitary_and_uniform():
    rng = np.random.default_rng(5)
    us = np.stack([inputs.haar_u4(rng) for _ in range(4000)])
    err = np.abs(np.einsum("nji,njk->nik", us.conj(), us) - np.eye(4)).max()
    assert err < 1e-14
    # Haar measure: E|U_ij|^2 = 1/4 and E|U_ij|^4 = 1/10 for U(4)
    m2 = (np.abs(us) ** 2).mean()
    m4 = (np.abs(us) ** 4).mean()
    assert abs(m2 - 0.25) < 1e-12  # exact: rows are unit vectors
    assert abs(m4 - 0.1) < 0.004


# ---------------------------------------------------------- closed forms ---

def test_bell_pair_schmidt_values():
    mps = oracle.product_state(2)
    u = CNOT_LR @ np.kron(H, I2)
    res = oracle.apply_layer(mps, [u], 0, chi_max=4, cutoff=1e-12)
    np.testing.assert_allclose(mps.lambdas[0], [2 ** -0.5, 2 ** -0.5], atol=1e-15)
    psi = sv.from_vidal(mps)
    np.testing.assert_allclose(psi, [2 ** -0.5, 0, 0, 2 ** -0.5], atol=1e-15)
    assert res.eps_total == 0.0 and res.bonds[0].nu == 1.0


def test_cnot_orientation_and_gate_layout():
    # |10>: CNOT with control on the left site flips the right one -> |11>;
    # with control on the right site nothing happens.
    for gate, expect in ((CNOT_LR, 3), (CNOT_RL, 2)):
        mps = oracle.product_state(2)
        oracle.apply_bonds(mps, [0], [np.kron(X, I2)], 4, 1e-12)
        oracle.apply_bonds(mps, [0], [gate], 4, 1e-12)
        psi = sv.from_vidal(mps)
        assert abs(abs(psi[expect]) - 1.0) < 1e-14


def test_ghz_chain_closed_form():
    n = 7
    mps = oracle.product_state(n)
    oracle.apply_bonds(mps, [0], [CNOT_LR @ np.kron(H, I2)], 8, 1e-12)
    for b in range(1, n - 1):
        oracle.apply_bonds(mps, [b], [CNOT_LR], 8, 1e-12)
    for b in range(n - 1):
        np.testing.assert_allclose(mps.lambdas[b], [2 ** -0.5] * 2, atol=1e-14)
    for j in range(n):
        assert abs(oracle.expect_one_site(mps, j, Z)) < 1e-14
        assert abs(oracle.expect_one_site(mps, j, X)) < 1e-14
    for j in range(n - 1):
        assert abs(oracle.expect_two_site(mps, j, np.kron(Z, Z)) - 1.0) < 1e-14
    assert abs(oracle.norm(mps) - 1.0) < 1e-14


def test_product_gate_keeps_bond_dimension_one():
    rng = np.random.default_rng(3)
    a = inputs.haar_u4(rng)[:2, :2]
    a, _ = np.linalg.qr(a)
    b, _ = np.linalg.qr(rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)))
    mps = oracle.product_state(4)
    oracle.apply_layer(mps, [np.kron(a, b), np.kron(b, a)], 0, 8, 1e-12)
    assert all(mps.chi(x) == 1 for x in range(3))


def test_single_bond_truncation_closed_form():
    # cos(t)|00> + sin(t)|11>, truncated to chi = 1: eps = sin^2 t, nu = 1/cos t,
    # F_2 = cos^2 t and the stabilised norm n* = n nu = 1 exactly.
    t = 0.3
    ry = np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]], dtype=complex)
    u = CNOT_LR @ np.kron(ry, I2)
    mps = oracle.product_state(2)
    res = oracle.apply_bonds(mps, [0], [u], chi_max=1, cutoff=1e-12)
    r = res.bonds[0]
    assert r.k == 1
    assert abs(r.eps - np.sin(t) ** 2) < 1e-15
    assert abs(r.nu - 1 / np.cos(t)) < 1e-14
    assert abs(oracle.norm(mps) - 1.0) < 1e-14
    psi = sv.from_vidal(mps)
    exact = np.array([np.cos(t), 0, 0, np.sin(t)], dtype=complex)
    assert abs(sv.fidelity(psi, exact) - np.cos(t) ** 2) < 1e-14


# ----------------------------------------------- exact parallel TEBD (no trunc)

@pytest.mark.parametrize("n,depth", [(8, 8), (11, 9)])
def test_untruncated_layers_match_statevector(n, depth):
    mps = oracle.product_state(n)
    psi = sv.zero_state(n)
    for parity, bonds, gates in inputs.brickwork_circuit(11, n, depth):
        res = oracle.apply_layer(mps, gates, parity, chi_max=64, cutoff=1e-12)
        for b, u in zip(bonds, gates):
            psi = sv.apply_two_qubit(psi, n, int(b), u)
        assert sv.fidelity(sv.from_vidal(mps), psi) > 1 - 1e-12
        assert res.eps_total < 1e-24
        # Lambda_b are the Schmidt values of the state at cut b (Sec. II B)
        for b in range(n - 1):
            ref = sv.schmidt_values(psi, n, b)
            ref = ref[ref > 1e-12 * ref[0]]
            lam = mps.lambdas[b]
            assert len(lam) == len(ref)
            assert np.abs(lam - ref).max() < 1e-12 * ref[0]
            assert abs(np.sum(lam ** 2) - 1.0) < 1e-12
        # parallel TEBD without truncation keeps the canonical form (Sec. II C)
        assert oracle.distance_to_canonical(mps) < 1e-12


def test_measurements_match_statevector():
    n = 9
    mps, psi = run_circuit(n, 6, 64, seed=2)
    op = inputs.random_one_site_op(4)
    for j in (0, 4, n - 1):
        full = np.kron(np.kron(np.eye(2 ** j), op), np.eye(2 ** (n - j - 1)))
        ref = np.vdot(psi, full @ psi) / np.vdot(psi, psi)
        assert abs(oracle.expect_one_site(mps, j, op) - ref) < 1e-13
    op2 = inputs.haar_u4(np.random.default_rng(8))
    for j in (0, 3, n - 2):
        full = np.kron(np.kron(np.eye(2 ** j), op2), np.eye(2 ** (n - j - 2)))
        ref = np.vdot(psi, full @ psi) / np.vdot(psi, psi)
        assert abs(oracle.expect_two_site(mps, j, op2) - ref) < 1e-13
    other, psi2 = run_circuit(n, 5, 64, seed=3)
    assert abs(oracle.overlap(mps, other) - np.vdot(psi, psi2)) < 1e-13


def test_canonicalize_gives_schmidt_values():
    n = 9
    tens = inputs.random_mps_tensors(1, n, 8)
    mps = oracle.canonicalize(tens)
    psi = sv.from_vidal(mps)
    assert abs(np.vdot(psi, psi).real - 1) < 1e-13
    acc = np.ones((1, 1), dtype=complex)
    for t in tens:
        acc = np.einsum("pa,sab->psb", acc, t).reshape(-1, t.shape[2])
    raw = acc.reshape(-1)
    assert sv.fidelity(raw, psi) > 1 - 1e-13
    for b in range(n - 1):
        ref = sv.schmidt_values(psi, n, b)[: mps.chi(b)]
        assert np.abs(mps.lambdas[b] - ref).max() < 1e-13
    assert oracle.distance_to_canonical(mps) < 1e-12


# -------------------------------------------------- truncation theorems ----

def canonical_random(n, chi, seed):
    return oracle.canonicalize(inputs.random_mps_tensors(seed, n, chi))


@pytest.mark.parametrize("seed,mode", [(0, "schmidt"), (1, "relative"), (2, "absolute"), (3, "schmidt")])
def test_gate_layer_truncation_against_exact_state(seed, mode):
    # Canonical input, one gate layer, truncated on the gated bonds: Theorem 1
    # (F_2 >= 1 - 2 eps, || Psi - Psi~_T ||^2 <= 2 eps), Lemma 2 (1 - sqrt(2 eps) <= n <= 1)
    # and Theorem 3 (n*_lower <= n* <= n*_upper, n*_lower <= 1 <= n*_upper).
    n = 10
    mps = canonical_random(n, 16, seed)
    psi0 = sv.from_vidal(mps)
    parity, bonds, gates = inputs.brickwork_layer(seed, n, 1)
    exact = psi0.copy()
    for b, u in zip(bonds, gates):
        exact = sv.apply_two_qubit(exact, n, int(b), u)
    res = oracle.apply_layer(mps, gates, parity, chi_max=6, cutoff=1e-12, eps_mode=mode)
    eps = res.eps_total
    prod_nu = np.exp(res.log_nu_total)
    assert eps > 1e-3  # the case truncates for real
    psi_star = sv.from_vidal(mps)            # stabilised state
    psi_t = psi_star / prod_nu               # the projected state Psi~_T
    n_plain = np.linalg.norm(psi_t)
    n_star = np.linalg.norm(psi_star)
    assert np.linalg.norm(exact - psi_t) ** 2 <= 2 * eps + 1e-13
    assert sv.fidelity(exact, psi_t) >= 1 - 2 * eps - 1e-13
    assert 1 - np.sqrt(2 * eps) - 1e-13 <= n_plain <= 1 + 1e-13
    lo, hi = (1 - np.sqrt(2 * eps)) * prod_nu, prod_nu
    assert lo - 1e-13 <= n_star <= hi + 1e-13
    assert lo <= 1 + 1e-13 and hi >= 1 - 1e-13
    assert abs(oracle.norm(mps) - n_star) < 1e-12


def test_truncating_every_bond_obeys_theorem_1():
    n = 10
    mps = canonical_random(n, 16, 7)
    psi = sv.from_vidal(mps)
    eps = sum(float(np.sum(mps.lambdas[b][8:] ** 2)) for b in range(n - 1))
    cut = oracle.truncate_all_bonds(mps, 8)
    psi_t = sv.from_vidal(cut)
    assert eps > 1e-3
    assert np.linalg.norm(psi - psi_t) ** 2 <= 2 * eps + 1e-13
    assert sv.fidelity(psi, psi_t) >= 1 - 2 * eps
    # the looser bound of Sec. III B
    eps_i = [float(np.sum(mps.lambdas[b][8:] ** 2)) for b in range(n - 1)]
    assert sv.fidelity(psi, psi_t) >= 1 - 2 * sum(np.sqrt(eps_i))


def test_single_truncated_bond_is_schmidt_truncation():
    # A canonical state and one truncated bond: the layer equals the dense
    # Schmidt truncation of U|Psi> at that cut, and n* = 1 exactly.
    n = 8
    mps, psi = run_circuit(n, 6, 64, seed=4)
    b = 3
    u = inputs.haar_u4(np.random.default_rng(77))
    res = oracle.apply_bonds(mps, [b], [u], chi_max=5, cutoff=1e-12)
    psi = sv.apply_two_qubit(psi, n, b, u)
    m = psi.reshape(2 ** (b + 1), -1)
    uu, s, vh = np.linalg.svd(m, full_matrices=False)
    ref = (uu[:, :5] * s[:5]) @ vh[:5]
    ref = ref.reshape(-1) / np.linalg.norm(s[:5])
    got = sv.from_vidal(mps)
    assert abs(res.bonds[0].eps - np.sum(s[5:] ** 2)) < 1e-13
    assert sv.fidelity(got, ref) > 1 - 1e-12
    assert abs(np.linalg.norm(got) - 1.0) < 1e-12


# ------------------------------------------------------------------ PtSU ---

@pytest.mark.parametrize("n", [10, 11])
def test_ptsu_restores_canonical_form_within_theorem_4(n):
    # Random-MPS recipe of Sec. III D: canonicalised random MPS, every bond
    # truncated to chi/2, norm set back to 1, then PtSU steps.
    mps = canonical_random(n, 16, 3)
    cut = oracle.scale_to_unit_norm(oracle.truncate_all_bonds(mps, 8))
    psi_before = sv.from_vidal(cut)
    c0 = oracle.distance_to_canonical(cut)
    assert c0 > 1e-3
    steps = n // 2 if n % 2 == 0 else (n - 1) // 2
    cs = [c0]
    for _ in range(steps):
        oracle.ptsu_step(cut, chi_max=64, cutoff=1e-14)
        cs.append(oracle.distance_to_canonical(cut))
    assert cs[-1] < 1e-10
    assert cs[1] < c0  # the first step already moves towards the canonical form
    # tSU never changes the state (identity gate)
    assert sv.fidelity(sv.from_vidal(cut), psi_before) > 1 - 1e-12
    assert abs(np.linalg.norm(sv.from_vidal(cut)) - 1.0) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 7])
def test_scale_to_unit_norm_keeps_canonical_form(n):
    # A canonical MPS multiplied by c with the factor spread as PtSU leaves it
    # (every Lambda times c, every interior Gamma divided by c) is not
    # canonical at the end sites; scaling to unit norm restores the canonical
    # conditions everywhere and gives back the same normalised vector.
    mps = canonical_random(n, 8, 11)
    c = 3.0 ** (1.0 / max(1, n - 1)) if n > 1 else 3.0
    big = mps.copy()
    if n == 1:
        big.gammas[0] = big.gammas[0] * c
    else:
        big.lambdas = [l * c for l in big.lambdas]
        for s in range(1, n - 1):
            big.gammas[s] = big.gammas[s] / c
    psi = sv.from_vidal(mps)
    assert abs(np.linalg.norm(sv.from_vidal(big)) - c) < 1e-12 * c
    if n > 1:
        assert oracle.distance_to_canonical(big) > 0.01
    out = oracle.scale_to_unit_norm(big)
    assert oracle.distance_to_canonical(out) < 1e-12
    assert np.abs(sv.from_vidal(out) - psi).max() < 1e-12


def test_tsu_on_canonical_state_is_identity_on_lambda():
    mps, _ = run_circuit(9, 7, 64, seed=9)
    before = [l.copy() for l in mps.lambdas]
    oracle.ptsu_step(mps, 64, 1e-12)
    for a, b in zip(before, mps.lambdas):
        assert len(a) == len(b) and np.abs(a - b).max() < 1e-12


# ------------------------------------------------------ norm stabilisation ---

def test_norm_decays_without_nu_and_stays_near_one_with_nu():
    # Sec. IV B 2: without the local factors nu the norm decays with depth;
    # with them the stabilised norm stays close to 1.
    n, depth = 14, 40
    mps = oracle.product_state(n)
    log_prod_nu = 0.0
    for parity, bonds, gates in inputs.brickwork_circuit(21, n, depth):
        res = oracle.apply_layer(mps, gates, parity, chi_max=16, cutoff=1e-12)
        log_prod_nu += res.log_nu_total
    n_star = oracle.norm(mps)
    n_plain = n_star * np.exp(-log_prod_nu)
    assert n_plain < 0.2
    assert 0.7 < n_star < 1.5


def test_eps_readings_agree_on_canonical_input():
    # On a normalised canonical state |S| = 1 on every bond, so the three
    # readings of eps_b and of the stabilised Lambda_b coincide (Sec. III C).
    n = 10
    base = canonical_random(n, 16, 5)
    parity, bonds, gates = inputs.brickwork_layer(5, n, 0)
    runs = {}
    for mode in ("schmidt", "relative", "absolute"):
        m = base.copy()
        runs[mode] = (oracle.apply_layer(m, gates, parity, 6, 1e-12, eps_mode=mode), m)
    ra, a = runs["schmidt"]
    for mode in ("relative", "absolute"):
        rb, b = runs[mode]
        assert abs(ra.eps_total - rb.eps_total) < 1e-13
        for x, y in zip(a.lambdas, b.lambdas):
            assert np.abs(x - y).max() < 1e-13


def test_schmidt_reading_gives_unit_bond_weight_off_canonical_form():
    # Closed form of the stabilised update: Lambda_b = nu_b S_kept / |S| with
    # nu_b^2 = 1 / (1 - eps_b) and eps_b = |S_dropped|^2 / |S|^2, so
    # sum Lambda_b^2 = 1 on every gated bond whatever the gauge; the relative
    # reading keeps sum Lambda_b^2 = |S|^2 instead.
    n = 10
    ts = [np.asarray(t) for t in inputs.random_mps_tensors(8, n, 8)]
    raw = oracle.Vidal(ts, [np.linspace(1.5, 0.2, ts[b].shape[2]) for b in range(n - 1)])
    parity, bonds, gates = inputs.brickwork_layer(8, n, 0)
    a, b = raw.copy(), raw.copy()
    ra = oracle.apply_layer(a, gates, parity, 4, 1e-12, eps_mode="schmidt")
    rb = oracle.apply_layer(b, gates, parity, 4, 1e-12, eps_mode="relative")
    assert sum(r.eps > 1e-3 for r in ra.bonds) >= 2
    for r, q in zip(ra.bonds, rb.bonds):
        total = float(np.sum(r.s_full ** 2))
        assert abs(total - 1.0) > 1e-2  # off the canonical form
        assert abs(np.sum(a.lambdas[r.bond] ** 2) - 1.0) < 1e-12
        assert abs(np.sum(b.lambdas[q.bond] ** 2) - total) < 1e-12 * total
        assert abs(r.nu ** 2 * (1 - r.eps) - 1.0) < 1e-12


def test_stabilised_norm_stays_near_one_over_many_truncating_layers():
    # Sec. IV C: with the stabilisation the wavefunction norm stays close to 1
    # with depth (1D and 2D circuits, g = 0).  A 1D brickwork that truncates
    # on every layer (N = 40, chi = 8, 60 layers): the Schmidt reading stays
    # near 1; the relative reading, which leaves |S| in Lambda, grows
    # exponentially and so cannot be the paper's update.
    n, chi, depth = 40, 8, 60
    norms = {}
    for mode in ("schmidt", "relative"):
        mps = oracle.product_state(n)
        for parity, bonds, gates in inputs.brickwork_circuit(3, n, depth):
            oracle.apply_layer(mps, gates, parity, chi, 1e-12, eps_mode=mode)
        norms[mode] = oracle.norm(mps)
    assert 0.5 < norms["schmidt"] < 2.0
    assert norms["relative"] > 100.0


# ------------------------------------------------------- planted mistakes ---

def test_planted_transposed_gate_is_caught(monkeypatch):
    real = oracle.mps.apply_two_site_gate
    monkeypatch.setattr(oracle.mps, "apply_two_site_gate", lambda th, u: real(th, np.asarray(u).T))
    mps, psi = run_circuit(6, 4, 64, seed=1)
    assert sv.fidelity(sv.from_vidal(mps), psi) < 1 - 1e-6


def test_planted_missing_lambda_division_is_caught(monkeypatch):
    real_svd = np.linalg.svd

    def tsu_free_update(mps, b, gate, chi_max, cutoff, stabilise=True, eps_mode="schmidt"):
        # same as the oracle but forgets Lambda_{b+1}^{-1} on the right tensor
        theta = oracle.two_site_tensor(mps, b)
        if gate is not None:
            theta = oracle.apply_two_site_gate(theta, gate)
        ns, chil, nt, chir = theta.shape
        u, s, vh = real_svd(theta.reshape(ns * chil, nt * chir), full_matrices=False)
        k = oracle.truncation_rank(s, chi_max, cutoff)
        mps.gammas[b] = u[:, :k].reshape(ns, chil, k) / mps.lam(b - 1)[None, :, None]
        mps.gammas[b + 1] = vh[:k].reshape(k, nt, chir).transpose(1, 0, 2)
        mps.lambdas[b] = s[:k]
        return oracle.BondResult(b, k, len(s), 0.0, 1.0, s)

    monkeypatch.setattr(oracle.mps, "update_bond", tsu_free_update)
    mps, psi = run_circuit(6, 4, 64, seed=1)
    assert sv.fidelity(sv.from_vidal(mps), psi) < 1 - 1e-6


def test_planted_missing_nu_breaks_theorem_3(monkeypatch):
    real = oracle.mps.update_bond

    def no_nu(mps, b, gate, chi_max, cutoff, stabilise=True, eps_mode="schmidt"):
        return real(mps, b, gate, chi_max, cutoff, False, eps_mode)

    monkeypatch.setattr(oracle.mps, "update_bond", no_nu)
    mps = oracle.product_state(2)
    t = 0.3
    ry = np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]], dtype=complex)
    oracle.apply_bonds(mps, [0], [CNOT_LR @ np.kron(ry, I2)], 1, 1e-12)
    assert abs(oracle.norm(mps) - 1.0) > 1e-3


# ------------------------------------------------------------------ sampling

def test_sampling_follows_statevector_marginals():
    # the sampler's decisions against conditional probabilities computed
    # directly from the 2^N amplitudes (a different computation)
    n = 8
    mps, psi = run_circuit(n, 6, 64, seed=6)
    rng = np.random.default_rng(0)
    u = rng.random((200, n))
    bits = oracle.sample(mps, u)
    prob = (np.abs(psi) ** 2).reshape([2] * n)
    prob = prob / prob.sum()
    for k in range(u.shape[0]):
        marg = prob  # sites drawn from the right end
        for s in range(n - 1, -1, -1):
            m = marg.reshape(-1, 2).sum(axis=0)
            p0 = m[0] / m.sum()
            if abs(u[k, s] - p0) < 1e-9:
                break  # a tie: both choices are valid
            x = 0 if u[k, s] < p0 else 1
            assert bits[k, s] == x
            marg = marg[..., x]


def test_sampling_frequencies_on_a_truncated_state():
    # a non-canonical (truncated) state: empirical frequencies of the sampler
    # against |Psi|^2 / <Psi|Psi> (total variation distance)
    n = 6
    mps, _ = run_circuit(n, 8, 2, seed=7)
    psi = sv.from_vidal(mps)
    p = np.abs(psi) ** 2
    p /= p.sum()
    u = np.random.default_rng(1).random((20000, n))
    bits = oracle.sample(mps, u)
    idx = bits @ (2 ** np.arange(n - 1, -1, -1))
    freq = np.bincount(idx, minlength=2 ** n) / len(idx)
    assert 0.5 * np.abs(freq - p).sum() < 0.03
