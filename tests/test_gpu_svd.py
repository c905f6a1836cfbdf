"""The batched SVD entry point (the layer's Jacobi kernel on caller matrices)
against closed forms and the oracle's SVD primitive."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02667_gb300 import ptebd
    return torch, ptebd


def haar(n, rng):
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_ginibre_512(env, prec, tol):
    torch, ptebd = env
    rng = np.random.default_rng(0)
    a = (rng.standard_normal((3, 512, 512)) + 1j * rng.standard_normal((3, 512, 512))) / np.sqrt(2 * 512)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    at = torch.from_numpy(a).to(dt).cuda()
    sig, u = ptebd.svd_batched(at, want_u=True)
    sig = sig.cpu().numpy()
    u = u.cpu().numpy().astype(np.complex128)
    a_in = at.cpu().numpy().astype(np.complex128)  # the rounded input the kernel saw
    for i in range(3):
        ref = np.linalg.svd(a_in[i], compute_uv=False)
        assert np.abs(sig[i] - ref).max() <= tol * ref[0]
        assert np.abs(u[i].conj().T @ u[i] - np.eye(512)).max() <= (1e-12 if prec == "fp64" else 2e-5)
        # U^H A has orthogonal rows of length sigma: A = U S V^H
        rows = u[i].conj().T @ a_in[i]
        assert np.abs(np.linalg.norm(rows, axis=1) - sig[i]).max() <= tol * 10 * ref[0]


def test_mixed_columns_orthogonal_to_the_threshold(env):
    # The complex64 sweeps stop after a sweep without rotations or after one whose
    # rotations all had cos^2 < 256 tol^2 (tol = 8 sqrt(m) u, the rotation
    # threshold).  Either way every pair of output columns must be orthogonal to
    # about tol: the largest |u_i^H u_j| (unit columns, formed in complex128 from
    # the stored complex64 U) stays below 1.5 tol.  A stopping rule that quit in
    # the quadratic phase (cos ~ 1e-3) would leave pairs far above it.
    torch, ptebd = env
    rng = np.random.default_rng(11)
    m = 512
    tol = 8.0 * np.sqrt(m) * 2.0 ** -24
    gin = (rng.standard_normal((2, m, m)) + 1j * rng.standard_normal((2, m, m))) / np.sqrt(2 * m)
    lam = 10.0 ** (-6.0 * np.arange(m) / m)
    graded = np.stack([haar(m, rng) @ np.diag(lam) @ haar(m, rng).conj().T for _ in range(2)])
    a = np.concatenate([gin, graded])
    _, u = ptebd.svd_batched(torch.from_numpy(a).to(torch.complex64).cuda(), want_u=True)
    u = u.cpu().numpy().astype(np.complex128)
    for i in range(a.shape[0]):
        ui = u[i] / np.linalg.norm(u[i], axis=0)[None, :]
        g = np.abs(ui.conj().T @ ui)
        np.fill_diagonal(g, 0.0)
        assert g.max() <= 1.5 * tol, (i, g.max() / tol)


@pytest.mark.parametrize("prec,shifts", [("mixed", [-100, -40, 40, 100]), ("fp64", [-700, 600])])
def test_range_guard_scale_invariance(env, prec, shifts):
    # sigma(2^k A) = 2^k sigma(A): the kernel forms squared norms and |a^H b|^2 in
    # its own precision, so without its range guard 2^40 A (complex64) overflows and
    # rotations turn into plain scalings.  Power-of-two scalings are exact, so the
    # scaled runs reproduce the unscaled singular values to rounding.
    torch, ptebd = env
    rng = np.random.default_rng(7)
    n = 256
    a = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2 * n)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    base = torch.from_numpy(a[None]).to(dt).cuda()
    s0, _ = ptebd.svd_batched(base)
    s0 = s0.cpu().numpy()[0]
    tol = 1e-12 if prec == "fp64" else 1e-6
    for k in shifts:
        sk, _ = ptebd.svd_batched(base * (2.0 ** k))
        sk = sk.cpu().numpy()[0] * 2.0 ** -k
        assert np.all(np.isfinite(sk))
        assert np.abs(sk - s0).max() <= tol * s0[0], (k, np.abs(sk - s0).max() / s0[0])


def test_graded_spectrum_closed_form(env):
    # lambda_a = 10^(-12 a / n): singular values known exactly
    torch, ptebd = env
    rng = np.random.default_rng(1)
    n = 128
    lam = 10.0 ** (-12.0 * np.arange(n) / n)
    a = haar(n, rng) @ np.diag(lam) @ haar(n, rng).conj().T
    sig, _ = ptebd.svd_batched(torch.from_numpy(a[None]).cuda())
    sig = sig.cpu().numpy()[0]
    assert np.abs(sig - lam).max() <= 1e-13
    # the large ones to high relative accuracy
    assert np.abs(sig[:32] / lam[:32] - 1).max() <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rank_deficient_and_small_shapes(env, prec):
    torch, ptebd = env
    rng = np.random.default_rng(2)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    x = rng.standard_normal((256, 64)) + 1j * rng.standard_normal((256, 64))
    y = rng.standard_normal((64, 200)) + 1j * rng.standard_normal((64, 200))
    a = (x @ y) / 100
    sig, _ = ptebd.svd_batched(torch.from_numpy(a[None]).to(dt).cuda())
    sig = sig.cpu().numpy()[0]
    ref = np.linalg.svd(a, compute_uv=False)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.abs(sig - ref).max() <= tol * ref[0]
    assert sig[64:].max() <= (1e-13 if prec == "fp64" else 1e-5) * ref[0]
    for rows, cols in ((2, 1), (2, 2), (4, 3), (34, 34)):
        b = rng.standard_normal((5, rows, cols)) + 1j * rng.standard_normal((5, rows, cols))
        s2, u2 = ptebd.svd_batched(torch.from_numpy(b).to(dt).cuda(), want_u=True)
        for i in range(5):
            ref = np.linalg.svd(b[i].astype(np.complex64 if prec == "mixed" else np.complex128).astype(complex),
                                compute_uv=False)
            assert np.abs(s2.cpu().numpy()[i] - ref).max() <= tol * ref[0]


def test_bad_arguments(env):
    torch, ptebd = env
    with pytest.raises(ptebd.PtebdError):
        ptebd.ptebd_svd_workspace_bytes(0, 1, 8, 9)  # wide
    with pytest.raises(ptebd.PtebdError):
        ptebd.ptebd_svd_workspace_bytes(0, 1, 1024, 8)  # too tall
    with pytest.raises(ptebd.PtebdError):
        ptebd.ptebd_svd_workspace_bytes(0, 1, 7, 3)  # odd rows
