"""Vidal-form MPS and the pTEBD layer, written from the paper (oracle).

TEST INFRASTRUCTURE ONLY: see the package docstring.

Notation (build convention): sites s = 0..N-1 carry Gamma[s] with shape
(2, chi_{s-1}, chi_s); bond b = 0..N-2 joins sites b, b+1 and carries the real
vector Lambda[b] (descending).  The open boundary vectors Lambda_{-1} and
Lambda_{N-1} are (1) (Sec. II B, Eq. of the canonical decomposition).  The
paper's site i is our site i-1 and its bond i our bond i-1.

Readings of points the paper leaves open (listed with the rest in the design
notes):

* truncation rank k = min(chi_max, #{lambda_a > cutoff * lambda_1}), at least 1;
  everything dropped (by chi_max or by the cutoff) counts in eps_b;
* the bond vector is the Schmidt spectrum of the normalised two-site
  wavefunction, lambda^ = S / |S| (Sec. II B: sum lambda^2 = 1), and the norm
  stabilisation acts on it (Sec. III C): eps_b = sum_dropped lambda^^2,
  nu_b = (1 - eps_b)^(-1/2), Lambda_b <- nu_b lambda^_kept
  (``eps_mode="schmidt"``, the default).  On a normalised canonical state
  |S| = 1 and this is the paper's update word for word.  Off the canonical
  form |S| drifts from 1; this reading keeps the wavefunction norm near 1 over
  many layers in 1D and 2D circuits, which is what the paper reports for its
  stabilised runs (Sec. IV C, figure of the norms versus depth).  Two other
  readings are kept for comparison: ``"relative"`` (eps_b = dropped / all S^2,
  Lambda_b <- nu_b S_kept: the norm then grows exponentially with depth once
  the bonds truncate, e.g. n* ~ 8e3 after 60 layers at N = 40, chi = 8) and
  ``"absolute"`` (eps_b = sum_dropped S^2 taken literally, Lambda_b <- nu_b
  S_kept: eps_b >= 1 within tens of Haar-random layers);
* Gamma rebuilt by literal division by the neighbouring Lambda (Sec. II C);
* nu_b is applied to every gated bond (it is exactly 1 when nothing is
  dropped); tSU steps never apply nu;
* when the layer asks for g > 0, g PtSU steps follow every layer;
* a PtSU step = tSU on bonds b = 0, 2, 4, ... (the paper's odd bonds), then on
  b = 1, 3, 5, ... (Sec. III D).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Vidal",
    "product_state",
    "two_site_tensor",
    "apply_two_site_gate",
    "truncation_rank",
    "BondResult",
    "update_bond",
    "tsu",
    "ptsu_step",
    "apply_layer",
    "apply_bonds",
    "LayerResult",
    "overlap",
    "norm",
    "expect_one_site",
    "expect_two_site",
    "distance_to_canonical",
    "canonicalize",
    "from_mps_tensors",
    "truncate_all_bonds",
    "scale_to_unit_norm",
    "left_environments",
    "sample",
]


class OracleError(RuntimeError):
    pass


@dataclass
class Vidal:
    """{Gamma[s], Lambda[b]} of an open MPS (Sec. II B)."""

    gammas: list
    lambdas: list

    @property
    def n_sites(self) -> int:
        return len(self.gammas)

    def lam(self, b: int) -> np.ndarray:
        """Lambda_b with the open-boundary convention Lambda_{-1} = Lambda_{N-1} = (1)."""
        if b < 0 or b >= self.n_sites - 1:
            return np.ones(1)
        return self.lambdas[b]

    def chi(self, b: int) -> int:
        return len(self.lam(b))

    def copy(self) -> "Vidal":
        return Vidal([g.copy() for g in self.gammas], [l.copy() for l in self.lambdas])


def product_state(n_sites: int) -> Vidal:
    """|0...0> with every bond dimension 1 (Sec. IV A: chi_0 = 1)."""
    g = np.zeros((2, 1, 1), dtype=np.complex128)
    g[0, 0, 0] = 1.0
    return Vidal([g.copy() for _ in range(n_sites)], [np.ones(1) for _ in range(n_sites - 1)])


def two_site_tensor(mps: Vidal, b: int) -> np.ndarray:
    """Psi_{i,i+1} = Lambda^{[i-1]} Gamma^{[i]} Lambda^{[i]} Gamma^{[i+1]} Lambda^{[i+1]}
    (Sec. II C), returned with indices (s, alpha, t, gamma)."""
    ll, lm, lr = mps.lam(b - 1), mps.lam(b), mps.lam(b + 1)
    x = ll[None, :, None] * mps.gammas[b] * lm[None, None, :]
    y = mps.gammas[b + 1] * lr[None, None, :]
    return np.einsum("sab,tbc->satc", x, y)


def apply_two_site_gate(theta: np.ndarray, gate: np.ndarray) -> np.ndarray:
    """Psi' = U Psi on the two physical indices (Sec. II C); the gate is
    U[(2 s' + t'), (2 s + t)] with s the left site."""
    u = np.asarray(gate, dtype=np.complex128).reshape(2, 2, 2, 2)
    return np.einsum("xyst,satc->xayc", u, theta)


def truncation_rank(s: np.ndarray, chi_max: int, cutoff: float) -> int:
    """Number of singular values kept by the projector P_i (Sec. III B):
    the chi' = min(chi_max, #{lambda > cutoff * lambda_1}) largest, at least one."""
    if s.size == 0 or not s[0] > 0.0:
        raise OracleError("two-site tensor is zero: nothing to keep")
    above = int(np.count_nonzero(s > cutoff * s[0]))
    return max(1, min(chi_max, above))


@dataclass
class BondResult:
    bond: int
    k: int              # kept rank chi_b
    rank_in: int        # number of singular values of theta' (its smaller side)
    eps: float          # discarded weight eps_b (Theorem 1 definition)
    nu: float           # nu_b = (1 - eps_b)^(-1/2), 1 for tSU
    s_full: np.ndarray  # all singular values of theta', descending


def update_bond(mps: Vidal, b: int, gate, chi_max: int, cutoff: float,
                stabilise: bool = True, eps_mode: str = "schmidt") -> BondResult:
    """One TEBD procedure on bond b with parallel truncation and norm
    stabilisation, in place.

    1. theta = Lambda_{b-1} Gamma_b Lambda_b Gamma_{b+1} Lambda_{b+1}   (Sec. II C)
    2. theta' = U theta (skipped when ``gate is None``: tSU, Sec. III D)
    3. theta' = U S V^dagger (SVD, descending S)                        (Sec. II C)
    4. keep k values (projector P_b); the Schmidt values of the normalised
       two-site wavefunction are S / |S|, eps_b = sum of the dropped ones
       squared                                                       (Sec. II B, III B, Theorem 1)
    5. Lambda_b <- nu_b S[:k] / |S|, nu_b = (1 - eps_b)^(-1/2)          (Sec. III C, stabilised norm)
       (tSU, no stabilisation: Lambda_b <- S[:k], the state unchanged)
    6. Gamma_b <- Lambda_{b-1}^{-1} U[:, :k],
       Gamma_{b+1} <- V^dagger[:k, :] Lambda_{b+1}^{-1}                (Sec. II C)
    """
    theta = two_site_tensor(mps, b)
    if gate is not None:
        theta = apply_two_site_gate(theta, gate)
    ns, chil, nt, chir = theta.shape
    mat = theta.reshape(ns * chil, nt * chir)
    u, s, vh = np.linalg.svd(mat, full_matrices=False)
    k = truncation_rank(s, chi_max, cutoff)
    dropped, total = float(np.sum(s[k:] ** 2)), float(np.sum(s ** 2))
    if eps_mode in ("schmidt", "relative"):
        eps = dropped / total
    elif eps_mode == "absolute":
        eps = dropped
    else:
        raise ValueError(eps_mode)
    if stabilise:
        if not eps < 1.0:
            raise OracleError(f"bond {b}: discarded weight {eps} >= 1, nu undefined")
        nu = (1.0 - eps) ** -0.5
    else:
        nu = 1.0
    ll, lr = mps.lam(b - 1), mps.lam(b + 1)
    gl = u[:, :k].reshape(ns, chil, k) / ll[None, :, None]
    gr = vh[:k, :].reshape(k, nt, chir).transpose(1, 0, 2) / lr[None, None, :]
    mps.gammas[b] = np.ascontiguousarray(gl)
    mps.gammas[b + 1] = np.ascontiguousarray(gr)
    if stabilise and eps_mode == "schmidt":
        mps.lambdas[b] = nu * (s[:k] / np.sqrt(total))
    else:
        mps.lambdas[b] = nu * s[:k].copy()
    return BondResult(b, k, len(s), eps, nu, s)


def tsu(mps: Vidal, b: int, chi_max: int, cutoff: float) -> BondResult:
    """Trivial simple update: the TEBD procedure with the identity gate skipped
    and no norm stabilisation (Sec. II C end, Sec. III D)."""
    return update_bond(mps, b, None, chi_max, cutoff, stabilise=False)


def ptsu_step(mps: Vidal, chi_max: int, cutoff: float) -> list:
    """One PtSU step: tSU on all of the paper's odd bonds (our b = 0, 2, ...)
    then on all of its even bonds (our b = 1, 3, ...) (Sec. III D)."""
    res = []
    for first in (0, 1):
        for b in range(first, mps.n_sites - 1, 2):
            res.append(tsu(mps, b, chi_max, cutoff))
    return res


@dataclass
class LayerResult:
    bonds: list = field(default_factory=list)   # BondResult per gated bond
    tsu: list = field(default_factory=list)     # BondResult per tSU

    @property
    def eps_total(self) -> float:
        return float(sum(r.eps for r in self.bonds))

    @property
    def log_nu_total(self) -> float:
        return float(sum(np.log(r.nu) for r in self.bonds))


def apply_bonds(mps: Vidal, bonds, gates, chi_max: int, cutoff: float, g: int = 0,
                eps_mode: str = "schmidt") -> LayerResult:
    """One circuit layer on a set of pairwise non-adjacent bonds (Algorithm 1,
    one pass of the loop over m): the TEBD procedure with compression and
    stabilisation on every listed bond, then g PtSU steps.  The bonds of one
    layer never touch, so processing them one after another equals processing
    them at once (Sec. II C: parallel TEBD)."""
    bonds = [int(b) for b in bonds]
    for a, c in zip(sorted(bonds), sorted(bonds)[1:]):
        if c - a < 2:
            raise OracleError(f"bonds {a} and {c} overlap")
    out = LayerResult()
    for b, u in zip(bonds, gates):
        out.bonds.append(update_bond(mps, b, u, chi_max, cutoff, True, eps_mode))
    for _ in range(g):
        out.tsu.extend(ptsu_step(mps, chi_max, cutoff))
    return out


def apply_layer(mps: Vidal, gates, parity: int, chi_max: int, cutoff: float, g: int = 0,
                eps_mode: str = "schmidt") -> LayerResult:
    """A brickwork layer: gates[j] acts on bond b = parity + 2 j."""
    bonds = list(range(parity, mps.n_sites - 1, 2))
    if len(gates) != len(bonds):
        raise OracleError(f"{len(gates)} gates for {len(bonds)} bonds")
    return apply_bonds(mps, bonds, gates, chi_max, cutoff, g, eps_mode)


# --------------------------------------------------------------------------
# Measurements (full contractions; exact for any MPS, canonical or not)
# --------------------------------------------------------------------------

def _site_matrix(mps: Vidal, s: int) -> np.ndarray:
    """Gamma_s Lambda_s with Lambda_{N-1} = (1); Lambda_{-1} = (1) is implicit."""
    return mps.gammas[s] * mps.lam(s)[None, None, :]


def _transfer(e: np.ndarray, ma: np.ndarray, mb: np.ndarray) -> np.ndarray:
    """E' = sum_s M_a[s]^dag E M_b[s]: one step of the left-to-right transfer
    matrices, written as the two matrix products per physical index."""
    out = np.zeros((ma.shape[2], mb.shape[2]), dtype=np.complex128)
    for s in range(ma.shape[0]):
        out += ma[s].conj().T @ (e @ mb[s])
    return out


def overlap(a: Vidal, b: Vidal) -> complex:
    """<a|b> by left-to-right transfer matrices (Eq. of the MPS decomposition,
    Sec. II A)."""
    if a.n_sites != b.n_sites:
        raise OracleError("different lengths")
    e = np.ones((1, 1), dtype=np.complex128)
    for s in range(a.n_sites):
        e = _transfer(e, _site_matrix(a, s), _site_matrix(b, s))
    return complex(e[0, 0])


def norm(mps: Vidal) -> float:
    """n = || |Psi> ||."""
    return float(np.sqrt(max(overlap(mps, mps).real, 0.0)))


def expect_one_site(mps: Vidal, site: int, op: np.ndarray) -> complex:
    """<Psi| O_site |Psi> / <Psi|Psi>, O[sigma', sigma] a 2x2 matrix."""
    op = np.asarray(op, dtype=np.complex128)
    e = np.ones((1, 1), dtype=np.complex128)
    for s in range(mps.n_sites):
        m = _site_matrix(mps, s)
        if s == site:
            # sum_{x,y} O[x,y] M[x]^dag E M[y]
            me = np.einsum("xy,yab->xab", op, m)
            e = _transfer(e, m, me)
        else:
            e = _transfer(e, m, m)
    return complex(e[0, 0]) / overlap(mps, mps)


def expect_two_site(mps: Vidal, site: int, op: np.ndarray) -> complex:
    """<Psi| O_{site,site+1} |Psi> / <Psi|Psi>, O a 4x4 matrix in the gate layout."""
    op = np.asarray(op, dtype=np.complex128).reshape(2, 2, 2, 2)  # [x', y', x, y]
    e = np.ones((1, 1), dtype=np.complex128)
    s = 0
    while s < mps.n_sites:
        if s == site:
            m1, m2 = _site_matrix(mps, s), _site_matrix(mps, s + 1)
            pair = np.einsum("xab,ybc->xyac", m1, m2).reshape(4, m1.shape[1], m2.shape[2])
            opair = np.einsum("ij,jac->iac", op.reshape(4, 4), pair)
            e = _transfer(e, pair, opair)
            s += 2
        else:
            m = _site_matrix(mps, s)
            e = _transfer(e, m, m)
            s += 1
    return complex(e[0, 0]) / overlap(mps, mps)


def distance_to_canonical(mps: Vidal) -> float:
    """C = (1/2N) sum_i ( ||sum_s A^dag A - I|| + ||sum_s B B^dag - I|| ), Frobenius
    norms, A_i = Lambda_{i-1} Gamma_i, B_i = Gamma_i Lambda_i (Sec. III D); the
    paper takes the MPS normalised to 1, and so does this function."""
    n = mps.n_sites
    total = 0.0
    for s in range(n):
        a = mps.lam(s - 1)[None, :, None] * mps.gammas[s]
        bm = mps.gammas[s] * mps.lam(s)[None, None, :]
        left = np.einsum("sai,saj->ij", a.conj(), a)
        right = np.einsum("sai,sbi->ab", bm, bm.conj())
        total += np.linalg.norm(left - np.eye(left.shape[0]))
        total += np.linalg.norm(right - np.eye(right.shape[0]))
    return total / (2 * n)


# --------------------------------------------------------------------------
# Preparation helpers (sequential; used to build test inputs and as the
# final Canonicalize of Algorithm 1)
# --------------------------------------------------------------------------

def canonicalize(tensors) -> Vidal:
    """Vidal canonical form of a general open MPS M[s] (d, chi_l, chi_r),
    normalised to 1: a left-to-right QR sweep makes every site left-orthonormal,
    then a right-to-left SVD sweep exposes the Schmidt values of every cut
    (Sec. II B; the standard construction of Schollwoeck 2011)."""
    m = [np.asarray(t, dtype=np.complex128).copy() for t in tensors]
    n = len(m)
    for s in range(n - 1):
        d, cl, cr = m[s].shape
        q, r = np.linalg.qr(m[s].transpose(1, 0, 2).reshape(cl * d, cr))
        k = q.shape[1]
        m[s] = q.reshape(cl, d, k).transpose(1, 0, 2)
        m[s + 1] = np.einsum("ab,sbc->sac", r, m[s + 1])
    lambdas = [None] * (n - 1)
    bmats = [None] * n
    carry = m[n - 1]
    for s in range(n - 1, 0, -1):
        d, cl, cr = carry.shape
        u, sv, vh = np.linalg.svd(carry.transpose(1, 0, 2).reshape(cl, d * cr), full_matrices=False)
        keep = max(1, int(np.count_nonzero(sv > 1e-14 * sv[0])))
        u, sv, vh = u[:, :keep], sv[:keep], vh[:keep]
        bmats[s] = vh.reshape(keep, d, cr).transpose(1, 0, 2)
        lambdas[s - 1] = sv
        carry = np.einsum("sab,bc->sac", m[s - 1], u * sv[None, :])
    nrm = np.linalg.norm(carry)
    bmats[0] = carry / nrm
    lambdas = [l / nrm for l in lambdas]
    gam = []
    for s in range(n):
        lr = lambdas[s] if s < n - 1 else np.ones(1)
        gam.append(bmats[s] / lr[None, None, :])
    # Gamma_0 was built as B_0 scaled by the norm: B_0 = Gamma_0 Lambda_0 with
    # Lambda_0 the normalised Schmidt values of the first cut.
    return Vidal(gam, lambdas)


def from_mps_tensors(tensors) -> Vidal:
    """Canonical, normalised Vidal form of random tensors (see ``canonicalize``)."""
    return canonicalize(tensors)


def truncate_all_bonds(mps: Vidal, chi_keep: int) -> Vidal:
    """Insert the projector P_b on every bond at once (Sec. III B): keep the
    chi_keep largest Lambda of each bond and the matching Gamma slices."""
    out = mps.copy()
    for b in range(mps.n_sites - 1):
        k = min(chi_keep, mps.chi(b))
        out.lambdas[b] = mps.lambdas[b][:k].copy()
    for s in range(mps.n_sites):
        kl = out.chi(s - 1)
        kr = out.chi(s)
        out.gammas[s] = mps.gammas[s][:, :kl, :kr].copy()
    return out


def scale_to_unit_norm(mps: Vidal) -> Vidal:
    """Multiply the state by 1/n (n = its norm): every Lambda_b is divided by n
    and the Gamma of every interior site multiplied by n, a factor
    n^-(N-1) n^(N-2) = 1/n (N = 1: Gamma_0 / n).  A state that is in canonical
    form up to a scalar (what PtSU converges to from a state of norm n,
    Sec. III D) becomes the canonical form of the normalised state: the
    conditions on A_i = Lambda_{i-1} Gamma_i and B_i = Gamma_i Lambda_i hold at
    every site afterwards, the end sites included."""
    out = mps.copy()
    n = norm(mps)
    if mps.n_sites == 1:
        out.gammas[0] = out.gammas[0] / n
        return out
    out.lambdas = [l / n for l in out.lambdas]
    for s in range(1, mps.n_sites - 1):
        out.gammas[s] = out.gammas[s] * n
    return out


# --------------------------------------------------------------------------
# Sampling (Sec. IV A: bit strings are drawn from the final state)
# --------------------------------------------------------------------------

def left_environments(mps: Vidal) -> list:
    """L[s] = the transfer matrix of sites 0..s-1 (L[0] = (1)):
    L[s+1] = sum_sigma M_s[sigma]^dag L[s] M_s[sigma], M_s = Gamma_s Lambda_s."""
    envs = [np.ones((1, 1), dtype=np.complex128)]
    for s in range(mps.n_sites):
        m = _site_matrix(mps, s)
        envs.append(_transfer(envs[-1], m, m))
    return envs


def sample(mps: Vidal, uniforms: np.ndarray) -> np.ndarray:
    """Bit strings drawn from |Psi|^2 / <Psi|Psi> (exact for any MPS), site by
    site from the right end: with the suffix vector v (chi_s x 1),
    P(sigma | suffix) is proportional to t^dag L[s] t with t = M_s[sigma] v;
    sigma = 0 when u < P(0 | suffix).  uniforms: (n_samples, N) numbers in
    [0, 1), uniforms[k, s] used for site s of sample k."""
    u = np.asarray(uniforms, dtype=np.float64)
    envs = left_environments(mps)
    out = np.zeros(u.shape, dtype=np.int32)
    for k in range(u.shape[0]):
        v = np.ones((1, 1), dtype=np.complex128)
        for s in range(mps.n_sites - 1, -1, -1):
            m = _site_matrix(mps, s)
            t = [m[x] @ v for x in range(2)]
            w = [float((t[x].conj().T @ envs[s] @ t[x]).real[0, 0]) for x in range(2)]
            p0 = w[0] / (w[0] + w[1])
            x = 0 if u[k, s] < p0 else 1
            out[k, s] = x
            v = t[x] / np.linalg.norm(t[x])
    return out
