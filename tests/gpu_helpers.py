"""Shared helpers of the GPU parity tests: move states between the CUDA
library (through its C ABI) and the oracle, and compare gauge-invariant
results (Lambda, chi, eps, fidelities)."""
import numpy as np

import oracle


def to_oracle(st) -> "oracle.Vidal":
    gammas, lambdas = st.export()
    return oracle.Vidal([np.array(g) for g in gammas], [np.array(l) for l in lambdas])


def load_into(st, mps: "oracle.Vidal"):
    st.load(mps.gammas, mps.lambdas)


def fidelity(a: "oracle.Vidal", b: "oracle.Vidal") -> float:
    ab = oracle.overlap(a, b)
    return abs(ab) ** 2 / (oracle.overlap(a, a).real * oracle.overlap(b, b).real)


def compare_spectra(lg, lo, tol, thr_rel, chi_max):
    """Normwise comparison of two singular-value vectors (descending):
    |lg_a - lo_a| <= tol * lo_1 over the common prefix, and the kept counts
    agree unless a value lies within tol * lo_1 of the threshold or the two
    counts are both at chi_max.  Returns the largest normwise deviation."""
    lg = np.asarray(lg)
    lo = np.asarray(lo)
    n = min(len(lg), len(lo))
    dev = float(np.abs(lg[:n] - lo[:n]).max() / lo[0]) if n else 0.0
    assert dev <= tol, f"spectrum deviates by {dev:.3e} > {tol:.1e}"
    if len(lg) != len(lo):
        longer = lg if len(lg) > len(lo) else lo
        extra = longer[n:]
        assert np.all(np.abs(extra - thr_rel * lo[0]) <= tol * lo[0] + thr_rel * lo[0]), \
            f"kept counts differ ({len(lg)} vs {len(lo)}) away from the threshold"
    return dev


def mini_vidal(lam_left, gam_b, lam_b, gam_b1, lam_right):
    """A 4-site Vidal object whose bond 1 has the given environment, for
    running the oracle's single-bond update on sampled bonds of a large state."""
    dl = np.zeros((2, 1, gam_b.shape[1]), complex)
    dr = np.zeros((2, gam_b1.shape[2], 1), complex)
    return oracle.Vidal([dl, np.array(gam_b), np.array(gam_b1), dr],
                        [np.array(lam_left), np.array(lam_b), np.array(lam_right)])
