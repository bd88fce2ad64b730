"""The library's Lanczos estimate of A's extreme eigenvalues from CG coefficients (host code, no GPU).

CG's alpha_k, beta_k define the Lanczos tridiagonal matrix T of the operator on the Krylov space of the
source; its extreme eigenvalues approach the operator's. Pins, independent of the library:
  * T built here from random coefficients, its extremes from numpy's dense symmetric eigensolver;
  * CG run here (plain numpy) on a diagonal operator holding the closed-form free-field spectrum of
    A = 4m^2 - D_eo D_oe at unit links, lambda(p) = 4m^2 + 4 sum_mu (sin p_mu - sin(3 p_mu)/24)^2 with
    antiperiodic time momenta: run to convergence, the estimates equal that spectrum's min and max, and
    their ratio its condition number;
  * restart marks (alpha = 0) split the coefficients, and the longest run is used.
"""
import numpy as np
import pytest

from test_oracle_dslash import free_field_eigs


@pytest.fixture(scope="module")
def hisq():
    from paper_2111_10354_gb300 import build
    build.build()
    import paper_2111_10354_gb300 as h
    h.lib()
    return h


def tridiag(alpha, beta):
    n = len(alpha)
    T = np.zeros((n, n))
    for k in range(n):
        T[k, k] = 1 / alpha[k] + (beta[k - 1] / alpha[k - 1] if k > 0 else 0.0)
        if k + 1 < n:
            T[k, k + 1] = T[k + 1, k] = np.sqrt(beta[k]) / alpha[k]
    return T


def cg_coefficients(lam, b, tol):
    """Plain CG on diag(lam) x = b, returning its alpha_k and beta_k."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    al, be = [], []
    for _ in range(10 * len(b)):
        Ap = lam * p
        a = rr / (p @ Ap)
        x += a * p
        r -= a * Ap
        rr_new = r @ r
        al.append(a)
        be.append(rr_new / rr)
        if np.sqrt(rr_new) <= tol * np.linalg.norm(b):
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return np.array(al), np.array(be)


def test_extremes_match_dense_eigensolver(hisq):
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 60):
        alpha = rng.uniform(0.2, 3.0, n)
        beta = rng.uniform(0.01, 0.9, n)
        ev = np.linalg.eigvalsh(tridiag(alpha, beta))
        lo, hi = hisq.hisq_lanczos_extremes(alpha, beta)
        assert abs(lo - ev[0]) <= 1e-12 * abs(ev[-1]) and abs(hi - ev[-1]) <= 1e-12 * abs(ev[-1]), (n, lo, hi, ev)


@pytest.mark.parametrize("mass", [0.1, 0.01])
def test_free_field_condition_number(hisq, mass):
    L = (8, 8, 8, 8)
    lam_all = free_field_eigs(L, mass).ravel()
    lam = np.unique(np.round(lam_all, 13))  # the distinct eigenvalues (CG sees each once)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(len(lam)) + 1.0
    alpha, beta = cg_coefficients(lam, b, 1e-13)
    lo, hi = hisq.hisq_lanczos_extremes(alpha, beta)
    assert abs(lo - lam_all.min()) <= 1e-8 * lam_all.min()
    assert abs(hi - lam_all.max()) <= 1e-8 * lam_all.max()
    kappa = hi / lo
    assert abs(kappa / (lam_all.max() / lam_all.min()) - 1) < 1e-7


def test_restart_marks_split_the_coefficients(hisq):
    rng = np.random.default_rng(8)
    a1, b1 = rng.uniform(0.2, 3.0, 5), rng.uniform(0.01, 0.9, 5)
    a2, b2 = rng.uniform(0.2, 3.0, 12), rng.uniform(0.01, 0.9, 12)
    alpha = np.concatenate([a1, [0.0], a2])
    beta = np.concatenate([b1, [0.0], b2])
    ev = np.linalg.eigvalsh(tridiag(a2, b2))
    lo, hi = hisq.hisq_lanczos_extremes(alpha, beta)
    assert abs(lo - ev[0]) <= 1e-12 * ev[-1] and abs(hi - ev[-1]) <= 1e-12 * ev[-1]
    with pytest.raises(hisq.HisqError):
        hisq.hisq_lanczos_extremes(np.zeros(3), np.zeros(3))
