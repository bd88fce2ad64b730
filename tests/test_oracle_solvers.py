"""Pins for the oracle's solvers.

* Free field: A is diagonal in (antiperiodic-in-t) momentum space, so the exact solution of
  (A + sigma) x = b follows from an FFT; CG and every shift of multi-shift CG must reach it.
* General fields: the true FP64 residual, recomputed from the operator, meets the tolerance,
  and each multi-shift solution agrees with an independent single-shift CG.
"""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
from test_oracle_dslash import FLAGS, folded, unit_links


def fft_solve(L, mass, sigma, b_even):
    """x = (4m^2 + sigma - D^2)^-1 b on the full lattice at unit links (exact, via FFT)."""
    Lx, Ly, Lz, Lt = L
    full = oracle.to_full(L, even=b_even).reshape(Lt, Lz, Ly, Lx, 3)
    t = np.arange(Lt).reshape(Lt, 1, 1, 1, 1)
    twist = np.exp(1j * np.pi * t / Lt)  # antiperiodic in t -> periodic after the twist
    g = np.fft.fftn(full / twist, axes=(0, 1, 2, 3))
    ks = [2 * np.pi * (np.fft.fftfreq(n) * n + (0.5 if ax == 0 else 0.0)) / n
          for ax, n in enumerate((Lt, Lz, Ly, Lx))]
    Pt, Pz, Py, Px = np.meshgrid(*ks, indexing="ij")
    s = sum((np.sin(p) - np.sin(3 * p) / 24) ** 2 for p in (Px, Py, Pz, Pt))
    lam = (4 * mass ** 2 + sigma + 4 * s)[..., None]
    x = np.fft.ifftn(g / lam, axes=(0, 1, 2, 3)) * twist
    x = x.reshape(-1, 3)
    return oracle.from_full(L, x, 0), oracle.from_full(L, x, 1)


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (4, 6, 8, 10)])
def test_cg_free_field_exact(L):
    mass = 0.1
    fat, lng = oracle.fold_links(L, *unit_links(L), FLAGS)
    b = hin.gen_source(2000, oracle.volume(L) // 2)[0]
    x_exact, x_odd = fft_solve(L, mass, 0.0, b)
    assert np.abs(x_odd).max() < 1e-12  # the even source stays on even sites
    # the FFT solution satisfies the oracle operator (ties FFT conventions to the operator)
    assert oracle.true_residual(L, fat, lng, mass, b, x_exact) < 1e-13
    x, it = oracle.cg(L, fat, lng, mass, b, tol=1e-12)
    assert it > 0
    assert np.linalg.norm(x - x_exact) / np.linalg.norm(x_exact) < 1e-10


def test_multishift_free_field_exact():
    L = (4, 6, 8, 10)
    mass = 0.0025
    sigmas = np.logspace(-5, 0, 14)
    fat, lng = oracle.fold_links(L, *unit_links(L), FLAGS)
    b = hin.gen_source(2002, oracle.volume(L) // 2)[0]
    xs, its, base = oracle.multishift_cg(L, fat, lng, mass, sigmas, b, 1e-11)
    assert all(i >= 0 for i in its)
    for k, s in enumerate(sigmas):
        x_exact, _ = fft_solve(L, mass, s, b)
        assert np.linalg.norm(xs[k] - x_exact) / np.linalg.norm(x_exact) < 1e-9


def test_cg_random_field_true_residual():
    """The 8^4 plain-method workload: m = 0.1, eps = 0.3 links, Gaussian source, to 1e-10."""
    L = (8, 8, 8, 8)
    fat, lng = folded(L, seed=1000)
    b = hin.gen_source(2000, oracle.volume(L) // 2)[0]
    x, it = oracle.cg(L, fat, lng, 0.1, b, tol=1e-10)
    assert it > 0
    assert oracle.true_residual(L, fat, lng, 0.1, b, x) < 1.5e-10


def test_cg_initial_guess_and_shift():
    L = (4, 6, 8, 10)
    fat, lng = folded(L, seed=5)
    b = hin.gen_source(7, oracle.volume(L) // 2)[0]
    x1, _ = oracle.cg(L, fat, lng, 0.05, b, tol=1e-12, sigma=0.3)
    assert oracle.true_residual(L, fat, lng, 0.05, b, x1, sigma=0.3) < 2e-12
    # a converged guess needs no further iterations
    x2, it = oracle.cg(L, fat, lng, 0.05, b, tol=1e-10, sigma=0.3, x0=x1)
    assert it == 0 and np.array_equal(x1, x2)


def test_multishift_matches_single_shift():
    L = (4, 6, 8, 10)
    mass = 0.0025
    fat, lng = folded(L, seed=1002)
    b = hin.gen_source(2002, oracle.volume(L) // 2)[0]
    sigmas = np.logspace(-5, 0, 14)
    xs, its, base = oracle.multishift_cg(L, fat, lng, mass, sigmas, b, 1e-10)
    assert all(i >= 0 for i in its)
    assert its[0] == base  # the smallest shift converges last
    for k, s in enumerate(sigmas):
        r = oracle.true_residual(L, fat, lng, mass, b, xs[k], sigma=s)
        assert r < 1e-9
        xk, _ = oracle.cg(L, fat, lng, mass, b, tol=1e-12, sigma=s)
        assert np.linalg.norm(xs[k] - xk) / np.linalg.norm(xk) < 1e-7


def test_rational_apply_matches_eigendecomposition():
    """Closed form on 4^4: r(A) b = V diag(a0 + sum_k a_k / (lambda + sigma_k)) V^dag b from a dense
    eigendecomposition of the oracle's A (numpy), against the multi-shift route."""
    from test_oracle_dslash import dense_A
    L = (4, 4, 4, 4)
    mass = 0.05
    fat, lng = folded(L, seed=1234)
    A = dense_A(L, fat, lng, mass)
    lam, V = np.linalg.eigh(A)
    b = hin.gen_source(55, oracle.volume(L) // 2)[0]
    a0, coeffs, sigmas = 0.3, [0.5, 0.2, 1.1], [0.01, 0.2, 1.5]
    f = a0 + sum(a / (lam + s) for a, s in zip(coeffs, sigmas))
    ref = (V @ (f * (V.conj().T @ b.ravel()))).reshape(-1, 3)
    got = oracle.rational_apply(L, fat, lng, mass, b, a0, coeffs, sigmas, tol=1e-13)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
