"""Pins for the oracle's operator: what the mathematics fixes, independently of the oracle's code.

* point-source probe (brute force): D_eo applied to a delta is non-zero only at the 16 hop
  targets, with values read straight off the link arrays;
* free field (closed form): the spectrum of A = 4m^2 - D_eo D_oe at unit links is
  4m^2 + 4 sum_mu (c1 sin p_mu + c3 sin 3p_mu)^2 with antiperiodic momenta in t;
* gauge covariance under random SU(3) transformations;
* anti-hermiticity D_eo^dag = -D_oe;
* A Hermitian and bounded below by 4m^2 (dense, 4^4).
"""
import itertools

import numpy as np
import pytest

import hisq_inputs as hin
import oracle

FLAGS = oracle.APPLY_PHASES | oracle.ANTIPERIODIC_T


def lex(L, c):
    return int((c[0] % L[0]) + L[0] * ((c[1] % L[1]) + L[1] * ((c[2] % L[2]) + L[2] * (c[3] % L[3]))))


def links(L, seed=1000, eps=0.3, noise=0.1):
    fat, lng = hin.gen_links(L, seed, eps, noise)
    return fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3)


def folded(L, seed=1000, eps=0.3, noise=0.1):
    fat, lng = links(L, seed, eps, noise)
    return oracle.fold_links(L, fat, lng, FLAGS)


def unit_links(L):
    V = oracle.volume(L)
    fat = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    lng = -fat / 24.0
    return fat, lng


def fold_signs(L, c, mu):
    """eta_mu(x) and the antiperiodic-t sign of the fat and long link at site c, direction mu."""
    eta = (-1) ** (sum(c[:mu]) % 2)
    sf = sl = eta
    if mu == 3 and c[3] == L[3] - 1:
        sf = -sf
    if mu == 3 and c[3] >= L[3] - 3:
        sl = -sl
    return sf, sl


def random_vec(rng, n):
    return rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))


# ----------------------------------------------------------------------------- fold

def test_fold_flags():
    L = (4, 4, 4, 6)
    fat, lng = links(L)
    f0, l0 = oracle.fold_links(L, fat, lng, 0)
    assert np.array_equal(f0, fat) and np.array_equal(l0, lng)
    f1, l1 = oracle.fold_links(L, fat, lng, FLAGS)
    rng = np.random.default_rng(1)
    for _ in range(50):
        c = [int(rng.integers(0, n)) for n in L]
        mu = int(rng.integers(0, 4))
        sf, sl = fold_signs(L, c, mu)
        i = lex(L, c)
        assert np.array_equal(f1[i, mu], sf * fat[i, mu]) and np.array_equal(l1[i, mu], sl * lng[i, mu])


# ----------------------------------------------------------------------------- point-source probe

@pytest.mark.parametrize("L", [(8, 10, 12, 14), (4, 6, 8, 10)])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_point_source_probe(L, out_parity):
    """Brute force: D applied to delta_{y,c}; expected values read off the raw link arrays."""
    fat_raw, lng_raw = links(L, seed=11)
    fat, lng = oracle.fold_links(L, fat_raw, lng_raw, FLAGS)
    V = oracle.volume(L)
    in_sites = oracle.parity_sites(L, 1 - out_parity)
    out_sites = oracle.parity_sites(L, out_parity)
    out_pos = {int(s): k for k, s in enumerate(out_sites)}
    rng = np.random.default_rng(3)
    for trial in range(3):
        k = int(rng.integers(0, V // 2))
        y = int(in_sites[k])
        col = int(rng.integers(0, 3))
        cy = list(oracle.coords(L, y))
        vec = np.zeros((V // 2, 3), np.complex128)
        vec[k, col] = 1.0
        got = oracle.dslash(L, fat, lng, out_parity, vec)
        expect = np.zeros_like(got)
        for mu in range(4):
            for hop in (1, 3):
                # x = y - hop*mu: term +W_mu(x) chi(x + hop*mu) picks column col of W_mu(x)
                cx = list(cy)
                cx[mu] -= hop
                cx = [c % n for c, n in zip(cx, L)]
                xi = lex(L, cx)
                sf, sl = fold_signs(L, cx, mu)
                W = fat_raw[xi, mu] * sf if hop == 1 else lng_raw[xi, mu] * sl
                expect[out_pos[xi]] += W[:, col]
                # x = y + hop*mu: term -W_mu(y)^dag chi(y) picks -conj(row col of W_mu(y))
                cx = list(cy)
                cx[mu] += hop
                xi = lex(L, cx)
                sf, sl = fold_signs(L, cy, mu)
                W = fat_raw[y, mu] * sf if hop == 1 else lng_raw[y, mu] * sl
                expect[out_pos[xi]] -= W[col, :].conj()
        assert np.abs(got - expect).max() < 1e-15
        nz = np.count_nonzero(np.abs(got).sum(axis=1) > 0)
        if min(L) >= 8:
            assert nz == 16  # all 16 targets distinct
        else:
            assert nz < 16  # aliasing lattice: coinciding hops were accumulated


# ----------------------------------------------------------------------------- free field

def free_field_eigs(L, mass, sigma=0.0, c1=1.0, c3=-1.0 / 24.0):
    """Closed-form eigenvalues of 4m^2 + sigma - D^2 at unit links over all V momenta."""
    ps = []
    for mu, n in enumerate(L):
        k = np.arange(n)
        ps.append(2 * np.pi * (k + (0.5 if mu == 3 else 0.0)) / n)
    P = np.meshgrid(*ps, indexing="ij")
    s = sum((c1 * np.sin(p) + c3 * np.sin(3 * p)) ** 2 for p in P)
    return 4 * mass ** 2 + sigma + 4 * s


def dense_A(L, fat, lng, mass):
    n = oracle.volume(L) // 2 * 3
    A = np.empty((n, n), np.complex128)
    e = np.zeros(n, np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        A[:, j] = oracle.apply_A(L, fat, lng, mass, e.reshape(-1, 3)).ravel()
    return A


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (4, 6, 4, 8)])
def test_free_field_spectrum(L):
    mass = 0.1
    fat, lng = oracle.fold_links(L, *unit_links(L), FLAGS)
    A = dense_A(L, fat, lng, mass)
    assert np.abs(A - A.conj().T).max() < 1e-14
    ev = np.sort(np.linalg.eigvalsh(A))
    lam = np.sort(np.repeat(free_field_eigs(L, mass).ravel(), 3))[::2]  # p and p+pi pair up on one parity
    assert ev.shape == lam.shape
    assert np.abs(ev - lam).max() < 1e-12


def test_free_field_plane_wave():
    """A plane wave restricted to even sites is an eigenvector, on a lattice with distinct extents."""
    L = (6, 8, 10, 12)
    mass = 0.05
    fat, lng = oracle.fold_links(L, *unit_links(L), FLAGS)
    ev_sites = oracle.parity_sites(L, 0)
    x, y, z, t = oracle.coords(L, ev_sites)
    for n in [(1, 2, 3, 0), (0, 0, 0, 5), (5, 7, 9, 11)]:
        p = [2 * np.pi * n[0] / L[0], 2 * np.pi * n[1] / L[1], 2 * np.pi * n[2] / L[2],
             2 * np.pi * (n[3] + 0.5) / L[3]]
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        v = np.zeros((len(ev_sites), 3), np.complex128)
        v[:, 1] = phase
        lam = 4 * mass ** 2 + 4 * sum((np.sin(q) - np.sin(3 * q) / 24) ** 2 for q in p)
        assert np.abs(oracle.apply_A(L, fat, lng, mass, v) - lam * v).max() < 1e-12


def test_free_field_wrong_boundary_differs():
    """Periodic time (flags without the t sign) gives a different spectrum: the BC pin bites."""
    L = (4, 4, 4, 4)
    fat, lng = oracle.fold_links(L, *unit_links(L), oracle.APPLY_PHASES)
    ev = np.sort(np.linalg.eigvalsh(dense_A(L, fat, lng, 0.1)))
    lam = np.sort(np.repeat(free_field_eigs(L, 0.1).ravel(), 3))[::2]
    assert np.abs(ev - lam).max() > 1e-3


# ----------------------------------------------------------------------------- invariants

def transform_links(L, fat, lng, omega):
    """F_mu(x) -> O(x) F_mu(x) O(x+mu)^dag, L_mu(x) -> O(x) L_mu(x) O(x+3mu)^dag."""
    V = oracle.volume(L)
    idx = np.arange(V)
    c = np.stack(oracle.coords(L, idx), axis=1)
    f2, l2 = np.empty_like(fat), np.empty_like(lng)
    for mu in range(4):
        d1, d3 = c.copy(), c.copy()
        d1[:, mu] = (d1[:, mu] + 1) % L[mu]
        d3[:, mu] = (d3[:, mu] + 3) % L[mu]
        n1 = d1[:, 0] + L[0] * (d1[:, 1] + L[1] * (d1[:, 2] + L[2] * d1[:, 3]))
        n3 = d3[:, 0] + L[0] * (d3[:, 1] + L[1] * (d3[:, 2] + L[2] * d3[:, 3]))
        f2[:, mu] = omega @ fat[:, mu] @ omega[n1].conj().transpose(0, 2, 1)
        l2[:, mu] = omega @ lng[:, mu] @ omega[n3].conj().transpose(0, 2, 1)
    return f2, l2


@pytest.mark.parametrize("L", [(8, 10, 12, 14), (4, 6, 8, 10), (4, 4, 4, 4)])
def test_gauge_covariance(L):
    fat, lng = folded(L, seed=21)
    omega = hin.gen_gauge_xform(L, 99, 1.0)
    f2, l2 = transform_links(L, fat, lng, omega)
    rng = np.random.default_rng(5)
    V = oracle.volume(L)
    chi = random_vec(rng, V)
    lhs = oracle.dslash_full(L, f2, l2, np.einsum("nij,nj->ni", omega, chi))
    rhs = np.einsum("nij,nj->ni", omega, oracle.dslash_full(L, fat, lng, chi))
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()
    # the even/odd halves transform the same way
    for p in (0, 1):
        src = oracle.parity_sites(L, 1 - p)
        dst = oracle.parity_sites(L, p)
        v = chi[src]
        lhs = oracle.dslash(L, f2, l2, p, np.einsum("nij,nj->ni", omega[src], v))
        rhs = np.einsum("nij,nj->ni", omega[dst], oracle.dslash(L, fat, lng, p, v))
        assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()


@pytest.mark.parametrize("L", [(8, 10, 12, 14), (4, 6, 8, 10)])
def test_anti_hermiticity(L):
    fat, lng = folded(L, seed=31)
    rng = np.random.default_rng(7)
    n = oracle.volume(L) // 2
    u, v = random_vec(rng, n), random_vec(rng, n)
    lhs = np.vdot(u, oracle.dslash(L, fat, lng, 0, v))
    rhs = -np.vdot(oracle.dslash(L, fat, lng, 1, u), v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_dense_blocks_and_positivity():
    """Dense 4^4 brute force: D from the full-lattice operator, A = 4m^2 - D_eo D_oe, Hermitian, >= 4m^2."""
    L = (4, 4, 4, 4)
    mass = 0.1
    fat, lng = folded(L, seed=41)
    V = oracle.volume(L)
    D = np.empty((3 * V, 3 * V), np.complex128)
    e = np.zeros((V, 3), np.complex128)
    for j in range(3 * V):
        e[:] = 0
        e.ravel()[j] = 1
        D[:, j] = oracle.dslash_full(L, fat, lng, e).ravel()
    assert np.abs(D + D.conj().T).max() < 1e-14  # D anti-Hermitian on the full lattice
    ev, od = oracle.parity_sites(L, 0), oracle.parity_sites(L, 1)
    ce = (3 * ev[:, None] + np.arange(3)).ravel()
    co = (3 * od[:, None] + np.arange(3)).ravel()
    assert np.abs(D[np.ix_(ce, ce)]).max() == 0 and np.abs(D[np.ix_(co, co)]).max() == 0
    Deo, Doe = D[np.ix_(ce, co)], D[np.ix_(co, ce)]
    A = dense_A(L, fat, lng, mass)
    assert np.abs(A - (4 * mass ** 2 * np.eye(len(ce)) - Deo @ Doe)).max() < 1e-13
    assert np.abs(A - A.conj().T).max() < 1e-13
    assert np.linalg.eigvalsh(A).min() >= 4 * mass ** 2 - 1e-12
    # M = 2m + D: M^dag M restricted to even sites is A
    M = 2 * mass * np.eye(3 * V) + D
    MM = M.conj().T @ M
    assert np.abs(MM[np.ix_(ce, ce)] - A).max() < 1e-12
    assert np.abs(MM[np.ix_(ce, co)]).max() < 1e-12


def test_A_hermitian_positive_random():
    L = (8, 10, 12, 14)
    fat, lng = folded(L, seed=51)
    rng = np.random.default_rng(9)
    n = oracle.volume(L) // 2
    u, v = random_vec(rng, n), random_vec(rng, n)
    m = 0.05
    Au, Av = oracle.apply_A(L, fat, lng, m, u), oracle.apply_A(L, fat, lng, m, v)
    assert abs(np.vdot(u, Av) - np.conj(np.vdot(v, Au))) < 1e-12 * abs(np.vdot(u, Av))
    assert np.vdot(v, Av).real >= 4 * m * m * np.vdot(v, v).real


def test_dslash_sites_matches_dslash():
    L = (8, 10, 12, 14)
    fat, lng = folded(L, seed=61)
    rng = np.random.default_rng(11)
    n = oracle.volume(L) // 2
    v = random_vec(rng, n)
    for p in (0, 1):
        full = oracle.dslash(L, fat, lng, p, v)
        cbs = rng.choice(n, 100, replace=False)
        assert np.array_equal(oracle.dslash_sites(L, fat, lng, p, v, cbs), full[cbs])


def test_fat_only_and_long_only_sum():
    L = (4, 6, 8, 10)
    fat, lng = folded(L, seed=71)
    rng = np.random.default_rng(13)
    v = random_vec(rng, oracle.volume(L) // 2)
    both = oracle.dslash(L, fat, lng, 0, v)
    parts = oracle.dslash(L, fat, None, 0, v) + oracle.dslash(L, None, lng, 0, v)
    assert np.abs(both - parts).max() < 1e-14
