"""Pins of the smearing oracle (oracle/smear.py) against results fixed by the mathematics, not by the
oracle's own code: closed forms on unit links and on a constant abelian field strength, gauge
covariance, the nested single-staple construction that defines the fat7 paths, and the polar
decomposition (scipy) for the U(3) projection."""
import numpy as np
import pytest

import hisq_inputs as hin
from oracle import smear as sm
from oracle import volume, coords

# fat7 level: the product over the three transverse directions of (1 + Delta_rho^2 / 4), expanded
# and symmetrised over orderings: one link (1/2)^3, a staple (1/4)(1/2)^2, a five-link staple
# (1/4)^2 (1/2) / 2!, a seven-link staple (1/4)^3 / 3!; the weights sum to 1 on unit links.
FAT7 = dict(c1=1 / 8, c3=1 / 16, c5=1 / 64, c7=1 / 384)
RANDOM = dict(c1=0.31, c3=-0.17, c5=0.053, c7=-0.029, cL=0.071, cN=-0.43)


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def test_path_counts_and_endpoints():
    for mu in range(4):
        p = sm.staple_paths(mu)
        assert [len(p[k]) for k in ("three", "five", "seven", "lepage")] == [6, 24, 48, 6]
        for kind, paths in p.items():
            assert len({tuple(s) for s in paths}) == len(paths), kind
            for steps in paths:
                disp = np.zeros(4, int)
                for d, s in steps:
                    disp[d] += s
                assert list(disp) == [int(d == mu) for d in range(4)]


def test_unit_links_closed_form():
    L = (4, 6, 4, 6)
    V = volume(L)
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    c = RANDOM
    F, Lg = sm.smear(L, U, **c)
    total = c["c1"] + 6 * c["c3"] + 24 * c["c5"] + 48 * c["c7"] + 6 * c["cL"]
    np.testing.assert_allclose(F, total * U, atol=1e-14)
    np.testing.assert_allclose(Lg, c["cN"] * U, atol=1e-14)
    F7, _ = sm.smear(L, U, **FAT7)
    np.testing.assert_allclose(F7, U, atol=1e-14)


@pytest.mark.parametrize("plane", [(0, 1), (2, 3), (3, 1)])
def test_constant_abelian_field_closed_form(plane):
    """U_beta(x) = exp(i B x_alpha) (a constant field strength B in the alpha-beta plane), all other
    links 1. A closed path picks up exp(i B * signed area) of its projection on that plane; counting the
    staples that enclose one plaquette (either orientation) gives, for mu in {alpha, beta},
      F_mu / U_mu = c1 + c3 (2 cos B + 4) + c5 (16 cos B + 8) + c7 (48 cos B) + cL (2 cos 2B + 4)
    and the plain coefficient sum for the other two directions."""
    a, b = plane
    L = (6, 4, 8, 6)
    V = volume(L)
    B = 2 * np.pi / L[a]
    xa = coords(L, np.arange(V))[a]
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    U[:, b] *= np.exp(1j * B * xa)[:, None, None]
    c = RANDOM
    F, Lg = sm.smear(L, U, **c)
    flux = (c["c1"] + c["c3"] * (2 * np.cos(B) + 4) + c["c5"] * (16 * np.cos(B) + 8) + c["c7"] * 48 * np.cos(B)
            + c["cL"] * (2 * np.cos(2 * B) + 4))
    free = c["c1"] + 6 * c["c3"] + 24 * c["c5"] + 48 * c["c7"] + 6 * c["cL"]
    for mu in range(4):
        want = (flux if mu in plane else free) * U[:, mu]
        np.testing.assert_allclose(F[:, mu], want, atol=1e-13)
        naik = c["cN"] * (np.exp(3j * B * xa)[:, None, None] * np.eye(3) if mu == b else np.eye(3))
        np.testing.assert_allclose(Lg[:, mu], np.broadcast_to(naik, (V, 3, 3)), atol=1e-13)


def shift(L, d, k):
    idx = np.arange(volume(L))
    c = list(coords(L, idx))
    c[d] = (c[d] + k) % L[d]
    return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]))


def test_gauge_covariance():
    """F_mu(x) -> O(x) F_mu(x) O(x+mu)^dag and L_mu(x) -> O(x) L_mu(x) O(x+3mu)^dag under
    U_mu(x) -> O(x) U_mu(x) O(x+mu)^dag, for links that are not unitary."""
    L = (4, 6, 4, 8)
    V = volume(L)
    U = hin.gen_thin(L, 11, 0.4).reshape(V, 4, 3, 3)
    U = U + 0.2 * hin.gen_links(L, 12, 0.3, 1.0)[0].reshape(V, 4, 3, 3)
    Om = hin.gen_gauge_xform(L, 13)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[:, mu] = Om @ U[:, mu] @ dag(Om[shift(L, mu, 1)])
    F, Lg = sm.smear(L, U, **RANDOM)
    Fg, Lgg = sm.smear(L, Ug, **RANDOM)
    for mu in range(4):
        np.testing.assert_allclose(Fg[:, mu], Om @ F[:, mu] @ dag(Om[shift(L, mu, 1)]), atol=1e-12)
        np.testing.assert_allclose(Lgg[:, mu], Om @ Lg[:, mu] @ dag(Om[shift(L, mu, 3)]), atol=1e-12)


def staple(L, U, X, mu, nu, sign):
    """One-signed staple of the link field X (in direction mu) in direction nu: the single smearing
    step that the fat7 construction nests."""
    if sign > 0:
        return U[:, nu] @ X[shift(L, nu, 1)] @ dag(U[shift(L, mu, 1), nu])
    m = shift(L, nu, -1)
    return dag(U[m, nu]) @ X[m] @ U[shift(L, mu, 1)[m], nu]


def test_paths_equal_nested_staples():
    """The five- and seven-link staples are staples of staples (rho around the nu-staple, sigma around
    that), the Lepage term the same-signed staple of a staple in one direction: summing those nested
    products reproduces the enumerated paths."""
    L = (4, 4, 6, 4)
    V = volume(L)
    U = hin.gen_thin(L, 21, 0.5).reshape(V, 4, 3, 3) + 0.1 * hin.gen_links(L, 22, 0.3, 1.0)[0].reshape(V, 4, 3, 3)
    c = dict(c1=0.7, c3=0.11, c5=-0.05, c7=0.013, cL=-0.09, cN=0.0)
    F, _ = sm.smear(L, U, **c)
    for mu in range(4):
        others = [d for d in range(4) if d != mu]
        want = c["c1"] * U[:, mu]
        for nu in others:
            for s in (1, -1):
                s3 = staple(L, U, U[:, mu], mu, nu, s)
                want = want + c["c3"] * s3 + c["cL"] * staple(L, U, s3, mu, nu, s)
                for rho in others:
                    if rho == nu:
                        continue
                    for r in (1, -1):
                        s5 = staple(L, U, s3, mu, rho, r)
                        want = want + c["c5"] * s5
                        sig = [d for d in others if d not in (nu, rho)][0]
                        for q in (1, -1):
                            want = want + c["c7"] * staple(L, U, s5, mu, sig, q)
        np.testing.assert_allclose(F[:, mu], want, atol=1e-12)


def test_project_u3_polar_decomposition():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(5)
    # well-conditioned, like a smeared link (the projection squares the condition number)
    W = 2 * np.eye(3) + 0.5 * (rng.normal(size=(50, 3, 3)) + 1j * rng.normal(size=(50, 3, 3)))
    P = sm.project_u3(W)
    np.testing.assert_allclose(dag(P) @ P, np.broadcast_to(np.eye(3), P.shape), atol=1e-13)
    for k in range(len(W)):
        u, _ = scipy_linalg.polar(W[k], side="right")
        np.testing.assert_allclose(P[k], u, atol=1e-12)
    # a unitary matrix is its own projection; V H (H Hermitian positive) projects to V
    Vu = sm.project_u3(rng.normal(size=(20, 3, 3)) + 1j * rng.normal(size=(20, 3, 3)))
    np.testing.assert_allclose(sm.project_u3(Vu), Vu, atol=1e-13)
    G = rng.normal(size=(20, 3, 3)) + 1j * rng.normal(size=(20, 3, 3))
    H = dag(G) @ G + 0.5 * np.eye(3)
    np.testing.assert_allclose(sm.project_u3(Vu @ H), Vu, atol=1e-12)


def test_two_level_unit_links():
    """Level 1 (fat7) of unit links is the unit field, which the projection keeps; level 2 then gives
    the coefficient sum and the Naik coefficient."""
    L = (4, 4, 4, 4)
    V = volume(L)
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    W, _ = sm.smear(L, U, **FAT7)
    W = sm.project_u3(W)
    np.testing.assert_allclose(W, U, atol=1e-14)
    F, Lg = sm.smear(L, W, **RANDOM)
    total = RANDOM["c1"] + 6 * RANDOM["c3"] + 24 * RANDOM["c5"] + 48 * RANDOM["c7"] + 6 * RANDOM["cL"]
    np.testing.assert_allclose(F, total * U, atol=1e-14)


def test_two_levels_gauge_covariant():
    """Each level and the U(3) projection are covariant (W -> O W O'^dag gives W (W^dag W)^(-1/2) ->
    O [W (W^dag W)^(-1/2)] O'^dag), so the HISQ fat and long links transform like single links."""
    L = (4, 6, 4, 6)
    V = volume(L)
    U = hin.gen_thin(L, 31, 0.4).reshape(V, 4, 3, 3)
    Om = hin.gen_gauge_xform(L, 32)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[:, mu] = Om @ U[:, mu] @ dag(Om[shift(L, mu, 1)])
    level2 = dict(c1=5 / 8, c3=1 / 16, c5=1 / 64, c7=1 / 384, cL=-1 / 16, cN=-1 / 24)
    F, Lg = sm.hisq_links(L, U, FAT7, level2)
    Fg, Lgg = sm.hisq_links(L, Ug, FAT7, level2)
    for mu in range(4):
        np.testing.assert_allclose(Fg[:, mu], Om @ F[:, mu] @ dag(Om[shift(L, mu, 1)]), atol=1e-12)
        np.testing.assert_allclose(Lgg[:, mu], Om @ Lg[:, mu] @ dag(Om[shift(L, mu, 3)]), atol=1e-12)
