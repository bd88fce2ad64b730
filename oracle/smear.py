"""ORACLE (test infrastructure only) -- link smearing of the HISQ kind, written from its definition.

The HISQ action builds its fat and long links from the thin links by weighted sums of
parallel-transport paths, with a projection back onto U(3) between two smearing levels (the HISQ
action the paper's simulations use, Sec. 1; its coefficients are not in the paper and are inputs
here). One level maps links U to

  F_mu(x) = c1 U_mu(x)
          + c3 * (sum of the  6 three-link staples: nu, mu, -nu for nu != mu, both signs of nu)
          + c5 * (sum of the 24 five-link staples: rho, nu, mu, -nu, -rho; nu, rho, mu distinct)
          + c7 * (sum of the 48 seven-link staples: sigma, rho, nu, mu, -nu, -rho, -sigma; all distinct)
          + cL * (sum of the  6 Lepage staples: nu, nu, mu, -nu, -nu)
  L_mu(x) = cN U_mu(x) U_mu(x+mu) U_mu(x+2mu)

where a path (d1, d2, ...) from x is the ordered product of the links it walks (the link U_d(y)
for a step +d from y, U_d(y-d)^dag for a step -d). Every path is enumerated and multiplied out
explicitly. The U(3) projection is W -> W (W^dag W)^{-1/2}, computed with numpy's Hermitian
eigendecomposition. Only tests/ may import this module.

Pins (tests/test_oracle_smear.py, with planted mistakes in tests/test_oracle_mutations.py): closed
forms on unit links and on a constant abelian field strength, gauge covariance of fat and long links,
equality with the nested single-staple construction, and the polar decomposition from scipy.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import coords, volume


def _shift_index(L, d: int, k: int, idx):
    """Lexicographic index of x + k*d-hat for the sites x with lexicographic indices idx."""
    c = list(coords(L, idx))
    c[d] = (c[d] + k) % L[d]
    return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]))


def path_product(L, U, steps, sites=None):
    """Product of the links along `steps` (list of (direction, +1/-1)) starting at every site (or at
    the lexicographic indices `sites`). U: (V, 4, 3, 3) complex. Returns (n, 3, 3)."""
    at = np.arange(volume(L)) if sites is None else np.asarray(sites)  # current site of each walk
    M = np.broadcast_to(np.eye(3, dtype=np.complex128), (len(at), 3, 3)).copy()
    for d, s in steps:
        if s > 0:
            M = M @ U[at, d]
            at = _shift_index(L, d, +1, at)
        else:
            at = _shift_index(L, d, -1, at)
            M = M @ np.conj(np.swapaxes(U[at, d], -1, -2))
    return M


def staple_paths(mu: int):
    """The paths of each kind for direction mu: dict kind -> list of step lists."""
    others = [d for d in range(4) if d != mu]
    paths = {"three": [], "five": [], "seven": [], "lepage": []}
    for nu in others:
        for s in (1, -1):
            paths["three"].append([(nu, s), (mu, 1), (nu, -s)])
            paths["lepage"].append([(nu, s), (nu, s), (mu, 1), (nu, -s), (nu, -s)])
    for nu, rho in itertools.permutations(others, 2):
        for s, r in itertools.product((1, -1), repeat=2):
            paths["five"].append([(rho, r), (nu, s), (mu, 1), (nu, -s), (rho, -r)])
    for nu, rho, sigma in itertools.permutations(others, 3):
        for s, r, q in itertools.product((1, -1), repeat=3):
            paths["seven"].append([(sigma, q), (rho, r), (nu, s), (mu, 1), (nu, -s), (rho, -r), (sigma, -q)])
    return paths


def smear(L, U, c1=0.0, c3=0.0, c5=0.0, c7=0.0, cL=0.0, cN=0.0, sites=None):
    """One smearing level. U: (V, 4, 3, 3) complex128. Returns (fat, long), each (V, 4, 3, 3), or
    (len(sites), 4, 3, 3) for the links of the given sites only."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    sel = np.arange(volume(L)) if sites is None else np.asarray(sites)
    F = c1 * U[sel].copy()
    Lg = np.zeros_like(F)
    for mu in range(4):
        paths = staple_paths(mu)
        for kind, coef in (("three", c3), ("five", c5), ("seven", c7), ("lepage", cL)):
            if coef == 0.0:
                continue
            for steps in paths[kind]:
                F[:, mu] += coef * path_product(L, U, steps, sel)
        if cN != 0.0:
            Lg[:, mu] = cN * path_product(L, U, [(mu, 1), (mu, 1), (mu, 1)], sel)
    return F, Lg


def project_u3(W):
    """W (W^dag W)^{-1/2} for every 3x3 matrix of W (..., 3, 3): the nearest U(3) matrix."""
    Q = np.conj(np.swapaxes(W, -1, -2)) @ W
    lam, vec = np.linalg.eigh(Q)
    inv_sqrt = (vec * (1.0 / np.sqrt(lam))[..., None, :]) @ np.conj(np.swapaxes(vec, -1, -2))
    return W @ inv_sqrt


def hisq_links(L, U, level1, level2):
    """The two HISQ levels: V = level-1 smearing of U (its fat part), W = project_u3(V), then the
    level-2 smearing of W gives the fat links and W's Naik product the long links. level1, level2:
    coefficient dicts for smear()."""
    V, _ = smear(L, U, **level1)
    W = project_u3(V)
    return smear(L, W, **level2)
