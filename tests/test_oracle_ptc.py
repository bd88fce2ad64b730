"""Pins for the oracle's PTC layers and network:

* identity-hop weights reduce a layer to a scalar multiple;
* weights +1 on the forward hops and -1 on the backward hops reproduce the fat-link part of the
  (independently pinned) staggered Dslash: sum_mu (T_+mu - T_-mu) psi = D_fat psi;
* T_+mu^dag = T_-mu numerically (adjointness used by the backward pass);
* gauge equivariance N_{Omega U}(Omega r) = Omega N_U(r); linearity;
* gradients against central finite differences in FP64.
"""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
import oracle.ptc as ptc
from test_oracle_dslash import folded, random_vec, transform_links

L = (4, 6, 8, 10)


@pytest.fixture(scope="module")
def fat():
    return folded(L, seed=321)[0]


def test_identity_hop_is_scalar(fat):
    rng = np.random.default_rng(1)
    psi = random_vec(rng, oracle.volume(L))[None]
    W = np.zeros((1, 1, 9), np.complex128)
    W[0, 0, 0] = 0.7 - 0.2j
    out = ptc.layer_forward(L, fat, W, psi)
    assert np.abs(out[0] - (0.7 - 0.2j) * psi[0]).max() < 1e-15


def test_hops_reproduce_fat_dslash(fat):
    rng = np.random.default_rng(2)
    psi = random_vec(rng, oracle.volume(L))
    W = np.zeros((1, 1, 9), np.complex128)
    W[0, 0, 1:5] = 1.0
    W[0, 0, 5:9] = -1.0
    out = ptc.layer_forward(L, fat, W, psi[None])[0]
    ref = oracle.dslash_full(L, fat, None, psi)
    assert np.abs(out - ref).max() < 1e-13


@pytest.mark.parametrize("h", range(1, 9))
def test_transport_adjoint(fat, h):
    rng = np.random.default_rng(3 + h)
    u, v = random_vec(rng, oracle.volume(L)), random_vec(rng, oracle.volume(L))
    lhs = np.vdot(v, ptc.transport(L, fat, u, h))
    rhs = np.vdot(ptc.transport_adjoint(L, fat, v, h), u)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_network_equivariance_and_linearity():
    fat, lng = folded(L, seed=77)
    W1, W2 = ptc.init_weights(5)
    omega = hin.gen_gauge_xform(L, 55, 1.0)
    f2, _ = transform_links(L, fat, lng, omega)
    rng = np.random.default_rng(4)
    n = oracle.volume(L) // 2
    r = random_vec(rng, n)
    ev = oracle.parity_sites(L, 0)
    z, _ = ptc.network_forward(L, fat, W1, W2, r)
    z2, _ = ptc.network_forward(L, f2, W1, W2, np.einsum("nij,nj->ni", omega[ev], r))
    assert np.abs(z2 - np.einsum("nij,nj->ni", omega[ev], z)).max() < 1e-13 * np.abs(z).max()
    r2 = random_vec(rng, n)
    a = 0.3 - 1.1j
    za, _ = ptc.network_forward(L, fat, W1, W2, a * r + r2)
    zb, _ = ptc.network_forward(L, fat, W1, W2, r2)
    assert np.abs(za - (a * z + zb)).max() < 1e-13 * np.abs(za).max()


def test_gradients_finite_differences():
    fat, _ = folded(L, seed=88)
    W1, W2 = ptc.init_weights(6)
    n = oracle.volume(L) // 2
    bs = hin.gen_source(10, n, 2)
    xs = hin.gen_source(20, n, 2)
    loss, g1, g2 = ptc.loss_and_grads(L, fat, W1, W2, list(bs), list(xs))
    rng = np.random.default_rng(7)
    eps = 1e-6
    for which, W, G in (("W1", W1, g1), ("W2", W2, g2)):
        for _ in range(4):
            idx = tuple(int(rng.integers(0, s)) for s in W.shape)
            for d in (1.0, 1j):
                Wp, Wm = W.copy(), W.copy()
                Wp[idx] += eps * d
                Wm[idx] -= eps * d
                args_p = (Wp, W2) if which == "W1" else (W1, Wp)
                args_m = (Wm, W2) if which == "W1" else (W1, Wm)
                lp = ptc.loss_and_grads(L, fat, *args_p, list(bs), list(xs))[0]
                lm = ptc.loss_and_grads(L, fat, *args_m, list(bs), list(xs))[0]
                fd = (lp - lm) / (2 * eps)
                an = 2 * (np.conj(G[idx]) * d).real
                assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (which, idx, d, fd, an)


def test_input_gradient_finite_differences(fat):
    rng = np.random.default_rng(9)
    V = oracle.volume(L)
    W = (rng.standard_normal((3, 2, 9)) + 1j * rng.standard_normal((3, 2, 9))) * 0.3
    psi = np.stack([random_vec(rng, V) for _ in range(2)])
    tgt = np.stack([random_vec(rng, V) for _ in range(3)])

    def loss(p):
        e = ptc.layer_forward(L, fat, W, p) - tgt
        return np.vdot(e, e).real

    g_out = ptc.layer_forward(L, fat, W, psi) - tgt
    _, g_in = ptc.layer_backward(L, fat, W, psi, g_out)
    eps = 1e-3  # the loss is exactly quadratic in psi: central differences carry only roundoff
    for _ in range(6):
        idx = (int(rng.integers(0, 2)), int(rng.integers(0, V)), int(rng.integers(0, 3)))
        for d in (1.0, 1j):
            pp, pm = psi.copy(), psi.copy()
            pp[idx] += eps * d
            pm[idx] -= eps * d
            fd = (loss(pp) - loss(pm)) / (2 * eps)
            an = 2 * (np.conj(g_in[idx]) * d).real
            assert abs(fd - an) <= 1e-8 * max(1.0, abs(an))


def test_tied_network_is_hermitian_psd():
    fat, _ = folded(L, seed=99)
    W1, _ = ptc.init_weights(8)
    W2 = ptc.tie(W1)
    rng = np.random.default_rng(12)
    n = oracle.volume(L) // 2
    u, v = random_vec(rng, n), random_vec(rng, n)
    Nu, _ = ptc.network_forward(L, fat, W1, W2, u)
    Nv, _ = ptc.network_forward(L, fat, W1, W2, v)
    assert abs(np.vdot(u, Nv) - np.conj(np.vdot(v, Nu))) < 1e-12 * abs(np.vdot(u, Nv))
    assert np.vdot(v, Nv).real > 0 and abs(np.vdot(v, Nv).imag) < 1e-12 * np.vdot(v, Nv).real
    # N v = B^dag B v: <v, N v> equals the squared norm of the layer-1 output
    psi1 = ptc.layer_forward(L, fat, W1, oracle.to_full(L, even=v)[None])
    assert abs(np.vdot(v, Nv).real - np.vdot(psi1, psi1).real) < 1e-10 * np.vdot(psi1, psi1).real


def test_tied_gradient_finite_differences():
    fat, _ = folded(L, seed=101)
    W1, _ = ptc.init_weights(9)
    n = oracle.volume(L) // 2
    bs = list(hin.gen_source(31, n, 2))
    xs = list(hin.gen_source(32, n, 2))
    loss, G = ptc.loss_and_grads_tied(L, fat, W1, bs, xs)
    rng = np.random.default_rng(13)
    eps = 1e-6
    for _ in range(6):
        idx = tuple(int(rng.integers(0, s)) for s in W1.shape)
        for d in (1.0, 1j):
            Wp, Wm = W1.copy(), W1.copy()
            Wp[idx] += eps * d
            Wm[idx] -= eps * d
            fd = (ptc.loss_and_grads_tied(L, fat, Wp, bs, xs)[0] - ptc.loss_and_grads_tied(L, fat, Wm, bs, xs)[0]) / (
                2 * eps)
            an = 2 * (np.conj(G[idx]) * d).real
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (idx, d, fd, an)
