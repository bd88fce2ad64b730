"""ORACLE -- test infrastructure only. Parallel-transport convolution (PTC) layers and the linear
PTC preconditioner network, plus their gradients, in plain numpy FP64.

The paper has no learned preconditioner; this is the project's extension of its CG with a learned
preconditioner for a flexible CG. The layer follows the gauge-equivariant parallel-transport
convolutions of Lehner & Wettig (2023), read as:
    psi'_a(x) = sum_b sum_h W[a, b, h] (T_h psi_b)(x),   h in {0, +mu, -mu}, mu = 0..3   (9 hops)
    T_0 psi(x)   = psi(x)
    T_+mu psi(x) = F_mu(x) psi(x + mu)
    T_-mu psi(x) = F_mu(x - mu)^dag psi(x - mu)
with the folded fat links F (staggered phases and antiperiodic-t sign included, as in the Dslash).
Hop order h = 0, +x, +y, +z, +t, -x, -y, -z, -t. The network is two linear layers 1 -> C -> 1
(C = 8); its input is an even-site vector embedded in the full lattice (zeros on odd sites), and
its output is restricted to even sites.

Gradients use the Wirtinger convention G = dLoss/d(conj W): for a real loss, dLoss = 2 Re(conj(G) dW).
Only tests/ (and the benchmark's CPU leg) may import this module.
"""
from __future__ import annotations

import numpy as np

from . import from_full, to_full, volume

NHOP = 9


def hop(h):
    """(mu, sign) of hop h; (None, 0) for the identity."""
    if h == 0:
        return None, 0
    return (h - 1) % 4, (1 if h <= 4 else -1)


def neighbours(L, mu, k):
    """Lexicographic index of x + k*mu for every site x (periodic wrap)."""
    V = volume(L)
    idx = np.arange(V)
    c = [idx % L[0], (idx // L[0]) % L[1], (idx // (L[0] * L[1])) % L[2], idx // (L[0] * L[1] * L[2])]
    c[mu] = (c[mu] + k) % L[mu]
    return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]))


def transport(L, fat, psi, h):
    """T_h psi for psi of shape (V, 3); fat: folded fat links (V, 4, 3, 3)."""
    mu, s = hop(h)
    if mu is None:
        return psi.copy()
    if s > 0:
        n = neighbours(L, mu, +1)
        return np.einsum("nij,nj->ni", fat[:, mu], psi[n])
    n = neighbours(L, mu, -1)
    return np.einsum("nji,nj->ni", fat[n, mu].conj(), psi[n])


def transport_adjoint(L, fat, psi, h):
    """T_h^dag psi: T_0^dag = T_0, T_+mu^dag = T_-mu, T_-mu^dag = T_+mu."""
    if h == 0:
        return psi.copy()
    return transport(L, fat, psi, h + 4 if h <= 4 else h - 4)


def layer_inputs(L, fat, psi):
    """u[b, h] = T_h psi_b for psi of shape (Cin, V, 3) -> (Cin, 9, V, 3)."""
    return np.stack([np.stack([transport(L, fat, psi[b], h) for h in range(NHOP)]) for b in range(psi.shape[0])])


def layer_forward(L, fat, W, psi):
    """psi'_a = sum_{b,h} W[a,b,h] T_h psi_b; W (Cout, Cin, 9), psi (Cin, V, 3) -> (Cout, V, 3)."""
    u = layer_inputs(L, fat, psi)
    return np.einsum("abh,bhvc->avc", W, u)


def layer_backward(L, fat, W, psi, g_out):
    """Given g_out = dLoss/d(conj psi'), return (dLoss/d(conj W), dLoss/d(conj psi))."""
    u = layer_inputs(L, fat, psi)
    gW = np.einsum("bhvc,avc->abh", u.conj(), g_out)
    mixed = np.einsum("abh,avc->bhvc", W.conj(), g_out)  # sum_a conj(W[a,b,h]) g_a
    g_in = np.zeros_like(psi)
    for b in range(psi.shape[0]):
        for h in range(NHOP):
            g_in[b] += transport_adjoint(L, fat, mixed[b, h], h)
    return gW, g_in


def network_forward(L, fat, W1, W2, r_even):
    """z = N(r): even-site r (V/2, 3) -> even-site z (V/2, 3); returns (z, cache)."""
    psi0 = to_full(L, even=r_even)[None]
    psi1 = layer_forward(L, fat, W1, psi0)
    psi2 = layer_forward(L, fat, W2, psi1)
    return from_full(L, psi2[0], 0), (psi0, psi1)


def loss_and_grads(L, fat, W1, W2, bs, xs):
    """Mean over pairs of |N(b) - x|^2 / |x|^2 and its Wirtinger gradients (gW1, gW2)."""
    gW1 = np.zeros_like(W1)
    gW2 = np.zeros_like(W2)
    loss = 0.0
    n = len(bs)
    for b, x in zip(bs, xs):
        z, (psi0, psi1) = network_forward(L, fat, W1, W2, b)
        nx = np.vdot(x, x).real
        e = z - x
        loss += np.vdot(e, e).real / nx / n
        g2 = to_full(L, even=e / nx / n)[None]  # dLoss/d(conj psi2), even sites only
        a, g1 = layer_backward(L, fat, W2, psi1, g2)
        gW2 += a
        c, _ = layer_backward(L, fat, W1, psi0, g1)
        gW1 += c
    return loss, gW1, gW2


def init_weights(seed, c=8, scale=0.2):
    """Deterministic initial weights: layer 1 (c, 1, 9), layer 2 (1, c, 9), complex."""
    rng = np.random.default_rng(seed)
    W1 = (rng.standard_normal((c, 1, NHOP)) + 1j * rng.standard_normal((c, 1, NHOP))) * scale
    W2 = (rng.standard_normal((1, c, NHOP)) + 1j * rng.standard_normal((1, c, NHOP))) * scale
    return W1, W2


# ---------------------------------------------------------------- tied (Hermitian) network
def adjoint_hop(h):
    """Index of T_h^dag among the hops: 0 -> 0, +mu <-> -mu."""
    return 0 if h == 0 else (h + 4 if h <= 4 else h - 4)


def tie(W1):
    """Layer-2 weights that make layer 2 the adjoint of layer 1: W2[0][a][h] = conj(W1[a][0][adj(h)]).
    Then N = B^dag B (B = layer 1 on the embedded even-site input) is Hermitian positive semi-definite."""
    C = W1.shape[0]
    W2 = np.zeros((1, C, NHOP), np.complex128)
    for a in range(C):
        for h in range(NHOP):
            W2[0, a, h] = np.conj(W1[a, 0, adjoint_hop(h)])
    return W2


def loss_and_grads_tied(L, fat, W1, bs, xs):
    """Loss and dLoss/d(conj W1) of the tied network: the layer-1 gradient plus the layer-2
    gradient carried back through W2 = conj(W1 o adj)."""
    W2 = tie(W1)
    loss, g1, g2 = loss_and_grads(L, fat, W1, W2, bs, xs)
    G = g1.copy()
    for a in range(W1.shape[0]):
        for h in range(NHOP):
            G[a, 0, h] += np.conj(g2[0, a, adjoint_hop(h)])
    return loss, G
