"""The seeded input generator: Philox known answers, link unitarity, the exp map, long links."""
import os

import numpy as np
import scipy.linalg

import hisq_inputs as hin

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    # Published Philox4x32-10 known-answer vectors (Random123, SC'11).
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(v, 16) for v in line.split()]
            assert hin.philox4x32_10(w[0:4], w[4:6]) == w[6:10]
            n += 1
    assert n == 3


def test_thin_links_are_su3():
    U = hin.gen_thin((4, 6, 4, 8), 1000, 0.3).reshape(-1, 3, 3)
    uu = np.einsum("nki,nkj->nij", U.conj(), U)
    assert np.abs(uu - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13


def test_thin_link_is_exp_of_generator():
    L = (4, 4, 4, 6)
    eps = 0.3
    thin = hin.gen_thin(L, 77, eps).reshape(-1, 4, 3, 3)
    for site, mu in [(0, 0), (5, 3), (123, 1), (383, 2)]:
        H = hin.thin_generator(L, 77, site, mu)
        assert np.allclose(H, H.conj().T, atol=0) and abs(np.trace(H)) < 1e-14
        assert np.allclose(thin[site, mu], scipy.linalg.expm(1j * eps * H), atol=1e-14, rtol=0)
        # Gell-Mann normalisation: tr(H^2) = sum_a h_a^2 / 2, the h_a being N(0,1) draws
    Hs = np.array([hin.thin_generator(L, 5, s, m) for s in range(400) for m in range(4)])
    tr = np.einsum("nij,nji->n", Hs, Hs).real
    assert abs(tr.mean() - 4.0) < 0.3  # E[sum of 8 squares]/2 = 4


def test_long_and_fat_links():
    L = (4, 6, 8, 6)
    eps, noise = 0.3, 0.1
    thin = hin.gen_thin(L, 9, eps)  # (Lt, Lz, Ly, Lx, 4, 3, 3)
    fat, lng = hin.gen_links(L, 9, eps, noise)
    Lx, Ly, Lz, Lt = L
    rng = np.random.default_rng(0)
    for _ in range(30):
        x, y, z, t, mu = (int(rng.integers(0, n)) for n in (Lx, Ly, Lz, Lt, 4))
        c = [x, y, z, t]

        def U(k):
            d = list(c)
            d[mu] = (d[mu] + k) % L[mu]
            return thin[d[3], d[2], d[1], d[0], mu]

        expect = -(U(0) @ U(1) @ U(2)) / 24.0
        assert np.allclose(lng[t, z, y, x, mu], expect, atol=1e-15, rtol=0)
    G = (fat - thin) / noise
    assert abs(np.mean(np.abs(G) ** 2) - 1.0) < 0.05
    assert abs(np.mean(G.real)) < 0.05 and abs(np.mean(G.imag)) < 0.05


def test_slab_generation_matches_whole():
    L = (4, 4, 6, 8)
    fat, lng = hin.gen_links(L, 3, 0.3, 0.1)
    f2, l2 = hin.gen_links(L, 3, 0.3, 0.1, t0=3, nt=4)
    assert np.array_equal(fat[3:7], f2) and np.array_equal(lng[3:7], l2)


def test_sources():
    s = hin.gen_source(2000, 5000, 3)
    assert s.shape == (3, 5000, 3)
    assert abs(np.mean(np.abs(s) ** 2) - 1.0) < 0.03
    assert not np.allclose(s[0], s[1])
    assert np.array_equal(hin.gen_source(2000, 5000, 1)[0], s[0])


def test_lattice_mix():
    mix = hin.lattice_mix_64()
    assert len(mix) == 64
    shapes = [m["dims"] for m in mix]
    assert shapes.count((16, 16, 16, 16)) == 32 and shapes.count((24, 24, 24, 8)) == 19
    assert shapes.count((32, 32, 32, 8)) == 13
    assert all(0.2 <= m["eps"] <= 0.4 and 0.005 <= m["mass"] <= 0.1 for m in mix)
