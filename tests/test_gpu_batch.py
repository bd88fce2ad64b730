"""Batched CG over lattices of uneven sizes through the C ABI: every lattice's solution is judged by
the oracle's true FP64 residual and compared with the single-lattice CG solution."""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle

pytestmark = pytest.mark.gpu

SMALL_MIX = [((8, 8, 8, 8), 0.1, 0.3), ((4, 6, 8, 10), 0.02, 0.25), ((8, 10, 12, 14), 0.05, 0.35),
             ((16, 16, 16, 16), 0.01, 0.3), ((8, 8, 8, 8), 0.007, 0.4)]


def build(hisq, mix, seed0=500):
    batch = hisq.Batch([m[0] for m in mix])
    folded, bs = [], []
    for l, (L, mass, eps) in enumerate(mix):
        fat, lng = hin.gen_links(L, seed0 + l, eps, 0.1)
        batch.load(l, fat, lng)
        folded.append(oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3)))
        bs.append(hin.gen_source(seed0 + 100 + l, oracle.volume(L) // 2, 1)[0])
    b = np.concatenate([v.reshape(-1) for v in bs]).reshape(-1, 3)
    return batch, folded, bs, b


@pytest.mark.parametrize("inner", [0, 1])
def test_batch_small_mix(hisq, inner):
    import torch
    batch, folded, bs, b = build(hisq, SMALL_MIX)
    masses = [m[1] for m in SMALL_MIX]
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    rc, st = batch.cg(x, torch.from_numpy(b).cuda(), masses, 1e-10, 5000, inner_prec=inner)
    assert rc == 0 and st["converged"] == 1
    xs = x.cpu().numpy()
    for l, (L, mass, eps) in enumerate(SMALL_MIX):
        o0, o1 = batch.offsets[l] // 3, batch.offsets[l + 1] // 3
        r = oracle.true_residual(L, folded[l][0], folded[l][1], mass, bs[l], xs[o0:o1])
        assert r <= 1e-10, (l, r)
        assert abs(r - st["lattice_residual"][l]) < 1e-11
        x_ref, _ = oracle.cg(L, folded[l][0], folded[l][1], mass, bs[l], tol=1e-12)
        assert np.linalg.norm(xs[o0:o1] - x_ref) / np.linalg.norm(x_ref) < 1e-7
    # lighter masses need more iterations; every lattice counted its own
    its = st["lattice_iters"]
    assert its[4] > its[0]
    assert st["kernel_launches"] > 0


def test_batch_matches_single_lattice_cg(hisq):
    import torch
    mix = SMALL_MIX[:3]
    batch, folded, bs, b = build(hisq, mix, seed0=700)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    batch.cg(x, torch.from_numpy(b).cuda(), [m[1] for m in mix], 1e-10, 5000, inner_prec=1)
    for l, (L, mass, eps) in enumerate(mix):
        fat, lng = hin.gen_links(L, 700 + l, eps, 0.1)
        lat = hisq.Lattice(L, precs=(0, 1)).load(fat, lng)
        xl = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
        lat.cg(xl, torch.from_numpy(bs[l]).reshape(1, -1, 3).cuda(), mass, 1e-10, 5000, inner_prec=1)
        o0, o1 = batch.offsets[l] // 3, batch.offsets[l + 1] // 3
        d = (x[o0:o1] - xl[0]).norm() / xl.norm()
        assert float(d) < 1e-8


def test_batch_host_buffers(hisq):
    mix = SMALL_MIX[:2]
    batch, folded, bs, b = build(hisq, mix, seed0=900)
    x = np.zeros_like(b)
    rc, st = batch.cg(x, b, [m[1] for m in mix], 1e-10, 5000, inner_prec=1)
    for l, (L, mass, eps) in enumerate(mix):
        o0, o1 = batch.offsets[l] // 3, batch.offsets[l + 1] // 3
        assert oracle.true_residual(L, folded[l][0], folded[l][1], mass, bs[l], x[o0:o1]) <= 1e-10


def test_batch_64_uneven_lattices(hisq):
    """The uneven-batch workload: 64 lattices (32 x 16^4, 19 x 24^3x8, 13 x 32^3x8), per-lattice eps and
    mass, FP32/FP64 mixed CG to 1e-10. Sampled lattices are checked with the oracle; all report <= 1e-10."""
    import torch
    mix = hin.lattice_mix_64()
    batch = hisq.Batch([m["dims"] for m in mix])
    bs = []
    for l, m in enumerate(mix):
        fat, lng = hin.gen_links(m["dims"], m["gauge_seed"], m["eps"], 0.1)
        batch.load(l, fat, lng)
        bs.append(hin.gen_source(m["source_seed"], oracle.volume(m["dims"]) // 2, 1)[0])
    b = np.concatenate([v.reshape(-1) for v in bs]).reshape(-1, 3)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    rc, st = batch.cg(x, torch.from_numpy(b).cuda(), [m["mass"] for m in mix], 1e-10, 5000, inner_prec=1)
    assert rc == 0 and st["converged"] == 1
    assert max(st["lattice_residual"]) <= 1e-10
    xs = x.cpu().numpy()
    for l in (0, 31, 32, 50, 51, 63):
        m = mix[l]
        L = m["dims"]
        fat, lng = hin.gen_links(L, m["gauge_seed"], m["eps"], 0.1)
        ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
        o0, o1 = batch.offsets[l] // 3, batch.offsets[l + 1] // 3
        assert oracle.true_residual(L, ff, lf, m["mass"], bs[l], xs[o0:o1]) <= 1e-10


def test_batch_errors(hisq):
    with pytest.raises(hisq.HisqError) as e:
        hisq.hisq_batch_create([(8, 8, 8, 7)])
    assert e.value.code == hisq.HISQ_EINVAL
    batch = hisq.Batch([(4, 6, 8, 10), (8, 8, 8, 8)])
    x = np.zeros((batch.offsets[-1] // 3, 3), np.complex128)
    with pytest.raises(hisq.HisqError) as e:
        batch.cg(x, x.copy(), [0.1, 0.1], 1e-10, 100)  # no links
    assert e.value.code == hisq.HISQ_ENOLINKS
