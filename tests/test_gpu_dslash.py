"""GPU Dslash and A = 4m^2 - D_eo D_oe against the FP64 oracle, element by element, through the C ABI.

Tolerance (relative global L2 over the whole output): FP64 1e-12, FP32 2e-6, FP16/BF16 5e-3; the
double-float precision (prec 4: FP64 vectors, links as FP32 pairs, 2^-47 rounding per operation) is held
to the FP64 tolerance.
Lattices: 8^4 (the plain-method workload), 8x10x12x14 (every hop distinct, ragged last block),
4x6x8x10 (hops alias and must accumulate), 16^3x8 (several tiles), 4^4 (the smallest lattice: the +3 and -1
hops coincide in every direction).
"""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-6, 2: 5e-3, 3: 5e-3, 4: 1e-12}
F64_LAYOUT = (0, 4)  # precisions whose boundary vectors are complex128
LATTICES = [(8, 8, 8, 8), (8, 10, 12, 14), (4, 6, 8, 10), (16, 16, 16, 8), (4, 4, 4, 4)]


def to_device(vec, prec):
    """complex128 numpy (nrhs, half, 3) -> torch tensor in the boundary layout of prec."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(vec))
    if prec in F64_LAYOUT:
        return t.cuda()
    if prec == 1:
        return t.to(torch.complex64).cuda()
    real = torch.view_as_real(t.to(torch.complex64))
    return real.to(torch.float16 if prec == 2 else torch.bfloat16).contiguous().cuda()


def from_device(t, prec):
    import torch
    t = t.cpu()
    if prec in (2, 3):
        t = torch.view_as_complex(t.float().contiguous())
    return t.to(torch.complex128).numpy()


def empty_like_prec(shape, prec):
    import torch
    if prec in F64_LAYOUT:
        return torch.empty(shape, dtype=torch.complex128, device="cuda")
    if prec == 1:
        return torch.empty(shape, dtype=torch.complex64, device="cuda")
    return torch.empty(shape + (2,), dtype=torch.float16 if prec == 2 else torch.bfloat16, device="cuda")


def rel_err(got, ref):
    return float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))


_cache = {}


def setup(hisq, L, seed=1000):
    key = (L, seed)
    if key not in _cache:
        fat, lng = hin.gen_links(L, seed, 0.3, 0.1)
        lat = hisq.Lattice(L, precs=(0, 1, 2, 3, 4)).load(fat, lng)
        ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
        _cache[key] = (lat, ff, lf)
    return _cache[key]


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("parity", [0, 1])
def test_dslash_parity(hisq, L, prec, parity):
    lat, ff, lf = setup(hisq, L)
    half = lat.half
    src = hin.gen_source(2000 + parity, half, 1)
    x = to_device(src, prec)
    y = empty_like_prec((1, half, 3), prec)
    lat.dslash(parity, y, x, prec, 1)
    got = from_device(y, prec)[0]
    ref = oracle.dslash(L, ff, lf, parity, src[0])
    assert rel_err(got, ref) <= TOL[prec], (L, prec, parity, rel_err(got, ref))


@pytest.mark.parametrize("nrhs", [2, 3, 4, 8, 16, 21])
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_dslash_multi_rhs(hisq, nrhs, prec):
    L = (8, 10, 12, 14)
    lat, ff, lf = setup(hisq, L)
    half = lat.half
    src = hin.gen_source(3000 + nrhs, half, nrhs)
    x = to_device(src, prec)
    y = empty_like_prec((nrhs, half, 3), prec)
    lat.dslash(0, y, x, prec, nrhs)
    got = from_device(y, prec)
    for r in range(nrhs):
        ref = oracle.dslash(L, ff, lf, 0, src[r])
        assert rel_err(got[r], ref) <= TOL[prec], (nrhs, prec, r)


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_apply_A_parity(hisq, prec):
    L = (8, 10, 12, 14)
    lat, ff, lf = setup(hisq, L)
    half = lat.half
    src = hin.gen_source(4000, half, 2)
    x = to_device(src, prec)
    y = empty_like_prec((2, half, 3), prec)
    mass, sigma = 0.05, 0.3
    lat.apply_A(y, x, mass, prec, 2, sigma=sigma)
    got = from_device(y, prec)
    for r in range(2):
        ref = oracle.apply_A(L, ff, lf, mass, src[r], sigma=sigma)
        # two Dslash applications: allow twice the single-operator tolerance
        assert rel_err(got[r], ref) <= 2 * TOL[prec]


def test_host_pointers(hisq):
    """Host numpy buffers are staged by the library (the end-to-end path)."""
    L = (4, 6, 8, 10)
    lat, ff, lf = setup(hisq, L)
    src = hin.gen_source(5, lat.half, 1)
    out = np.empty_like(src)
    lat.dslash(1, out, src, 0, 1)
    assert rel_err(out[0], oracle.dslash(L, ff, lf, 1, src[0])) <= 1e-12


def test_deterministic(hisq):
    import torch
    L = (16, 16, 16, 8)
    lat, ff, lf = setup(hisq, L)
    x = to_device(hin.gen_source(6, lat.half, 1), 1)
    y1 = empty_like_prec((1, lat.half, 3), 1)
    y2 = empty_like_prec((1, lat.half, 3), 1)
    lat.dslash(0, y1, x, 1, 1)
    lat.dslash(0, y2, x, 1, 1)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_programmatic_launch_changes_no_result(hisq, prec):
    """A chain of dependent Dslash launches (each reads the previous one's output) gives bitwise the same
    vectors with programmatic dependent launch as with plain stream-ordered launches, and the chain's end
    agrees with the oracle's D_eo D_oe D_eo D_oe x."""
    import torch
    L = (16, 16, 16, 8)
    lat, ff, lf = setup(hisq, L)
    src = hin.gen_source(7, lat.half, 1)
    x = to_device(src, prec)
    outs = {}
    for pdl in (1, 0, 1):
        hisq.hisq_set_pdl(lat.ctx, pdl)
        w = [x] + [empty_like_prec((1, lat.half, 3), prec) for _ in range(4)]
        for k in range(4):
            lat.dslash(1 - k % 2, w[k + 1], w[k], prec, 1)  # D_oe, D_eo, D_oe, D_eo
        torch.cuda.synchronize()
        outs.setdefault(pdl, []).append([t.clone() for t in w[1:]])
    hisq.hisq_set_pdl(lat.ctx, 1)
    for a, b in zip(outs[1][0], outs[0][0]):
        assert torch.equal(a, b)
    for a, b in zip(outs[1][0], outs[1][1]):
        assert torch.equal(a, b)
    ref = src[0]
    for k in range(4):
        ref = oracle.dslash(L, ff, lf, 1 - k % 2, ref)
    assert rel_err(from_device(outs[1][0][3], prec)[0], ref) <= 4 * TOL[prec]


def test_programmatic_launch_solve_bitwise(hisq):
    """The mixed CG returns the same bits with programmatic dependent launch on and off (its eager launches
    follow the switch; its captured graphs keep plain launches)."""
    import torch
    L = (8, 8, 8, 8)
    lat, ff, lf = setup(hisq, L)
    b = torch.from_numpy(hin.gen_source(2000, lat.half, 1)).cuda()
    xs, its = [], []
    for pdl in (1, 0, 1):
        hisq.hisq_set_pdl(lat.ctx, pdl)
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        rc, st = lat.cg(x, b, 0.1, 1e-10, 2000, inner_prec=1, reliable_period=50)
        torch.cuda.synchronize()
        xs.append(x.clone())
        its.append(st["iters"])
    hisq.hisq_set_pdl(lat.ctx, 1)
    assert its[0] == its[1] == its[2]
    assert torch.equal(xs[0], xs[1]) and torch.equal(xs[0], xs[2])


def test_free_field_eigenvector(hisq):
    """Unit links: a plane wave on even sites is an eigenvector of the GPU A with the closed-form eigenvalue."""
    import torch
    L = (8, 10, 12, 14)
    V = oracle.volume(L)
    fat = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    lat = hisq.Lattice(L, precs=(0, 1)).load(fat, -fat / 24)
    ev = oracle.parity_sites(L, 0)
    x, y, z, t = oracle.coords(L, ev)
    p = [2 * np.pi * 1 / L[0], 2 * np.pi * 3 / L[1], 2 * np.pi * 2 / L[2], 2 * np.pi * (4 + 0.5) / L[3]]
    v = np.zeros((1, len(ev), 3), np.complex128)
    v[0, :, 2] = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    mass = 0.1
    lam = 4 * mass ** 2 + 4 * sum((np.sin(q) - np.sin(3 * q) / 24) ** 2 for q in p)
    out = torch.empty((1, len(ev), 3), dtype=torch.complex128, device="cuda")
    lat.apply_A(out, torch.from_numpy(v).cuda(), mass, 0)
    assert np.abs(out.cpu().numpy() - lam * v).max() < 1e-12


def test_errors(hisq):
    import torch
    L = (4, 6, 8, 10)
    with pytest.raises(hisq.HisqError) as e:
        hisq.hisq_create((4, 6, 8, 9))
    assert e.value.code == hisq.HISQ_EINVAL
    lat = hisq.Lattice(L, precs=(0, 1))
    x = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(hisq.HisqError) as e:
        lat.dslash(0, y, x, 0, 1)
    assert e.value.code == hisq.HISQ_ENOLINKS
    fat, lng = hin.gen_links(L, 1)
    bad = fat.copy()
    bad[1, 2, 3, 1, 2, 0, 1] = np.nan
    with pytest.raises(hisq.HisqError) as e:
        lat.load(bad, lng)
    assert e.value.code == hisq.HISQ_ENONFINITE
    lat.load(fat, lng)
    with pytest.raises(hisq.HisqError) as e:
        lat.dslash(2, y, x, 0, 1)
    assert e.value.code == hisq.HISQ_EINVAL
    with pytest.raises(hisq.HisqError) as e:
        lat.dslash(0, y, x, 2, 1)  # FP16 not resident in this context
    assert e.value.code == hisq.HISQ_EINVAL
    with pytest.raises(hisq.HisqError) as e:
        lat.dslash(0, x, x, 0, 1)  # aliased
    assert e.value.code == hisq.HISQ_EINVAL


def test_double_float_close_to_fp64(hisq):
    """The double-float operator agrees with the FP64 one far inside the FP64 tolerance, on sources spanning
    twelve decades (and exact zeros), whose conversion to double-float is done with integer operations."""
    import torch
    L = (8, 10, 12, 14)
    lat, ff, lf = setup(hisq, L)
    src = hin.gen_source(9100, lat.half, 1)
    rng = np.random.default_rng(5)
    src = src * 10.0 ** rng.uniform(-6, 6, size=src.shape)
    src[0, ::7, 1] = 0.0
    x = torch.from_numpy(src).cuda()
    y64, ydf = torch.empty_like(x), torch.empty_like(x)
    lat.dslash(0, y64, x, 0)
    lat.dslash(0, ydf, x, 4)
    ref = oracle.dslash(L, ff, lf, 0, src[0])
    assert rel_err(ydf.cpu().numpy()[0], ref) <= 1e-13
    assert rel_err(ydf.cpu().numpy()[0], y64.cpu().numpy()[0]) <= 1e-13


def test_slab_loading_matches_whole(hisq):
    import torch
    L = (8, 10, 12, 14)
    fat, lng = hin.gen_links(L, 77)
    whole = hisq.Lattice(L, precs=(0,)).load(fat, lng)
    slab = hisq.Lattice(L, precs=(0,))
    for t0, nt in [(0, 5), (5, 4), (9, 5)]:
        hisq.hisq_load_links_slab(slab.ctx, t0, nt, fat[t0:t0 + nt], lng[t0:t0 + nt])
    x = torch.from_numpy(hin.gen_source(8, whole.half, 1)).cuda()
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    whole.dslash(0, y1, x, 0)
    slab.dslash(0, y2, x, 0)
    assert torch.equal(y1, y2)


# launch forms per rhs group (vectors per thread x threads per site), in the tuner's variant order;
# 8-vector groups exist below FP64 only. Groups of 1 and 8 have each form twice: sites in cb order, and
# sites in the tiled walk (tiles of z-planes walked along t; on this lattice two tiles of 6 planes); the
# 8-vector group's last two forms prefetch each next hop's vectors and link (cb order, tiled walk).
FORMS = {1: 2, 2: 2, 4: 3, 8: 8}


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_every_launch_form_matches_oracle(hisq, prec):
    """Each launch form the tuner can pick, forced through a loaded tune entry, against the oracle: the
    Dslash (plain epilogue) and A (fused axpy epilogue) for groups of 1, 2, 4 and 8 vectors."""
    L = (8, 10, 12, 14)
    lat, ff, lf = setup(hisq, L)
    half = lat.half
    sp = 0 if prec == 4 else prec  # the double-float operator takes FP64 vectors
    dims = "%dx%dx%dx%d" % L
    for nr, nforms in FORMS.items():
        if nr == 8 and prec in (0, 4):
            continue
        src = hin.gen_source(7000 + nr, half, nr)
        x = to_device(src, prec)
        for vi in range(nforms):
            for epi in (0, 1):
                key = "dslash/l%d/s%d/nr%d/e%d/c0" % (prec, sp, nr, epi)
                assert hisq.hisq_tune_load(lat.ctx, "%s %s -> %d\n" % (key, dims, vi * 10000 + 96)) == 1
            y = empty_like_prec((nr, half, 3), prec)
            lat.dslash(0, y, x, prec, nr)
            got = from_device(y, prec)
            for r in range(nr):
                assert rel_err(got[r], oracle.dslash(L, ff, lf, 0, src[r])) <= TOL[prec], (prec, nr, vi, r)
            lat.apply_A(y, x, 0.05, prec, nr)
            got = from_device(y, prec)
            for r in range(nr):
                ref = oracle.apply_A(L, ff, lf, 0.05, src[r])
                assert rel_err(got[r], ref) <= 2 * TOL[prec], (prec, nr, vi, r)
