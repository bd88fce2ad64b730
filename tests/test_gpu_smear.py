"""Link smearing on the GPU against the smearing oracle (oracle/smear.py):
- one level with every path kind, and the fat7 level without a Lepage term;
- the U(3) projection;
- the two HISQ levels.
These run on lattices with extents of 4 (where x+2 and x-2 coincide), non-cubic ones, and volumes
that leave a ragged last block. The full 48^3x12 size is checked on sampled sites. Smeared links
loaded into a context drive the Dslash the way the oracle-smeared ones do. Argument errors are
covered too. Tolerance: global relative L2 error 1e-12 for FP64 and for double-float arithmetic."""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
from oracle import smear as sm
from test_gpu_dslash import rel_err

pytestmark = pytest.mark.gpu

# fat7 level and an asqtad-type second level (tree level: the fat-link coefficients sum to 9/8 and
# with the Naik term -1/24 the free dispersion starts at p); other sets are arbitrary test values
FAT7 = dict(c1=1 / 8, c3=1 / 16, c5=1 / 64, c7=1 / 384)
LEVEL2 = dict(c1=5 / 8, c3=1 / 16, c5=1 / 64, c7=1 / 384, cL=-1 / 16, cN=-1 / 24)
RANDOM = dict(c1=0.31, c3=-0.17, c5=0.053, c7=-0.029, cL=0.071, cN=-0.43)
TOL = {0: 1e-12, 4: 1e-12}
LATTICES = [(4, 4, 4, 4), (6, 4, 4, 6), (10, 6, 4, 4), (8, 6, 4, 10)]


def links(L, seed, noise=0.1):
    """Thin SU(3) links plus a little Gaussian noise (general 3x3 matrices), (V, 4, 3, 3)."""
    U = hin.gen_thin(L, seed, 0.3).reshape(-1, 4, 3, 3)
    if noise:
        U = U + noise * hin.gen_links(L, seed + 1, 0.3, 1.0)[0].reshape(-1, 4, 3, 3)
    return np.ascontiguousarray(U)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def empty_links(L):
    import torch
    return torch.empty((int(np.prod(L)), 4, 3, 3), dtype=torch.complex128, device="cuda")


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("prec", [0, 4])
@pytest.mark.parametrize("cname", ["random", "fat7"])
def test_smear_level_matches_oracle(hisq, L, prec, cname):
    import torch
    coeffs = RANDOM if cname == "random" else FAT7
    U = links(L, 300 + sum(L))
    lat = hisq.Lattice(L, precs=(0,))
    fat, lng = empty_links(L), empty_links(L)
    lat.smear(fat, lng, dev(U), coeffs, prec)
    torch.cuda.synchronize()
    F, Lg = sm.smear(L, U, **coeffs)
    assert rel_err(fat.cpu().numpy(), F) <= TOL[prec]
    if coeffs.get("cN", 0.0):
        assert rel_err(lng.cpu().numpy(), Lg) <= TOL[prec]
    else:
        assert float(lng.abs().max()) == 0.0


def test_smear_without_long_output(hisq):
    import torch
    L = (6, 4, 4, 6)
    U = links(L, 41)
    lat = hisq.Lattice(L, precs=(0,))
    fat = empty_links(L)
    lat.smear(fat, None, dev(U), RANDOM)
    torch.cuda.synchronize()
    assert rel_err(fat.cpu().numpy(), sm.smear(L, U, **RANDOM)[0]) <= 1e-12


@pytest.mark.parametrize("inplace", [False, True])
def test_project_u3_matches_oracle(hisq, inplace):
    import torch
    L = (6, 4, 4, 6)
    W = links(L, 51, noise=0.3)
    lat = hisq.Lattice(L, precs=(0,))
    w = dev(W)
    out = w if inplace else empty_links(L)
    hisq.hisq_project_u3(lat.ctx, out, w)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert rel_err(got, sm.project_u3(W)) <= 1e-13
    eye = np.broadcast_to(np.eye(3), got.shape)
    assert np.abs(np.conj(np.swapaxes(got, -1, -2)) @ got - eye).max() <= 1e-13


def test_project_u3_singular_link_is_an_error(hisq):
    L = (4, 4, 4, 4)
    W = links(L, 52, noise=0.3)
    W[7, 2] = 0.0
    lat = hisq.Lattice(L, precs=(0,))
    out = empty_links(L)
    with pytest.raises(hisq.HisqError) as e:
        hisq.hisq_project_u3(lat.ctx, out, dev(W))
    assert e.value.code == hisq.HISQ_EINVAL
    got = out.cpu().numpy()
    assert np.array_equal(got[7, 2], W[7, 2])
    ok = np.ones(got.shape[:2], bool)
    ok[7, 2] = False
    assert rel_err(got[ok], sm.project_u3(W[ok])) <= 1e-13


@pytest.mark.parametrize("L", LATTICES[:3])
@pytest.mark.parametrize("prec", [0, 4])
def test_hisq_two_levels_match_oracle(hisq, L, prec):
    import torch
    U = links(L, 600 + sum(L), noise=0.0)
    lat = hisq.Lattice(L, precs=(0,))
    fat, lng = empty_links(L), empty_links(L)
    lat.hisq_links(fat, lng, dev(U), FAT7, LEVEL2, prec)
    torch.cuda.synchronize()
    F, Lg = sm.hisq_links(L, U, FAT7, LEVEL2)
    assert rel_err(fat.cpu().numpy(), F) <= TOL[prec]
    assert rel_err(lng.cpu().numpy(), Lg) <= TOL[prec]


def test_smeared_links_drive_the_dslash(hisq):
    """Links smeared on the device and loaded from device memory give the oracle's Dslash of the
    oracle-smeared links."""
    import torch
    L = (6, 4, 4, 6)
    U = links(L, 71, noise=0.0)
    lat = hisq.Lattice(L, precs=(0, 1))
    fat, lng = empty_links(L), empty_links(L)
    lat.hisq_links(fat, lng, dev(U), FAT7, LEVEL2)
    lat.load(fat, lng)
    F, Lg = sm.hisq_links(L, U, FAT7, LEVEL2)
    ff, lf = oracle.fold_links(L, F, Lg)
    src = hin.gen_source(72, lat.half, 1)
    y = torch.empty((1, lat.half, 3), dtype=torch.complex128, device="cuda")
    lat.dslash(0, y, dev(src), 0)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy()[0], oracle.dslash(L, ff, lf, 0, src[0])) <= 1e-12


def neighbourhood(L, sites, r=2):
    """Lexicographic indices of every site within offsets [-r, r] of the given sites in each direction:
    the level-2 paths and the Naik product from a site only use links that start there."""
    c = np.array(oracle.coords(L, np.asarray(sites))).T
    offs = np.array(np.meshgrid(*[np.arange(-r, r + 1)] * 4, indexing="ij")).reshape(4, -1).T
    pts = (c[:, None, :] + offs[None, :, :]) % np.array(L)
    idx = pts[..., 0] + L[0] * (pts[..., 1] + L[1] * (pts[..., 2] + L[2] * pts[..., 3]))
    return np.unique(idx.ravel())


@pytest.mark.parametrize("prec", [0, 4])
def test_full_size_sampled_sites(hisq, prec):
    """The two levels at 48^3x12 (the benchmark's size and launch shape), checked on 24 sampled sites
    (including the first and the last site, whose paths wrap around every boundary). The oracle's
    level-1 links are formed on the sites the sampled level-2 paths reach, then projected."""
    import torch
    L = (48, 48, 48, 12)
    V = int(np.prod(L))
    U = hin.gen_thin(L, 1001, 0.3).reshape(V, 4, 3, 3)
    lat = hisq.Lattice(L, precs=(0,))
    fat, lng = empty_links(L), empty_links(L)
    lat.hisq_links(fat, lng, dev(U), FAT7, LEVEL2, prec)
    torch.cuda.synchronize()
    rng = np.random.default_rng(23)
    samples = np.concatenate([[0, V - 1], rng.choice(V, 22, replace=False)])
    nb = neighbourhood(L, samples)
    F1, _ = sm.smear(L, U, **FAT7, sites=nb)
    W = np.zeros_like(U)
    W[nb] = sm.project_u3(F1)
    F, Lg = sm.smear(L, W, **LEVEL2, sites=samples)
    idx = torch.from_numpy(samples).cuda()
    assert rel_err(fat[idx].cpu().numpy(), F) <= TOL[prec]
    assert rel_err(lng[idx].cpu().numpy(), Lg) <= TOL[prec]


def test_argument_errors(hisq):
    L = (4, 4, 4, 4)
    U = links(L, 81)
    lat = hisq.Lattice(L, precs=(0,))
    u, fat, lng = dev(U), empty_links(L), empty_links(L)
    cases = [
        (lambda: lat.smear(fat, lng, U, RANDOM), "host input"),
        (lambda: lat.smear(fat, lng, u, RANDOM, 1), "FP32 arithmetic"),
        (lambda: lat.smear(u, lng, u, RANDOM), "output over the input"),
        (lambda: lat.smear(fat, fat, u, RANDOM), "fat and long outputs the same"),
        (lambda: lat.smear(fat, lng, u, dict(RANDOM, c5=float("nan"))), "NaN coefficient"),
        (lambda: hisq.hisq_project_u3(lat.ctx, u[1:], u), "output partly over the input"),
    ]
    for f, what in cases:
        with pytest.raises(hisq.HisqError) as e:
            f()
        assert e.value.code == hisq.HISQ_EINVAL, what


@pytest.mark.parametrize("prec", [0, 4])
def test_every_launch_form_matches_oracle(hisq, prec):
    """Each pass kernel in both register budgets (form 0: as many registers as the code wants, form 1: 128)
    and at several block sizes, forced through loaded tune entries, and the untuned fallback with the
    autotuner off, against the oracle."""
    import torch
    L = (6, 4, 4, 6)
    U = links(L, 91)
    F, Lg = sm.smear(L, U, **RANDOM)
    u = dev(U)
    dims = "%dx%dx%dx%d" % L
    name = "df64" if prec == 4 else "f64"
    for vi in (0, 1):
        for block in (64, 96, 256):
            lat = hisq.Lattice(L, precs=(0,))
            rep = "".join("smear/%s/%s %s -> %d\n" % (k, name, dims, vi * 10000 + block)
                          for k in ("staples", "middle", "fat"))
            assert hisq.hisq_tune_load(lat.ctx, rep) == 3
            fat, lng = empty_links(L), empty_links(L)
            lat.smear(fat, lng, u, RANDOM, prec)
            torch.cuda.synchronize()
            assert rel_err(fat.cpu().numpy(), F) <= TOL[prec], (vi, block)
            assert rel_err(lng.cpu().numpy(), Lg) <= TOL[prec], (vi, block)
            assert hisq.hisq_tune_report(lat.ctx).count("-> %d" % (vi * 10000 + block)) == 3
    lat = hisq.Lattice(L, precs=(0,))
    hisq.hisq_set_autotune(lat.ctx, False)
    fat, lng = empty_links(L), empty_links(L)
    lat.smear(fat, lng, u, RANDOM, prec)
    torch.cuda.synchronize()
    assert rel_err(fat.cpu().numpy(), F) <= TOL[prec]
