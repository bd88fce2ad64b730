"""Parity at the Dslash sweep's lattice sizes (32^3x8, 64^3x16, 96^3x24 of the precision workload), in the
launch configuration the sweep times: the library's Dslash in FP64/FP32/FP16/BF16/double-float against the oracle
evaluated one output site at a time on 2048 sampled sites of each parity, and anti-hermiticity of the GPU
operator over the whole lattice (<u, D_eo v> = -<D_oe u, v>), a property that holds at any size. Links are
generated and loaded t-slab by t-slab as in the sweep. 144^3x36 is checked by the sweep itself
(anti-hermiticity), since the oracle's full FP64 link arrays (248 GB) do not fit the host."""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
from test_gpu_dslash import TOL, empty_like_prec, from_device, rel_err, to_device

pytestmark = pytest.mark.gpu

SIZES = [(32, 32, 32, 8), (64, 64, 64, 16), (96, 96, 96, 24)]
PRECS = (0, 1, 2, 3, 4)
NSAMPLE = 2048


@pytest.fixture(scope="module", params=SIZES, ids=lambda L: "x".join(map(str, L)))
def sized(request, hisq):
    L = request.param
    lat = hisq.Lattice(L, precs=PRECS)
    nt = max(1, min(L[3], int(2e8 // (L[0] * L[1] * L[2] * 4 * 9 * 16))))
    fats, lngs = [], []
    for t0 in range(0, L[3], nt):
        n = min(nt, L[3] - t0)
        fat, lng = hin.gen_links(L, 1001, 0.3, 0.1, t0=t0, nt=n)
        hisq.hisq_load_links_slab(lat.ctx, t0, n, fat, lng)
        fats.append(fat)
        lngs.append(lng)
    fat = np.concatenate(fats).reshape(-1, 4, 3, 3)
    lng = np.concatenate(lngs).reshape(-1, 4, 3, 3)
    del fats, lngs
    ff, lf = oracle.fold_links(L, fat, lng)
    del fat, lng
    yield L, lat, ff, lf
    lat.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("parity", [0, 1])
def test_sampled_sites(sized, prec, parity):
    L, lat, ff, lf = sized
    src = hin.gen_source(2001 + parity, lat.half, 1)
    x = to_device(src, prec)
    y = empty_like_prec((1, lat.half, 3), prec)
    lat.dslash(parity, y, x, prec, 1)
    got = from_device(y, prec)[0]
    rng = np.random.default_rng(31 + parity)
    cbs = np.sort(rng.choice(lat.half, NSAMPLE, replace=False))
    ref = oracle.dslash_sites(L, ff, lf, parity, src[0], cbs)
    assert rel_err(got[cbs], ref) <= TOL[prec], (L, prec, parity, rel_err(got[cbs], ref))


@pytest.mark.parametrize("prec", PRECS)
def test_anti_hermiticity(sized, prec):
    import torch
    L, lat, ff, lf = sized
    u = hin.gen_source(11, lat.half, 1)
    v = hin.gen_source(12, lat.half, 1)
    Dv, Du = empty_like_prec((1, lat.half, 3), prec), empty_like_prec((1, lat.half, 3), prec)
    lat.dslash(0, Dv, to_device(v, prec), prec, 1)  # D_eo v
    lat.dslash(1, Du, to_device(u, prec), prec, 1)  # D_oe u
    # inner products of the vectors as the GPU held them (rounded to prec), summed in FP64
    uu = torch.from_numpy(from_device(to_device(u, prec), prec)).cuda().flatten()
    vv = torch.from_numpy(from_device(to_device(v, prec), prec)).cuda().flatten()
    lhs = complex(torch.vdot(uu, torch.from_numpy(from_device(Dv, prec)).cuda().flatten()))
    rhs = -complex(torch.vdot(torch.from_numpy(from_device(Du, prec)).cuda().flatten(), vv))
    # both sides are the same sum up to the rounding of the operator outputs (the rounded links still
    # define an exactly anti-hermitian operator): relative difference within the precision's tolerance
    assert abs(lhs - rhs) <= TOL[prec] * abs(lhs), (L, prec, abs(lhs - rhs) / abs(lhs))
