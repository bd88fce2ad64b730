"""Long-link compression (two stored rows, third reconstructed in the kernel) against the oracle:
Dslash and A in the compressed low precisions at the same tolerances, mixed CG to the same true
residual, and refusal of long links that are not naik * SU(3)."""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
from test_gpu_dslash import TOL, empty_like_prec, from_device, rel_err, to_device

pytestmark = pytest.mark.gpu

NAIK = -1.0 / 24.0


@pytest.fixture(scope="module")
def comp(hisq):
    L = (8, 10, 12, 14)
    fat, lng = hin.gen_links(L, 777, 0.3, 0.1)
    lat = hisq.Lattice(L).compress_long(NAIK).load(fat, lng)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    return L, lat, ff, lf


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 4, 16])
def test_compressed_dslash_parity(comp, prec, parity, nrhs):
    L, lat, ff, lf = comp
    src = hin.gen_source(100 + nrhs, lat.half, nrhs)
    x = to_device(src, prec)
    y = empty_like_prec((nrhs, lat.half, 3), prec)
    lat.dslash(parity, y, x, prec, nrhs)
    got = from_device(y, prec)
    for r in range(nrhs):
        assert rel_err(got[r], oracle.dslash(L, ff, lf, parity, src[r])) <= TOL[prec]


def test_compressed_fp64_untouched(comp):
    L, lat, ff, lf = comp
    src = hin.gen_source(5, lat.half, 1)
    x = to_device(src, 0)
    y = empty_like_prec((1, lat.half, 3), 0)
    lat.dslash(0, y, x, 0, 1)
    assert rel_err(from_device(y, 0)[0], oracle.dslash(L, ff, lf, 0, src[0])) <= 1e-12


@pytest.mark.parametrize("inner", [1, 2])
def test_compressed_mixed_cg(comp, inner):
    import torch
    L, lat, ff, lf = comp
    b = hin.gen_source(7, lat.half, 1)
    x = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
    rc, st = lat.cg(x, torch.from_numpy(b).cuda(), 0.02, 1e-10, 5000, inner_prec=inner)
    assert rc == 0
    assert oracle.true_residual(L, ff, lf, 0.02, b[0], x.cpu().numpy()[0]) <= 1e-10


def test_compression_refuses_non_su3_long_links(hisq):
    L = (4, 6, 8, 10)
    fat, lng = hin.gen_links(L, 3, 0.3, 0.1)
    lat = hisq.Lattice(L, precs=(0, 1)).compress_long(NAIK)
    with pytest.raises(hisq.HisqError) as e:
        lat.load(fat, fat)  # fat links are not naik * SU(3)
    assert e.value.code == hisq.HISQ_EINVAL
    with pytest.raises(hisq.HisqError) as e:
        lat.load(fat, lng * 1.01)  # wrong scale
    assert e.value.code == hisq.HISQ_EINVAL
    lat.load(fat, lng)
    lat.compress_long(0.0)  # off again: links must be reloaded
    x = torch_zeros(lat)
    with pytest.raises(hisq.HisqError) as e:
        lat.dslash(0, x.clone(), x, 0, 1)
    assert e.value.code == hisq.HISQ_ENOLINKS


def torch_zeros(lat):
    import torch
    return torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
