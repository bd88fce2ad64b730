"""Parity at the benchmark's full size (48^3x12, links 0.76 GB in FP32 -- far larger than L2), in the launch
configuration bench.py times: the library's Dslash in FP64/FP32/FP16/BF16/double-float, with and without compressed long links,
against the oracle evaluated one output site at a time on 4096 sampled sites; and the mixed-precision solve
of the benchmark step judged by the oracle's true residual over the whole lattice. Anti-hermiticity of the
GPU operator, a property that holds at any size, is checked on the whole lattice too."""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
from test_gpu_dslash import TOL, empty_like_prec, from_device, rel_err, to_device

pytestmark = pytest.mark.gpu

L = (48, 48, 48, 12)
NSAMPLE = 4096


@pytest.fixture(scope="module")
def full(hisq):
    fat, lng = hin.gen_links(L, 1001, 0.3, 0.1)  # the benchmark's gauge field
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    lat = hisq.Lattice(L, precs=(0, 1, 2, 3, 4)).load(fat, lng)
    comp = hisq.Lattice(L, precs=(0, 1, 2, 3)).compress_long(-1.0 / 24.0).load(fat, lng)
    return lat, comp, ff, lf


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("compressed", [False, True])
def test_sampled_sites_full_size(full, prec, compressed):
    lat, comp, ff, lf = full
    if compressed and prec in (0, 4):
        pytest.skip("FP64 and double-float are never compressed")
    use = comp if compressed else lat
    src = hin.gen_source(2001, lat.half, 1)
    x = to_device(src, prec)
    y = empty_like_prec((1, lat.half, 3), prec)
    use.dslash(0, y, x, prec, 1)
    got = from_device(y, prec)[0]
    rng = np.random.default_rng(17)
    cbs = np.sort(rng.choice(lat.half, NSAMPLE, replace=False))
    ref = oracle.dslash_sites(L, ff, lf, 0, src[0], cbs)
    assert rel_err(got[cbs], ref) <= TOL[prec], rel_err(got[cbs], ref)


def test_anti_hermiticity_full_size(full):
    import torch
    lat, comp, ff, lf = full
    u = torch.from_numpy(hin.gen_source(11, lat.half, 1)).cuda()
    v = torch.from_numpy(hin.gen_source(12, lat.half, 1)).cuda()
    Dv, Du = torch.empty_like(v), torch.empty_like(u)
    lat.dslash(0, Dv, v, 0, 1)  # D_eo v
    lat.dslash(1, Du, u, 0, 1)  # D_oe u
    lhs = torch.vdot(u.flatten(), Dv.flatten())
    rhs = -torch.vdot(Du.flatten(), v.flatten())
    assert abs(complex(lhs - rhs)) <= 1e-12 * abs(complex(lhs))


def test_benchmark_solve_true_residual(full):
    import torch
    lat, comp, ff, lf = full
    b = hin.gen_source(2001, lat.half, 1)
    for use, inner in ((lat, 1), (comp, 2)):
        x = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
        rc, st = use.cg(x, torch.from_numpy(b).cuda(), 0.01, 1e-10, 20000, inner_prec=inner)
        assert rc == 0
        r = oracle.true_residual(L, ff, lf, 0.01, b[0], x.cpu().numpy()[0])
        assert r <= 1e-10
        assert abs(r - st["true_rel_residual"]) < 1e-11
