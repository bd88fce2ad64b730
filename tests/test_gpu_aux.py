"""Auxiliary subsystems on the GPU: the failure path of the bounded device waits (made to run out on
purpose, without a fault or a hang) and the persistence of the autotuner's cache."""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
from test_gpu_dslash import rel_err

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives(hisq):
    import torch
    L = (8, 10, 12, 14)
    fat, lng = hin.gen_links(L, 77, 0.3, 0.1)
    lat = hisq.Lattice(L, precs=(0, 1)).load(fat, lng)
    assert hisq.hisq_selftest_bounded_wait(lat.ctx) == hisq.HISQ_ETIMEOUT
    assert "gave up" in hisq.hisq_last_error()
    # the context is still usable afterwards
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    src = hin.gen_source(5, lat.half, 1)
    y = torch.empty((1, lat.half, 3), dtype=torch.complex128, device="cuda")
    lat.dslash(0, y, torch.from_numpy(src).cuda(), 0)
    assert rel_err(y.cpu().numpy()[0], oracle.dslash(L, ff, lf, 0, src[0])) <= 1e-12


def test_tune_cache_report_and_load(hisq):
    import torch
    L = (8, 10, 12, 14)
    fat, lng = hin.gen_links(L, 78, 0.3, 0.1)
    a = hisq.Lattice(L, precs=(0, 1)).load(fat, lng)
    x = torch.from_numpy(hin.gen_source(6, a.half, 4)).to(torch.complex64).cuda()
    y = torch.empty_like(x)
    for n in (1, 4):
        a.dslash(0, y, x, 1, n)
    report = hisq.hisq_tune_report(a.ctx)
    assert len(report.splitlines()) >= 2
    # a second context of the same lattice takes the whole cache and reports it back unchanged
    b = hisq.Lattice(L, precs=(0, 1)).load(fat, lng)
    assert hisq.hisq_tune_load(b.ctx, report) == len(report.splitlines())
    assert hisq.hisq_tune_report(b.ctx) == report
    y2 = torch.empty_like(x)
    a.dslash(0, y, x, 1, 4)
    b.dslash(0, y2, x, 1, 4)  # uses the loaded launch form and block size: same result, bit for bit
    torch.cuda.synchronize()
    assert torch.equal(y, y2)
    # lines for other lattice dims are skipped; a malformed line is an error
    c = hisq.Lattice((4, 6, 8, 10), precs=(0, 1))
    assert hisq.hisq_tune_load(c.ctx, report) == 0
    with pytest.raises(hisq.HisqError) as e:
        hisq.hisq_tune_load(c.ctx, "not a tune line\n")
    assert e.value.code == hisq.HISQ_EINVAL
    # a loaded choice naming a launch form that does not exist is dropped and the kernel tuned again
    d = hisq.Lattice(L, precs=(0, 1)).load(fat, lng)
    key = [ln for ln in report.splitlines() if "/nr1/e0/" in ln and "/l1/" in ln][0].split()[0]
    assert hisq.hisq_tune_load(d.ctx, "%s %dx%dx%dx%d -> 90128\n" % ((key,) + L)) == 1
    y3 = torch.empty_like(x)
    d.dslash(0, y3, x, 1, 1)
    torch.cuda.synchronize()
    assert "-> 90128" not in hisq.hisq_tune_report(d.ctx)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    ref = oracle.dslash(L, ff, lf, 0, x.cpu().numpy().astype(np.complex128)[0])
    assert rel_err(y3.cpu().numpy()[0].astype(np.complex128), ref) <= 2e-6


def test_release_workspaces(hisq):
    """Freeing the workspaces returns their memory to the device; smearing and a graph-captured solve
    then allocate and capture again and still match the oracle."""
    import torch
    from oracle import smear as sm
    L = (16, 16, 16, 16)
    V = int(np.prod(L))
    U = hin.gen_thin(L, 90, 0.3).reshape(V, 4, 3, 3)
    fat, lng = hin.gen_links(L, 91, 0.3, 0.1)
    lat = hisq.Lattice(L, precs=(0, 1)).load(fat, lng)
    u = torch.from_numpy(U).cuda()
    f, l = torch.empty_like(u), torch.empty_like(u)
    coeffs = dict(c1=0.3, c3=0.1, c5=0.02, c7=0.004, cL=-0.05, cN=-0.2)
    lat.smear(f, l, u, coeffs)
    b = torch.from_numpy(hin.gen_source(92, lat.half, 1)).cuda()
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    lat.cg(x, b, 0.05, 1e-10, 2000, inner_prec=1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    hisq.hisq_release_workspaces(lat.ctx)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 - free0 >= 144 * 16 * V  # at least the smearing scratch
    f.zero_()
    lat.smear(f, l, u, coeffs)
    torch.cuda.synchronize()
    sample = np.arange(0, V, 97)
    F, _ = sm.smear(L, U, **coeffs, sites=sample)
    assert rel_err(f.cpu().numpy()[sample], F) <= 1e-12
    x.zero_()
    rc, st = lat.cg(x, b, 0.05, 1e-10, 2000, inner_prec=1)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    assert oracle.true_residual(L, ff, lf, 0.05, b.cpu().numpy()[0], x.cpu().numpy()[0]) <= 1.1e-10
    with pytest.raises(hisq.HisqError):
        hisq.hisq_release_workspaces(None)
