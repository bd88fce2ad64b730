"""The multi-RHS Dslash and A on the rhs-interleaved layout [cb][color][rhs] against the FP64 oracle,
element by element, through the C ABI.

The oracle applies the operator to one vector at a time; the interleaved layout is only a different
placement of the same numbers, so every vector of the GPU output must match the oracle's at the operator
tolerances (FP64 and double-float 1e-12, FP32 2e-6, FP16/BF16 5e-3; A, two Dslash applications, twice
those). Lattices: 8x10x12x14 (every hop distinct, ragged last block), 4x6x8x10 (hops alias and must
accumulate), 16^3x8 (several waves of blocks). Every launch form the tuner can pick is forced once.
"""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
from test_gpu_dslash import TOL, from_device, rel_err, setup, to_device

pytestmark = pytest.mark.gpu

# (precision, vectors per site): N a multiple of the granule (FP32 2, 16-bit 4), tails of the thread
# groups (N = 14 FP32: 7 granules), one thread per site (N = 64 FP32: 32 granules)
CASES = [(0, 1), (0, 3), (4, 2), (1, 2), (1, 8), (1, 14), (1, 16), (1, 64), (2, 4), (2, 8), (2, 16), (3, 8),
         (3, 12)]
LATS = [(8, 10, 12, 14), (4, 6, 8, 10), (16, 16, 16, 8)]


def interleave(vec):
    """(nrhs, half, 3) -> (half, 3, nrhs): the rhs-interleaved placement of the same vectors."""
    return np.ascontiguousarray(np.transpose(vec, (1, 2, 0)))


def deinterleave(vec):
    """(half, 3, nrhs) -> (nrhs, half, 3)."""
    return np.ascontiguousarray(np.transpose(vec, (2, 0, 1)))


def empty_interleaved(half, nrhs, prec):
    import torch
    if prec in (0, 4):
        return torch.full((half, 3, nrhs), float("nan"), dtype=torch.complex128, device="cuda")
    if prec == 1:
        return torch.full((half, 3, nrhs), float("nan"), dtype=torch.complex64, device="cuda")
    return torch.full((half, 3, nrhs, 2), float("nan"), dtype=torch.float16 if prec == 2 else torch.bfloat16,
                      device="cuda")


@pytest.mark.parametrize("L", LATS)
@pytest.mark.parametrize("prec,nrhs", CASES)
@pytest.mark.parametrize("parity", [0, 1])
def test_interleaved_dslash_matches_oracle(hisq, L, prec, nrhs, parity):
    lat, ff, lf = setup(hisq, L)
    src = hin.gen_source(700 + nrhs, lat.half, nrhs)
    x = to_device(interleave(src), prec)
    y = empty_interleaved(lat.half, nrhs, prec)
    lat.dslash_interleaved(parity, y, x, prec, nrhs)
    got = deinterleave(from_device(y, prec))
    for r in range(nrhs):
        ref = oracle.dslash(L, ff, lf, parity, src[r])
        assert rel_err(got[r], ref) <= TOL[prec], (L, prec, nrhs, parity, r, rel_err(got[r], ref))


@pytest.mark.parametrize("prec,nrhs", [(0, 3), (4, 2), (1, 2), (1, 14), (1, 16), (2, 8), (3, 12)])
def test_interleaved_apply_A_matches_oracle(hisq, prec, nrhs):
    L = (8, 10, 12, 14)
    lat, ff, lf = setup(hisq, L)
    src = hin.gen_source(800 + nrhs, lat.half, nrhs)
    x = to_device(interleave(src), prec)
    y = empty_interleaved(lat.half, nrhs, prec)
    mass, sigma = 0.05, 0.3
    lat.apply_A_interleaved(y, x, mass, prec, nrhs, sigma=sigma)
    got = deinterleave(from_device(y, prec))
    for r in range(nrhs):
        ref = oracle.apply_A(L, ff, lf, mass, src[r], sigma=sigma)
        assert rel_err(got[r], ref) <= 2 * TOL[prec], (prec, nrhs, r, rel_err(got[r], ref))


def _forms(prec, nrhs):
    """Number of launch forms for (prec, N): granules per thread 1, 2 and (FP32 vectors) 4, where they fit."""
    g = {0: 1, 4: 1, 1: 2, 2: 4, 3: 4}[prec]
    ngr = nrhs // g

    def ts(ng):
        t = 1
        while t < (ngr + ng - 1) // ng:
            t *= 2
        return t
    n = int(ts(1) <= 32) + int(ngr >= 2 and ts(2) <= 32)
    if prec == 1 and ngr >= 4:
        n += 1
    return n


@pytest.mark.parametrize("prec,nrhs", [(0, 3), (1, 14), (1, 16), (2, 16), (3, 8)])
@pytest.mark.parametrize("block", [64, 224])
def test_every_interleaved_launch_form(hisq, prec, nrhs, block):
    """Each form the tuner can choose, forced through a loaded tune entry, in both epilogues."""
    L = (8, 10, 12, 14)
    fat, lng = hin.gen_links(L, 1000, 0.3, 0.1)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    src = hin.gen_source(900 + nrhs, L[0] * L[1] * L[2] * L[3] // 2, nrhs)
    dims = "x".join(map(str, L))
    for form in range(_forms(prec, nrhs)):
        lat = hisq.Lattice(L, precs=(0, prec)).load(fat, lng)
        sp = prec
        for epi in (0, 1):
            hisq.hisq_tune_load(lat.ctx, "mrhs/l%d/s%d/n%d/e%d/c0 %s -> %d\n" % (prec, sp, nrhs, epi, dims,
                                                                               form * 10000 + block))
        x = to_device(interleave(src), prec)
        y = empty_interleaved(lat.half, nrhs, prec)
        lat.dslash_interleaved(1, y, x, prec, nrhs)
        got = deinterleave(from_device(y, prec))
        z = empty_interleaved(lat.half, nrhs, prec)
        lat.apply_A_interleaved(z, x, 0.1, prec, nrhs)
        gotA = deinterleave(from_device(z, prec))
        for r in range(nrhs):
            assert rel_err(got[r], oracle.dslash(L, ff, lf, 1, src[r])) <= TOL[prec], (form, r)
            assert rel_err(gotA[r], oracle.apply_A(L, ff, lf, 0.1, src[r])) <= 2 * TOL[prec], (form, r)
        report = hisq.hisq_tune_report(lat.ctx)
        assert "mrhs/l%d/s%d/n%d/e0/c0 %s -> %d" % (prec, sp, nrhs, dims, form * 10000 + block) in report
        lat.close()


@pytest.mark.parametrize("prec,nrhs", [(1, 8), (2, 8), (3, 4)])
def test_interleaved_compressed_long_links(hisq, prec, nrhs):
    L = (8, 10, 12, 14)
    fat, lng = hin.gen_links(L, 1000, 0.3, 0.1)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    lat = hisq.Lattice(L, precs=(0, 1, 2, 3)).compress_long(-1.0 / 24.0).load(fat, lng)
    src = hin.gen_source(950, lat.half, nrhs)
    for parity in (0, 1):
        y = empty_interleaved(lat.half, nrhs, prec)
        lat.dslash_interleaved(parity, y, to_device(interleave(src), prec), prec, nrhs)
        got = deinterleave(from_device(y, prec))
        for r in range(nrhs):
            assert rel_err(got[r], oracle.dslash(L, ff, lf, parity, src[r])) <= TOL[prec]
    lat.close()


def test_interleaved_rejects_partial_granules(hisq):
    L = (4, 6, 8, 10)
    lat, ff, lf = setup(hisq, L)
    for prec, nrhs in ((1, 3), (2, 6), (3, 2)):
        x = to_device(interleave(hin.gen_source(1, lat.half, nrhs)), prec)
        y = empty_interleaved(lat.half, nrhs, prec)
        with pytest.raises(hisq.HisqError) as e:
            lat.dslash_interleaved(0, y, x, prec, nrhs)
        assert e.value.code == hisq.HISQ_EINVAL and "multiple" in str(e.value)


@pytest.mark.parametrize("L", LATS)
@pytest.mark.parametrize("prec,nrhs", [(2, 16), (2, 64), (3, 32), (3, 64), (2, 44)])
@pytest.mark.parametrize("parity", [0, 1])
def test_tensor_core_interleaved_dslash_matches_oracle(hisq, L, prec, nrhs, parity):
    """The tcgen05 form (16-bit storage, 16-64 vectors), forced through a loaded tune entry: every vector
    against the oracle at the 16-bit tolerance (FP32 accumulation of exact 16-bit products)."""
    fat, lng = hin.gen_links(L, 1000, 0.3, 0.1)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    lat = hisq.Lattice(L, precs=(0, prec)).load(fat, lng)
    dims = "x".join(map(str, L))
    hisq.hisq_tune_load(lat.ctx, "dslash_path_il/l%d/n%d %s -> 2\n" % (prec, nrhs, dims))
    src = hin.gen_source(1700 + nrhs, lat.half, nrhs)
    y = empty_interleaved(lat.half, nrhs, prec)
    lat.dslash_interleaved(parity, y, to_device(interleave(src), prec), prec, nrhs)
    got = deinterleave(from_device(y, prec))
    for r in range(nrhs):
        ref = oracle.dslash(L, ff, lf, parity, src[r])
        assert rel_err(got[r], ref) <= TOL[prec], (L, prec, nrhs, parity, r, rel_err(got[r], ref))
    assert "dslash_path_il/l%d/n%d %s -> 2" % (prec, nrhs, dims) in hisq.hisq_tune_report(lat.ctx)
    lat.close()


def test_tensor_core_form_chooser(hisq):
    """Without a loaded entry the first call times both forms, keeps the faster and records it; the
    result is correct either way."""
    L = (16, 16, 16, 8)
    lat, ff, lf = setup(hisq, L)
    nrhs, prec = 32, 2
    src = hin.gen_source(1800, lat.half, nrhs)
    y = empty_interleaved(lat.half, nrhs, prec)
    lat.dslash_interleaved(0, y, to_device(interleave(src), prec), prec, nrhs)
    got = deinterleave(from_device(y, prec))
    for r in (0, 17, 31):
        assert rel_err(got[r], oracle.dslash(L, ff, lf, 0, src[r])) <= TOL[prec]
    rep = hisq.hisq_tune_report(lat.ctx)
    assert any(l.startswith("dslash_path_il/l2/n32 ") and l.split()[-1] in ("1", "2") for l in rep.splitlines())
