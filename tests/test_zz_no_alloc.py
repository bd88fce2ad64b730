"""The no-allocation variant of the A operator against the allocating one, through the C ABI.

hisq_apply_A_noalloc serves callers that cannot allocate device memory during the call
(framework-owned allocators, latency-critical loops): it keeps the
odd-site intermediate in a fixed device array instead of a cudaMalloc'ed workspace. Here its output
must match hisq_apply_A's within the operator tolerances, on two calls in a row, and sizes beyond
the fixed maximum must be refused with an error.
"""
import ctypes

import numpy as np
import pytest

import hisq_inputs as hin
import oracle

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-6, 2: 5e-3, 3: 5e-3, 4: 1e-12}


def _device_vec(torch, src, prec):
    t = torch.from_numpy(np.ascontiguousarray(src))
    if prec in (0, 4):
        return t.cuda()
    if prec == 1:
        return t.to(torch.complex64).cuda()
    r = torch.view_as_real(t.to(torch.complex64))
    return r.to(torch.float16 if prec == 2 else torch.bfloat16).contiguous().cuda()


def _to_numpy(torch, t, prec):
    t = t.cpu()
    if prec in (2, 3):
        t = torch.view_as_complex(t.float().contiguous())
    return t.to(torch.complex128).numpy()


def test_noalloc_matches_apply_A_two_calls(hisq):
    import torch
    L = (8, 10, 12, 14)
    fat, lng = hin.gen_links(L, 1234, 0.3, 0.1)
    lat = hisq.Lattice(L).load(fat, lng)
    cases = [(0, 1, 0.05, 0.3, 11), (1, 3, 0.02, 0.0, 12)]  # two calls in a row, different shapes
    for prec, nrhs, mass, sigma, seed in cases:
        src = hin.gen_source(seed, lat.half, nrhs)
        x = _device_vec(torch, src, prec)
        y_ref, y_na = torch.empty_like(x), torch.empty_like(x)
        lat.apply_A(y_ref, x, mass, prec, nrhs, sigma=sigma)
        hisq.hisq_apply_A_noalloc(lat.ctx, y_na, x, mass, sigma, prec, nrhs)
        torch.cuda.synchronize()
        a, b = _to_numpy(torch, y_na, prec), _to_numpy(torch, y_ref, prec)
        err = np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())
        assert err <= TOL[prec], (prec, nrhs, err)


def test_noalloc_refuses_oversize_and_host_vectors(hisq):
    import torch
    L = (16, 16, 16, 16)
    fat, lng = hin.gen_links(L, 99, 0.3, 0.1)
    lat = hisq.Lattice(L, precs=(0,)).load(fat, lng)
    # 16^4 FP64: 1.5 MiB of intermediate per rhs; 32 rhs exceed the fixed maximum
    nrhs = 32
    assert nrhs * lat.half * 6 * 8 > hisq.HISQ_NOALLOC_SCRATCH_BYTES
    x = torch.zeros((nrhs, lat.half, 3), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(hisq.HisqError) as e:
        hisq.hisq_apply_A_noalloc(lat.ctx, y, x, 0.1, 0.0, 0, nrhs)
    assert e.value.code == hisq.HISQ_EINVAL and "fixed maximum" in str(e.value)
    xh = np.zeros((1, lat.half, 3), np.complex128)
    with pytest.raises(hisq.HisqError) as e:
        hisq.hisq_apply_A_noalloc(lat.ctx, np.zeros_like(xh), xh, 0.1, 0.0, 0, 1)
    assert e.value.code == hisq.HISQ_EINVAL


def test_noalloc_16bit_multi_rhs_and_double_float_against_oracle(hisq):
    """The routes the first test does not reach, checked against the oracle's A directly: 16-bit storage
    with 8 vectors (one multi-vector launch per Dslash, its form picked by the autotuner at the first
    call) and the double-float operator, each called twice in a row on the shared scratch array."""
    import torch
    L = (8, 10, 12, 14)
    fat, lng = hin.gen_links(L, 1234, 0.3, 0.1)
    lat = hisq.Lattice(L, precs=(0, 2, 3, 4)).load(fat, lng)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    cases = [(2, 8, 0.05, 0.0, 21), (3, 8, 0.03, 0.2, 22), (4, 1, 0.05, 0.3, 23), (4, 2, 0.1, 0.0, 24)]
    for prec, nrhs, mass, sigma, seed in cases:
        src = hin.gen_source(seed, lat.half, nrhs)
        x = _device_vec(torch, src, prec)
        for call in range(2):
            y = torch.full_like(x, float("nan"))  # a stale result cannot pass
            hisq.hisq_apply_A_noalloc(lat.ctx, y, x, mass, sigma, prec, nrhs)
            torch.cuda.synchronize()
            got = _to_numpy(torch, y, prec)
            for r in range(nrhs):
                ref = oracle.apply_A(L, ff, lf, mass, src[r], sigma=sigma)
                err = np.linalg.norm((got[r] - ref).ravel()) / np.linalg.norm(ref.ravel())
                # two Dslash applications: twice the single-operator tolerance
                assert err <= 2 * TOL[prec], (prec, nrhs, call, r, err)


def test_noalloc_leaves_free_device_memory_unchanged(hisq):
    """What the entry point is for, observed from outside: once first calls have tuned the Dslash launches
    of each shape and looked up the scratch array, further calls of either shape, with other masses and
    shifts, leave the device's free memory exactly as it was."""
    import torch
    L = (16, 16, 16, 8)
    fat, lng = hin.gen_links(L, 77, 0.3, 0.1)
    lat = hisq.Lattice(L, precs=(0, 1)).load(fat, lng)
    x1 = torch.from_numpy(hin.gen_source(31, lat.half, 1)).to(torch.complex64).cuda()
    y1 = torch.empty_like(x1)
    hisq.hisq_apply_A_noalloc(lat.ctx, y1, x1, 0.05, 0.0, 1, 1)  # warm-up: tuning, symbol lookup
    x4 = torch.from_numpy(hin.gen_source(32, lat.half, 4)).to(torch.complex64).cuda()
    y4 = torch.empty_like(x4)
    hisq.hisq_apply_A_noalloc(lat.ctx, y4, x4, 0.05, 0.0, 1, 4)  # tunes the 4-vector launch forms
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for nrhs, x, y in ((1, x1, y1), (4, x4, y4), (1, x1, y1)):
        hisq.hisq_apply_A_noalloc(lat.ctx, y, x, 0.07, 0.1, 1, nrhs)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
