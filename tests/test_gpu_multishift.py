"""GPU multi-shift CG through the C ABI: every shift's solution is judged by its true FP64 residual,
recomputed by the oracle operator, and compared with the oracle's multi-shift solution and, at unit
links, with the FFT-exact solution of each shifted system."""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
from test_oracle_solvers import fft_solve

pytestmark = pytest.mark.gpu

SHIFTS = np.logspace(-5, 0, 14)


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_multishift_random_field(hisq, inner):
    import torch
    L = (8, 10, 12, 14)
    mass = 0.0025
    fat, lng = hin.gen_links(L, 1002, 0.3, 0.1)
    lat = hisq.Lattice(L).load(fat, lng)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    b = hin.gen_source(2002, lat.half, 1)
    x = torch.zeros((len(SHIFTS), lat.half, 3), dtype=torch.complex128, device="cuda")
    rc, st = lat.multishift_cg(x, torch.from_numpy(b).cuda(), SHIFTS, mass, 1e-9, 5000, inner_prec=inner)
    assert rc == 0 and st["converged"] == 1
    xs = x.cpu().numpy()
    x_ref, _, _ = oracle.multishift_cg(L, ff, lf, mass, SHIFTS, b[0], 1e-11)
    for k, s in enumerate(SHIFTS):
        r = oracle.true_residual(L, ff, lf, mass, b[0], xs[k], sigma=s)
        assert r <= 1e-9, (k, r)
        assert abs(r - st["shift_residual"][k]) < 1e-10
        assert np.linalg.norm(xs[k] - x_ref[k]) / np.linalg.norm(x_ref[k]) < 1e-6
    # larger shifts converge earlier in the shared Krylov space
    its = st["shift_iters"]
    assert all(i > 0 for i in its)
    assert its[-1] <= its[0]


def test_multishift_free_field_exact(hisq):
    import torch
    L = (8, 10, 12, 14)
    V = oracle.volume(L)
    fat = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    lat = hisq.Lattice(L, precs=(0, 1)).load(fat, -fat / 24)
    b = hin.gen_source(21, lat.half, 1)
    x = torch.zeros((len(SHIFTS), lat.half, 3), dtype=torch.complex128, device="cuda")
    lat.multishift_cg(x, torch.from_numpy(b).cuda(), SHIFTS, 0.0025, 1e-11, 5000, inner_prec=0)
    for k, s in enumerate(SHIFTS):
        x_exact, _ = fft_solve(L, 0.0025, s, b[0])
        assert np.linalg.norm(x.cpu().numpy()[k] - x_exact) / np.linalg.norm(x_exact) < 1e-9


def test_multishift_host_buffers_per_shift_tolerance(hisq):
    L = (4, 6, 8, 10)
    fat, lng = hin.gen_links(L, 9, 0.3, 0.1)
    lat = hisq.Lattice(L, precs=(0, 1)).load(fat, lng)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    b = hin.gen_source(90, lat.half, 1)
    shifts = np.array([0.5, 0.01, 0.1])
    tols = np.array([1e-6, 1e-10, 1e-8])
    x = np.zeros((3, lat.half, 3), np.complex128)
    rc, st = lat.multishift_cg(x, b, shifts, 0.05, tols, 2000, inner_prec=1)
    for k in range(3):
        assert oracle.true_residual(L, ff, lf, 0.05, b[0], x[k], sigma=shifts[k]) <= tols[k]


def test_multishift_errors(hisq):
    import torch
    L = (4, 6, 8, 10)
    fat, lng = hin.gen_links(L, 9)
    lat = hisq.Lattice(L, precs=(0,)).load(fat, lng)
    b = torch.from_numpy(hin.gen_source(1, lat.half, 1)).cuda()
    x = torch.zeros((2, lat.half, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(hisq.HisqError) as e:
        lat.multishift_cg(x, b, [0.1, -1.0], 0.1, 1e-8, 100)
    assert e.value.code == hisq.HISQ_EINVAL
    with pytest.raises(hisq.HisqError) as e:
        lat.multishift_cg(x, b, [0.1, 0.2], 0.1, 1e-8, 100, inner_prec=1)  # FP32 links not resident
    assert e.value.code == hisq.HISQ_EINVAL


@pytest.mark.parametrize("inner", [0, 1])
def test_rational_apply(hisq, inner):
    """RHMC's rational apply r(A) b = a0 b + sum_k a_k (A + s_k)^-1 b against the oracle's composition."""
    import torch
    L = (8, 10, 12, 14)
    mass = 0.01
    fat, lng = hin.gen_links(L, 321, 0.3, 0.1)
    lat = hisq.Lattice(L, precs=(0, 1)).load(fat, lng)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    b = hin.gen_source(322, lat.half, 1)[0]
    a0, coeffs, shifts = 0.25, [0.9, 0.4, 0.1, 0.05], [1e-4, 1e-2, 0.3, 2.0]
    out = torch.empty((lat.half, 3), dtype=torch.complex128, device="cuda")
    st = hisq.hisq_rational_apply(lat.ctx, out, torch.from_numpy(b).cuda(), a0, shifts, coeffs, mass, 1e-11, 5000,
                                  hisq.make_opts(inner_prec=inner))
    assert st["converged"] == 1
    ref = oracle.rational_apply(L, ff, lf, mass, b, a0, coeffs, shifts, tol=1e-13)
    assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-8
