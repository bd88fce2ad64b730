"""GPU solvers through the C ABI, judged by the oracle: every solve's true FP64 residual is recomputed by
the oracle operator on the returned x, and free-field solutions are compared with the FFT-exact answer."""
import numpy as np
import pytest

import hisq_inputs as hin
import oracle
from test_oracle_solvers import fft_solve

pytestmark = pytest.mark.gpu


def lattice(hisq, L, seed, eps=0.3, precs=(0, 1, 2, 3, 4)):
    fat, lng = hin.gen_links(L, seed, eps, 0.1)
    lat = hisq.Lattice(L, precs=precs).load(fat, lng)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    return lat, ff, lf


@pytest.mark.parametrize("inner,rel", [(0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (4, 4), (1, 4), (2, 4)])
def test_cg_8444_plain_method(hisq, inner, rel):
    """8^4, m = 0.1, eps = 0.3 links, Gaussian source, to relative residual 1e-10; inner 4 is plain CG with
    the double-float operator, rel 4 takes the reliable updates and true residuals in double-float."""
    import torch
    L = (8, 8, 8, 8)
    lat, ff, lf = lattice(hisq, L, 1000)
    b = hin.gen_source(2000, lat.half, 1)
    x = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
    rc, st = lat.cg(x, torch.from_numpy(b).cuda(), 0.1, 1e-10, 2000, inner_prec=inner, reliable_prec=rel)
    assert rc == 0 and st["converged"] == 1
    xs = x.cpu().numpy()[0]
    r_oracle = oracle.true_residual(L, ff, lf, 0.1, b[0], xs)
    assert r_oracle <= 1e-10
    assert abs(r_oracle - st["true_rel_residual"]) < 1e-11
    x_ref, _ = oracle.cg(L, ff, lf, 0.1, b[0], tol=1e-12)
    assert np.linalg.norm(xs - x_ref) / np.linalg.norm(x_ref) < 1e-8
    if inner not in (0, 4):
        assert st["reliable_updates"] >= 1


@pytest.mark.parametrize("inner", [1, 2])
def test_cg_every_single_vector_launch_form(hisq, inner):
    """Mixed CG (FP32 inner vectors, FP32 or FP16 links) with each single-vector Dslash launch form forced
    for both of its Dslash launches, the fused one reducing <p, Ap> over one resident wave of blocks: cb
    order and the tiled walk. Each solve is judged by the oracle's true residual; the forms reduce in
    different orders, so iteration counts may differ by a step or two."""
    import torch
    L = (8, 10, 12, 14)
    dims = "%dx%dx%dx%d" % L
    its = []
    for vi in range(2):
        lat, ff, lf = lattice(hisq, L, 1003, precs=(0, inner))
        for epi in (0, 1):
            key = "dslash/l%d/s1/nr1/e%d/c0" % (inner, epi)
            assert hisq.hisq_tune_load(lat.ctx, "%s %s -> %d\n" % (key, dims, vi * 10000 + 96)) == 1
        b = hin.gen_source(2003, lat.half, 1)
        x = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
        rc, st = lat.cg(x, torch.from_numpy(b).cuda(), 0.05, 1e-10, 4000, inner_prec=inner, reliable_period=50)
        assert rc == 0 and st["converged"] == 1, vi
        assert oracle.true_residual(L, ff, lf, 0.05, b[0], x.cpu().numpy()[0]) <= 1e-10, vi
        its.append(st["iters"])
        lat.close()
    assert max(its) - min(its) <= 2, its


@pytest.mark.parametrize("inner", [0, 1])
def test_cg_free_field_exact(hisq, inner):
    import torch
    L = (8, 10, 12, 14)
    V = oracle.volume(L)
    fat = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    lat = hisq.Lattice(L, precs=(0, 1)).load(fat, -fat / 24)
    b = hin.gen_source(11, lat.half, 1)
    x = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
    lat.cg(x, torch.from_numpy(b).cuda(), 0.05, 1e-11, 5000, inner_prec=inner)
    x_exact, _ = fft_solve(L, 0.05, 0.0, b[0])
    assert np.linalg.norm(x.cpu().numpy()[0] - x_exact) / np.linalg.norm(x_exact) < 1e-9


@pytest.mark.parametrize("inner,nrhs", [(0, 5), (1, 5), (2, 5), (1, 8), (1, 21), (3, 16)])
def test_cg_multi_rhs(hisq, inner, nrhs):
    """Groups of 8 and 16 vectors run with 2 and 4 threads per site; 21 = 16 + 4 + 1."""
    import torch
    L = (8, 10, 12, 14)
    lat, ff, lf = lattice(hisq, L, 7)
    b = hin.gen_source(70, lat.half, nrhs)
    b[3] *= 1e-3  # different scales per rhs
    x = torch.zeros((nrhs, lat.half, 3), dtype=torch.complex128, device="cuda")
    rc, st = lat.cg(x, torch.from_numpy(b).cuda(), 0.02, 1e-10, 5000, nrhs=nrhs, inner_prec=inner)
    xs = x.cpu().numpy()
    for r in range(nrhs):
        assert oracle.true_residual(L, ff, lf, 0.02, b[r], xs[r]) <= 1e-10


def test_cg_host_buffers_and_guess(hisq):
    """Host (numpy) x and b; a converged initial guess returns at once."""
    L = (4, 6, 8, 10)
    lat, ff, lf = lattice(hisq, L, 3)
    b = hin.gen_source(30, lat.half, 1)
    x = np.zeros_like(b)
    rc, st = lat.cg(x, b, 0.1, 1e-10, 1000, inner_prec=1)
    assert oracle.true_residual(L, ff, lf, 0.1, b[0], x[0]) <= 1e-10
    rc, st2 = lat.cg(x, b, 0.1, 1e-10, 1000)
    assert st2["iters"] == 0


def test_cg_no_graph_matches_graph(hisq):
    import torch
    L = (8, 10, 12, 14)
    lat, ff, lf = lattice(hisq, L, 5)
    b = torch.from_numpy(hin.gen_source(50, lat.half, 1)).cuda()
    x1 = torch.zeros_like(b)
    x2 = torch.zeros_like(b)
    _, s1 = lat.cg(x1, b, 0.05, 1e-10, 2000, inner_prec=1, use_graph=True)
    _, s2 = lat.cg(x2, b, 0.05, 1e-10, 2000, inner_prec=1, use_graph=False)
    assert s1["iters"] == s2["iters"]
    assert torch.equal(x1, x2)  # deterministic reductions, same launch shapes


def test_cg_errors(hisq):
    import torch
    L = (4, 6, 8, 10)
    lat, ff, lf = lattice(hisq, L, 3, precs=(0, 1))
    b = torch.from_numpy(hin.gen_source(30, lat.half, 1)).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(hisq.HisqError) as e:
        lat.cg(x, b, 0.0, 1e-10, 100)
    assert e.value.code == hisq.HISQ_EINVAL
    with pytest.raises(hisq.HisqError) as e:
        lat.cg(x, b, 0.1, 1e-10, 100, inner_prec=2)  # FP16 links not resident
    assert e.value.code == hisq.HISQ_EINVAL
    with pytest.raises(hisq.HisqError) as e:
        lat.cg(x, b, 0.1, 1e-10, 100, inner_prec=1, reliable_prec=4)  # double-float links not resident
    assert e.value.code == hisq.HISQ_EINVAL
    with pytest.raises(hisq.HisqError) as e:
        lat.cg(x, b, 0.1, 1e-10, 100, inner_prec=1, reliable_prec=1)  # reliable updates need FP64-class
    assert e.value.code == hisq.HISQ_EINVAL
    rc, st = hisq.hisq_cg(lat.ctx, x, b, 1, 0.001, 1e-12, 3, hisq.make_opts(poll_every=1), raise_on_error=False)
    assert rc == hisq.HISQ_ENOCONV and st["converged"] == 0
    assert st["true_rel_residual"] > 1e-12
    bad = b.clone()
    bad[0, 3, 1] = float("nan")
    with pytest.raises(hisq.HisqError) as e:
        lat.cg(torch.zeros_like(b), bad, 0.1, 1e-10, 100)
    assert e.value.code == hisq.HISQ_ENONFINITE


def test_cg_repeated_solves_reuse_graphs(hisq):
    """Solves on one context replay cached graphs keyed by their coefficients and buffers: alternating masses
    (different per-rhs diagonal captured in the graph) each meet their true residual, and repeating a solve
    reproduces it bit for bit."""
    import torch
    L = (8, 10, 12, 14)
    lat, ff, lf = lattice(hisq, L, 41)
    b = hin.gen_source(42, lat.half, 1)
    bt = torch.from_numpy(b).cuda()
    xs = []
    for mass in (0.1, 0.05, 0.1):
        x = torch.zeros_like(bt)
        rc, st = lat.cg(x, bt, mass, 1e-10, 5000, inner_prec=1)
        assert rc == 0
        assert oracle.true_residual(L, ff, lf, mass, b[0], x.cpu().numpy()[0]) <= 1e-10
        xs.append(x.cpu())
    assert torch.equal(xs[0], xs[2])
    assert not torch.equal(xs[0], xs[1])


def test_cg_zero_source_and_max_rhs(hisq):
    """Degenerate and maximal cases: a zero source returns x = 0 at once; 64 right-hand sides (the
    maximum) in one mixed solve, every one to its true residual."""
    import torch
    L = (4, 6, 8, 10)
    lat, ff, lf = lattice(hisq, L, 51, precs=(0, 1))
    z = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
    x = torch.ones_like(z)
    rc, st = lat.cg(x, z, 0.1, 1e-10, 100, inner_prec=1)
    assert rc == 0 and st["converged"] == 1 and st["iters"] == 0
    assert float(torch.linalg.vector_norm(x)) == 0.0 and st["true_rel_residual"] == 0.0
    b = hin.gen_source(52, lat.half, 64)
    x = torch.zeros((64, lat.half, 3), dtype=torch.complex128, device="cuda")
    rc, st = lat.cg(x, torch.from_numpy(b).cuda(), 0.1, 1e-10, 2000, nrhs=64, inner_prec=1)
    assert rc == 0
    xs = x.cpu().numpy()
    for r in (0, 17, 63):
        assert oracle.true_residual(L, ff, lf, 0.1, b[r], xs[r]) <= 1e-10


@pytest.mark.parametrize("inner,nrhs", [(1, 2), (1, 14), (2, 4), (3, 6)])
def test_cg_interleaved_inner_vectors_match_blocked(hisq, inner, nrhs):
    """Mixed-precision multi-RHS solves keep their inner vectors in the boundary layout (vector_layout 0,
    the default) or interleaved per site (vector_layout 1, even rhs counts). Both are judged by the
    oracle's true residual, and they take the same number of iterations up to rounding."""
    import torch
    L = (8, 10, 12, 14)
    lat, ff, lf = lattice(hisq, L, 7)
    b = hin.gen_source(71, lat.half, nrhs)
    b[1] *= 1e-3  # different scales per rhs
    its = []
    for layout in (0, 1):
        x = torch.zeros((nrhs, lat.half, 3), dtype=torch.complex128, device="cuda")
        rc, st = lat.cg(x, torch.from_numpy(b).cuda(), 0.02, 1e-10, 5000, nrhs=nrhs, inner_prec=inner,
                        vector_layout=layout)
        assert rc == 0 and st["converged"] == 1
        xs = x.cpu().numpy()
        for r in range(nrhs):
            assert oracle.true_residual(L, ff, lf, 0.02, b[r], xs[r]) <= 1e-10, (layout, r)
        its.append(st["iters"])
    assert abs(its[0] - its[1]) <= 3, its


@pytest.mark.parametrize("inner", [0, 1])
def test_cg_lanczos_estimate_free_field(hisq, inner):
    """The solve's Lanczos estimate of A's extreme eigenvalues (from rhs 0's CG coefficients) against the
    closed-form free-field spectrum at unit links: the largest converges within a few iterations, the
    smallest as the solve converges. Mixed precision restarts its search direction at every reliable
    update; its estimate comes from one cycle of 50 iterations and is looser."""
    import torch
    from test_oracle_dslash import free_field_eigs
    L = (8, 8, 8, 8)
    V = oracle.volume(L)
    fat = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    lat = hisq.Lattice(L, precs=(0, 1)).load(fat, -fat / 24)
    mass = 0.1
    lam = free_field_eigs(L, mass).ravel()
    b = hin.gen_source(13, lat.half, 1)
    x = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
    rc, st = lat.cg(x, torch.from_numpy(b).cuda(), mass, 1e-12, 5000, inner_prec=inner)
    assert rc == 0 and st["lanczos_steps"] >= 10
    tol_max, tol_min = (1e-8, 1e-6) if inner == 0 else (1e-4, 5e-2)
    assert abs(st["lambda_max"] / lam.max() - 1) < tol_max, (st["lambda_max"], lam.max())
    assert abs(st["lambda_min"] / lam.min() - 1) < tol_min, (st["lambda_min"], lam.min())


@pytest.mark.parametrize("prec,nrhs", [(2, 1), (3, 1), (2, 5), (3, 8)])
def test_cg_16bit_spinor_storage(hisq, prec, nrhs):
    """Mixed CG with the inner vectors stored in the links' 16-bit format (FP16 or BF16 r, p, Ap and Dslash
    intermediate; FP32 arithmetic, FP64 reductions, reliable updates and solution): every rhs reaches a true
    residual of 1e-10, judged by the oracle, at the benchmark mass on rough links, and within twice the
    iterations of the same solve with FP32 inner vectors."""
    import torch
    L = (8, 10, 12, 14)
    lat, ff, lf = lattice(hisq, L, 17)
    b = hin.gen_source(170, lat.half, nrhs)
    bd = torch.from_numpy(b).cuda()
    its = {}
    for sp in (1, prec):
        x = torch.zeros((nrhs, lat.half, 3), dtype=torch.complex128, device="cuda")
        rc, st = lat.cg(x, bd, 0.01, 1e-10, 5000, nrhs=nrhs, inner_prec=prec, spinor_prec=sp)
        assert rc == 0 and st["converged"] == 1
        xs = x.cpu().numpy()
        for r in range(nrhs):
            assert oracle.true_residual(L, ff, lf, 0.01, b[r], xs[r]) <= 1e-10, (sp, r)
        its[sp] = st["iters"]
    assert its[prec] <= 2 * its[1], its


def test_cg_16bit_spinor_storage_errors(hisq):
    """16-bit inner vectors need links of the same format and the blocked layout, and only hisq_cg has them."""
    import torch
    L = (4, 6, 8, 10)
    lat, ff, lf = lattice(hisq, L, 3, precs=(0, 1, 2, 3))
    b = torch.from_numpy(hin.gen_source(31, lat.half, 2)).cuda()
    x = torch.zeros_like(b)
    for inner, sp, layout in ((1, 2, 0), (2, 3, 0), (3, 2, 0), (2, 2, 1), (2, 0, 0), (2, 4, 0)):
        with pytest.raises(hisq.HisqError) as e:
            lat.cg(x, b, 0.1, 1e-10, 100, nrhs=2, inner_prec=inner, spinor_prec=sp, vector_layout=layout)
        assert e.value.code == hisq.HISQ_EINVAL, (inner, sp, layout)
    xs = torch.zeros((2, lat.half, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(hisq.HisqError) as e:
        lat.multishift_cg(xs, b[:1], [0.0, 0.1], 0.1, [1e-9, 1e-9], 100, inner_prec=2, spinor_prec=2)
    assert e.value.code == hisq.HISQ_EINVAL
