"""Python binding of the GB300 HISQ even/odd operator library (libhisq.so).

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels.
The functions carry the C ABI's names (include/hisq.h). Vectors may be torch tensors (device
or host) or numpy arrays; they are passed to the library as raw pointers.

If libhisq.so has not been built, every call raises RuntimeError: there is no CPU fallback.
Build it with ``paper_2111_10354_gb300.build.build()`` (needs nvcc) or ``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhisq.so")

HISQ_OK = 0
HISQ_EINVAL = -1
HISQ_ENOLINKS = -2
HISQ_ENOMEM = -3
HISQ_ECUDA = -4
HISQ_ENONFINITE = -5
HISQ_ENOCONV = -6
HISQ_EBREAKDOWN = -7
HISQ_ETIMEOUT = -8

HISQ_F64, HISQ_F32, HISQ_F16, HISQ_BF16, HISQ_DF64 = 0, 1, 2, 3, 4
PREC_NAMES = {HISQ_F64: "f64", HISQ_F32: "f32", HISQ_F16: "f16", HISQ_BF16: "bf16", HISQ_DF64: "df64"}
HISQ_APPLY_PHASES = 1
HISQ_ANTIPERIODIC_T = 2
HISQ_PREC_ALL = 0x1F
HISQ_NOALLOC_SCRATCH_BYTES = 32 << 20


def HISQ_PREC_BIT(p: int) -> int:
    return 1 << p


class hisq_solver_opts(ctypes.Structure):
    _fields_ = [("inner_prec", ctypes.c_int), ("reliable_period", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("poll_every", ctypes.c_int), ("reliable_prec", ctypes.c_int), ("vector_layout", ctypes.c_int),
                ("spinor_prec", ctypes.c_int)]


class hisq_solver_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("converged", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("dslash_bytes", ctypes.c_double), ("dslash_calls", ctypes.c_longlong),
                ("shift_iters", ctypes.c_int * 64), ("shift_residual", ctypes.c_double * 64),
                ("kernel_launches", ctypes.c_longlong), ("lambda_min", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("lanczos_steps", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("shift_iters", "shift_residual")}
        return d


class hisq_smear_coeffs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("one_link", "three_staple", "five_staple", "seven_staple", "lepage",
                                                "naik")]


def smear_coeffs(c1=0.0, c3=0.0, c5=0.0, c7=0.0, cL=0.0, cN=0.0) -> hisq_smear_coeffs:
    """Path coefficients of one smearing level: one link, 3-, 5-, 7-link staples, Lepage, Naik."""
    return hisq_smear_coeffs(c1, c3, c5, c7, cL, cN)


class HisqError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str, stats=None):
        self.code = code
        self.stats = stats
        super().__init__("%s: %s (%d): %s" % (where, hisq_strerror(code), code, detail))


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhisq.so is not built (%s); run paper_2111_10354_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.hisq_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ctypes.c_uint, vp]
    lib.hisq_destroy.argtypes = [vp]
    lib.hisq_load_links.argtypes = [vp, vp, vp, ctypes.c_uint]
    lib.hisq_load_links_slab.argtypes = [vp, ip, ip, vp, vp, ctypes.c_uint]
    lib.hisq_dslash.argtypes = [vp, ip, vp, vp, ip, ip]
    lib.hisq_apply_A.argtypes = [vp, vp, vp, dp, dp, ip, ip]
    lib.hisq_apply_A_noalloc.argtypes = [vp, vp, vp, dp, dp, ip, ip]
    lib.hisq_dslash_interleaved.argtypes = [vp, ip, vp, vp, ip, ip]
    lib.hisq_lanczos_extremes.argtypes = [vp, vp, ip, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
    lib.hisq_apply_A_interleaved.argtypes = [vp, vp, vp, dp, dp, ip, ip]
    lib.hisq_solver_opts_default.argtypes = [ctypes.POINTER(hisq_solver_opts)]
    lib.hisq_solver_opts_default.restype = None
    lib.hisq_cg.argtypes = [vp, vp, vp, ip, dp, dp, ip, ctypes.POINTER(hisq_solver_opts),
                            ctypes.POINTER(hisq_solver_stats)]
    if hasattr(lib, "hisq_multishift_cg"):
        lib.hisq_multishift_cg.argtypes = [vp, vp, vp, ip, vp, dp, vp, ip, ctypes.POINTER(hisq_solver_opts),
                                           ctypes.POINTER(hisq_solver_stats)]
    lib.hisq_strerror.argtypes = [ip]
    lib.hisq_strerror.restype = ctypes.c_char_p
    lib.hisq_last_error.argtypes = []
    lib.hisq_last_error.restype = ctypes.c_char_p
    lib.hisq_dslash_bytes.argtypes = [vp, ip, ip]
    lib.hisq_dslash_bytes.restype = ctypes.c_double
    lib.hisq_set_autotune.argtypes = [vp, ip]
    lib.hisq_set_pdl.argtypes = [vp, ip]
    lib.hisq_set_long_compression.argtypes = [vp, dp]
    lib.hisq_launch_count.argtypes = [vp]
    lib.hisq_launch_count.restype = ctypes.c_longlong
    lib.hisq_tune_report.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.hisq_tune_load.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
    lib.hisq_selftest_bounded_wait.argtypes = [vp]
    lib.hisq_release_workspaces.argtypes = [vp]
    cp = ctypes.POINTER(hisq_smear_coeffs)
    lib.hisq_smear.argtypes = [vp, vp, vp, vp, cp, ip]
    lib.hisq_project_u3.argtypes = [vp, vp, vp]
    lib.hisq_hisq_links.argtypes = [vp, vp, vp, vp, cp, cp, ip]
    lib.hisq_batch_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(ctypes.c_int), ctypes.c_uint, vp]
    lib.hisq_batch_destroy.argtypes = [vp]
    lib.hisq_batch_load_links.argtypes = [vp, ip, vp, vp, ctypes.c_uint]
    lib.hisq_batch_vector_offset.argtypes = [vp, ip]
    lib.hisq_batch_vector_offset.restype = ctypes.c_longlong
    lib.hisq_batch_launch_count.argtypes = [vp]
    lib.hisq_batch_launch_count.restype = ctypes.c_longlong
    lib.hisq_batch_cg.argtypes = [vp, vp, vp, vp, dp, ip, ctypes.POINTER(hisq_solver_opts),
                                  ctypes.POINTER(hisq_solver_stats), vp, vp]
    lib.hisq_rational_apply.argtypes = [vp, vp, vp, dp, ip, vp, vp, dp, vp, ip, ctypes.POINTER(hisq_solver_opts),
                                        ctypes.POINTER(hisq_solver_stats)]
    fp = ctypes.c_float
    lib.hisq_ptc_create.argtypes = [ctypes.POINTER(vp), vp, ip]
    lib.hisq_ptc_destroy.argtypes = [vp]
    lib.hisq_ptc_set_weights.argtypes = [vp, vp, vp]
    lib.hisq_ptc_get_weights.argtypes = [vp, vp, vp]
    lib.hisq_ptc_apply.argtypes = [vp, vp, vp, ip]
    lib.hisq_ptc_bind.argtypes = [vp, vp]
    lib.hisq_ptc_set_tied.argtypes = [vp, ip]
    lib.hisq_ptc_train_step.argtypes = [vp, vp, vp, ip, fp, vp, vp, vp]
    lib.hisq_fcg.argtypes = [vp, vp, vp, vp, dp, dp, ip, ctypes.POINTER(hisq_solver_opts),
                             ctypes.POINTER(hisq_solver_stats)]
    _lib = lib
    return lib


def lib():
    return _load()


def _check(rc: int, where: str, stats=None):
    if rc != HISQ_OK:
        raise HisqError(rc, where, hisq_last_error(), stats)


def _ptr(a):
    """Raw pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    raise TypeError("expected a torch tensor, numpy array or pointer, got %r" % type(a))


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream) if stream.cuda_stream else None
    return ctypes.c_void_p(int(stream))


# ---------------------------------------------------------------- C ABI, same names

def hisq_strerror(code: int) -> str:
    return _load().hisq_strerror(code).decode()


def hisq_last_error() -> str:
    return _load().hisq_last_error().decode()


def hisq_create(dims, prec_mask: int = HISQ_PREC_ALL, stream=None):
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(_load().hisq_create(ctypes.byref(h), d, prec_mask, _stream_handle(stream)), "hisq_create")
    return h


def hisq_destroy(ctx):
    _check(_load().hisq_destroy(ctx), "hisq_destroy")


def _links_arg(a):
    """Links as passed to the library: a complex128 torch tensor (host or device) as is, anything
    else as a contiguous complex128 numpy array."""
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != "torch.complex128":
            raise TypeError("links must be complex128, got %s" % a.dtype)
        return a
    return np.ascontiguousarray(a, dtype=np.complex128)


def hisq_load_links(ctx, fat, lng, flags: int = HISQ_APPLY_PHASES | HISQ_ANTIPERIODIC_T):
    """fat, lng: host or device arrays in the link layout (complex128)."""
    fat, lng = _links_arg(fat), _links_arg(lng)
    _check(_load().hisq_load_links(ctx, _ptr(fat), _ptr(lng), flags), "hisq_load_links")


def hisq_load_links_slab(ctx, t_begin: int, t_count: int, fat, lng,
                         flags: int = HISQ_APPLY_PHASES | HISQ_ANTIPERIODIC_T):
    fat, lng = _links_arg(fat), _links_arg(lng)
    _check(_load().hisq_load_links_slab(ctx, t_begin, t_count, _ptr(fat), _ptr(lng), flags), "hisq_load_links_slab")


def hisq_dslash(ctx, out_parity: int, out, in_, prec: int, nrhs: int = 1):
    _check(_load().hisq_dslash(ctx, out_parity, _ptr(out), _ptr(in_), prec, nrhs), "hisq_dslash")


def hisq_apply_A(ctx, out, in_, mass: float, sigma: float, prec: int, nrhs: int = 1):
    _check(_load().hisq_apply_A(ctx, _ptr(out), _ptr(in_), mass, sigma, prec, nrhs), "hisq_apply_A")


def hisq_dslash_interleaved(ctx, out_parity: int, out, in_, prec: int, nrhs: int):
    """hisq_dslash on the rhs-interleaved layout [cb][color][rhs]."""
    _check(_load().hisq_dslash_interleaved(ctx, out_parity, _ptr(out), _ptr(in_), prec, nrhs),
           "hisq_dslash_interleaved")


def hisq_apply_A_interleaved(ctx, out, in_, mass: float, sigma: float, prec: int, nrhs: int):
    """hisq_apply_A on the rhs-interleaved layout [cb][color][rhs]."""
    _check(_load().hisq_apply_A_interleaved(ctx, _ptr(out), _ptr(in_), mass, sigma, prec, nrhs),
           "hisq_apply_A_interleaved")


def hisq_lanczos_extremes(alpha, beta):
    """Extreme eigenvalues of the Lanczos tridiagonal matrix of CG coefficients alpha, beta (host)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError("alpha and beta differ in length")
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(_load().hisq_lanczos_extremes(a.ctypes.data, b.ctypes.data, len(a), ctypes.byref(lo), ctypes.byref(hi)),
           "hisq_lanczos_extremes")
    return lo.value, hi.value


def hisq_apply_A_noalloc(ctx, out, in_, mass: float, sigma: float, prec: int, nrhs: int = 1):
    """hisq_apply_A without any device allocation (fixed scratch array; device vectors only)."""
    _check(_load().hisq_apply_A_noalloc(ctx, _ptr(out), _ptr(in_), mass, sigma, prec, nrhs), "hisq_apply_A_noalloc")


def hisq_solver_opts_default() -> hisq_solver_opts:
    o = hisq_solver_opts()
    _load().hisq_solver_opts_default(ctypes.byref(o))
    return o


def make_opts(inner_prec: int = HISQ_F64, reliable_period: int = 50, use_graph: bool = True, poll_every: int = 25,
              reliable_prec: int = HISQ_F64, vector_layout: int = 0, spinor_prec: int = HISQ_F32):
    o = hisq_solver_opts_default()
    o.inner_prec, o.reliable_period, o.use_graph, o.poll_every = inner_prec, reliable_period, int(use_graph), \
        poll_every
    o.reliable_prec = reliable_prec
    o.vector_layout = vector_layout
    o.spinor_prec = spinor_prec
    return o


def hisq_cg(ctx, x, b, nrhs: int, mass: float, rel_tol: float, maxiter: int, opts=None, raise_on_error=True):
    """Returns (status, stats dict). x is updated in place."""
    st = hisq_solver_stats()
    o = opts if opts is not None else hisq_solver_opts_default()
    rc = _load().hisq_cg(ctx, _ptr(x), _ptr(b), nrhs, mass, rel_tol, maxiter, ctypes.byref(o), ctypes.byref(st))
    d = st.as_dict()
    if rc != HISQ_OK and raise_on_error:
        raise HisqError(rc, "hisq_cg", hisq_last_error(), d)
    return rc, d


def hisq_multishift_cg(ctx, x, b, shifts, mass: float, rel_tol, maxiter: int, opts=None, raise_on_error=True):
    """x: nshift vectors back to back. Returns (status, stats dict with per-shift lists)."""
    shifts = np.ascontiguousarray(shifts, dtype=np.float64)
    ns = len(shifts)
    tols = np.ascontiguousarray(np.broadcast_to(np.asarray(rel_tol, np.float64), (ns,)))
    st = hisq_solver_stats()
    o = opts if opts is not None else hisq_solver_opts_default()
    rc = _load().hisq_multishift_cg(ctx, _ptr(x), _ptr(b), ns, _ptr(shifts), mass, _ptr(tols), maxiter,
                                    ctypes.byref(o), ctypes.byref(st))
    d = st.as_dict()
    d["shift_iters"] = [int(st.shift_iters[k]) for k in range(ns)]
    d["shift_residual"] = [float(st.shift_residual[k]) for k in range(ns)]
    if rc != HISQ_OK and raise_on_error:
        raise HisqError(rc, "hisq_multishift_cg", hisq_last_error(), d)
    return rc, d


def hisq_rational_apply(ctx, out, b, a0: float, shifts, coeffs, mass: float, rel_tol, maxiter: int, opts=None):
    """out = a0 b + sum_k coeffs[k] (A + shifts[k])^-1 b; returns the multi-shift stats."""
    shifts = np.ascontiguousarray(shifts, dtype=np.float64)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    ns = len(shifts)
    tols = np.ascontiguousarray(np.broadcast_to(np.asarray(rel_tol, np.float64), (ns,)))
    st = hisq_solver_stats()
    o = opts if opts is not None else hisq_solver_opts_default()
    _check(_load().hisq_rational_apply(ctx, _ptr(out), _ptr(b), a0, ns, _ptr(shifts), _ptr(coeffs), mass, _ptr(tols),
                                       maxiter, ctypes.byref(o), ctypes.byref(st)), "hisq_rational_apply")
    return st.as_dict()


def hisq_dslash_bytes(ctx, prec: int, nrhs: int = 1) -> float:
    return float(_load().hisq_dslash_bytes(ctx, prec, nrhs))


def hisq_set_long_compression(ctx, naik: float):
    _check(_load().hisq_set_long_compression(ctx, naik), "hisq_set_long_compression")


def hisq_launch_count(ctx) -> int:
    return int(_load().hisq_launch_count(ctx))


def hisq_set_autotune(ctx, enable: bool):
    _check(_load().hisq_set_autotune(ctx, int(enable)), "hisq_set_autotune")


def hisq_set_pdl(ctx, enable: bool):
    _check(_load().hisq_set_pdl(ctx, int(enable)), "hisq_set_pdl")


def hisq_tune_report(ctx) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(_load().hisq_tune_report(ctx, buf, len(buf)), "hisq_tune_report")
    return buf.value.decode()


def hisq_tune_load(ctx, report: str) -> int:
    """Load a tune report (from hisq_tune_report) into a context; returns the entries taken."""
    n = ctypes.c_int(0)
    _check(_load().hisq_tune_load(ctx, report.encode(), ctypes.byref(n)), "hisq_tune_load")
    return n.value


def _coeffs(c):
    return c if isinstance(c, hisq_smear_coeffs) else smear_coeffs(**c)


def hisq_smear(ctx, fat, lng, thin, coeffs, prec: int = HISQ_F64):
    """One smearing level on the device (fat, lng, thin: device arrays in the link layout; lng may be
    None). coeffs: hisq_smear_coeffs or a dict of smear_coeffs' keywords."""
    c = _coeffs(coeffs)
    _check(_load().hisq_smear(ctx, _ptr(fat), _ptr(lng), _ptr(thin), ctypes.byref(c), prec), "hisq_smear")


def hisq_project_u3(ctx, out, in_):
    _check(_load().hisq_project_u3(ctx, _ptr(out), _ptr(in_)), "hisq_project_u3")


def hisq_hisq_links(ctx, fat, lng, thin, level1, level2, prec: int = HISQ_F64):
    c1, c2 = _coeffs(level1), _coeffs(level2)
    _check(_load().hisq_hisq_links(ctx, _ptr(fat), _ptr(lng), _ptr(thin), ctypes.byref(c1), ctypes.byref(c2), prec),
           "hisq_hisq_links")


def hisq_release_workspaces(ctx):
    _check(_load().hisq_release_workspaces(ctx), "hisq_release_workspaces")


def hisq_selftest_bounded_wait(ctx) -> int:
    """Status of the bounded-wait self-test (HISQ_ETIMEOUT when the wait gave up as intended)."""
    return _load().hisq_selftest_bounded_wait(ctx)


def hisq_batch_create(dims_list, prec_mask: int = HISQ_PREC_BIT(HISQ_F64) | HISQ_PREC_BIT(HISQ_F32), stream=None):
    h = ctypes.c_void_p()
    flat = [int(v) for d in dims_list for v in d]
    arr = (ctypes.c_int * len(flat))(*flat)
    _check(_load().hisq_batch_create(ctypes.byref(h), len(dims_list), arr, prec_mask, _stream_handle(stream)),
           "hisq_batch_create")
    return h


def hisq_batch_destroy(batch):
    _check(_load().hisq_batch_destroy(batch), "hisq_batch_destroy")


def hisq_batch_load_links(batch, lattice: int, fat, lng, flags: int = HISQ_APPLY_PHASES | HISQ_ANTIPERIODIC_T):
    fat = np.ascontiguousarray(fat, dtype=np.complex128)
    lng = np.ascontiguousarray(lng, dtype=np.complex128)
    _check(_load().hisq_batch_load_links(batch, lattice, _ptr(fat), _ptr(lng), flags), "hisq_batch_load_links")


def hisq_batch_vector_offset(batch, lattice: int) -> int:
    return int(_load().hisq_batch_vector_offset(batch, lattice))


def hisq_batch_launch_count(batch) -> int:
    return int(_load().hisq_batch_launch_count(batch))


def hisq_batch_cg(batch, x, b, masses, rel_tol: float, maxiter: int, opts=None, raise_on_error=True):
    """Returns (status, stats dict with per-lattice 'lattice_iters' and 'lattice_residual')."""
    masses = np.ascontiguousarray(masses, dtype=np.float64)
    nl = len(masses)
    iters = np.zeros(nl, np.int32)
    res = np.zeros(nl, np.float64)
    st = hisq_solver_stats()
    o = opts if opts is not None else hisq_solver_opts_default()
    rc = _load().hisq_batch_cg(batch, _ptr(x), _ptr(b), _ptr(masses), rel_tol, maxiter, ctypes.byref(o),
                               ctypes.byref(st), _ptr(iters), _ptr(res))
    d = st.as_dict()
    d["lattice_iters"] = iters.tolist()
    d["lattice_residual"] = res.tolist()
    if rc != HISQ_OK and raise_on_error:
        raise HisqError(rc, "hisq_batch_cg", hisq_last_error(), d)
    return rc, d


class Batch:
    """Owns one batch of lattices: ``Batch(dims_list)``, ``load(l, fat, lng)``, ``cg(x, b, masses)``."""

    def __init__(self, dims_list, precs=(HISQ_F64, HISQ_F32), stream=None):
        mask = 0
        for p in precs:
            mask |= HISQ_PREC_BIT(p)
        self.dims = [tuple(int(v) for v in d) for d in dims_list]
        self.h = hisq_batch_create(self.dims, mask, stream)
        self.offsets = [hisq_batch_vector_offset(self.h, l) for l in range(len(self.dims) + 1)]

    def close(self):
        if getattr(self, "h", None) is not None:
            hisq_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, lattice, fat, lng, flags=HISQ_APPLY_PHASES | HISQ_ANTIPERIODIC_T):
        hisq_batch_load_links(self.h, lattice, fat, lng, flags)

    def cg(self, x, b, masses, rel_tol=1e-10, maxiter=10000, **opts):
        return hisq_batch_cg(self.h, x, b, masses, rel_tol, maxiter, make_opts(**opts))


def hisq_ptc_create(ctx, channels: int = 8):
    h = ctypes.c_void_p()
    _check(_load().hisq_ptc_create(ctypes.byref(h), ctx, channels), "hisq_ptc_create")
    return h


def hisq_ptc_destroy(ptc):
    _check(_load().hisq_ptc_destroy(ptc), "hisq_ptc_destroy")


def hisq_ptc_set_weights(ptc, w1, w2):
    """w1: complex (C, 1, 9), w2: complex (1, C, 9) (numpy); stored as FP32 master weights."""
    a = np.ascontiguousarray(np.asarray(w1, np.complex64))
    b = np.ascontiguousarray(np.asarray(w2, np.complex64))
    _check(_load().hisq_ptc_set_weights(ptc, _ptr(a), _ptr(b)), "hisq_ptc_set_weights")


def hisq_ptc_get_weights(ptc, channels: int = 8):
    a = np.zeros((channels, 1, 9), np.complex64)
    b = np.zeros((1, channels, 9), np.complex64)
    _check(_load().hisq_ptc_get_weights(ptc, _ptr(a), _ptr(b)), "hisq_ptc_get_weights")
    return a, b


def hisq_ptc_set_tied(ptc, tied: bool):
    _check(_load().hisq_ptc_set_tied(ptc, int(tied)), "hisq_ptc_set_tied")


def hisq_ptc_bind(ptc, ctx):
    _check(_load().hisq_ptc_bind(ptc, ctx), "hisq_ptc_bind")


def hisq_ptc_apply(ptc, z, r, nvec: int = 1):
    _check(_load().hisq_ptc_apply(ptc, _ptr(z), _ptr(r), nvec), "hisq_ptc_apply")


def hisq_ptc_train_step(ptc, b, x, npairs: int, lr: float, channels: int = 8):
    """Returns (loss, g1, g2): the loss and the Wirtinger gradients before the (optional) Adam step."""
    loss = np.zeros(1, np.float32)
    g1 = np.zeros((channels, 1, 9), np.complex64)
    g2 = np.zeros((1, channels, 9), np.complex64)
    _check(_load().hisq_ptc_train_step(ptc, _ptr(b), _ptr(x), npairs, lr, _ptr(loss), _ptr(g1), _ptr(g2)),
           "hisq_ptc_train_step")
    return float(loss[0]), g1, g2


def hisq_fcg(ctx, ptc, x, b, mass: float, rel_tol: float, maxiter: int, opts=None, raise_on_error=True):
    st = hisq_solver_stats()
    o = opts if opts is not None else hisq_solver_opts_default()
    rc = _load().hisq_fcg(ctx, ptc, _ptr(x), _ptr(b), mass, rel_tol, maxiter, ctypes.byref(o), ctypes.byref(st))
    d = st.as_dict()
    if rc != HISQ_OK and raise_on_error:
        raise HisqError(rc, "hisq_fcg", hisq_last_error(), d)
    return rc, d


class Ptc:
    """The PTC preconditioner network bound to a Lattice (its FP32 fat links)."""

    def __init__(self, lattice, channels: int = 8):
        self.lattice = lattice
        self.C = channels
        self.h = hisq_ptc_create(lattice.ctx, channels)

    def close(self):
        if getattr(self, "h", None) is not None:
            hisq_ptc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, w1, w2):
        hisq_ptc_set_weights(self.h, w1, w2)

    def set_tied(self, tied=True):
        hisq_ptc_set_tied(self.h, tied)

    def bind(self, lattice):
        hisq_ptc_bind(self.h, lattice.ctx)
        self.lattice = lattice

    def get_weights(self):
        return hisq_ptc_get_weights(self.h, self.C)

    def apply(self, z, r, nvec=1):
        hisq_ptc_apply(self.h, z, r, nvec)

    def train_step(self, b, x, npairs, lr):
        return hisq_ptc_train_step(self.h, b, x, npairs, lr, self.C)

    def fcg(self, x, b, mass, rel_tol=1e-10, maxiter=10000, **opts):
        return hisq_fcg(self.lattice.ctx, self.h, x, b, mass, rel_tol, maxiter, make_opts(**opts))


# ---------------------------------------------------------------- convenience wrapper

class Lattice:
    """Owns one context: ``Lattice(dims).load(fat, lng)`` then ``dslash`` / ``cg``."""

    def __init__(self, dims, precs=(HISQ_F64, HISQ_F32, HISQ_F16, HISQ_BF16), stream=None):
        mask = 0
        for p in precs:
            mask |= HISQ_PREC_BIT(p)
        self.dims = tuple(int(v) for v in dims)
        self.half = int(np.prod(self.dims)) // 2
        self.ctx = hisq_create(self.dims, mask, stream)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            hisq_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, fat, lng, flags=HISQ_APPLY_PHASES | HISQ_ANTIPERIODIC_T):
        hisq_load_links(self.ctx, fat, lng, flags)
        return self

    def compress_long(self, naik=-1.0 / 24.0):
        """Keep the long links also as two rows (reconstructed in the kernel); reload links after."""
        hisq_set_long_compression(self.ctx, naik)
        return self

    def dslash(self, out_parity, out, in_, prec, nrhs=1):
        hisq_dslash(self.ctx, out_parity, out, in_, prec, nrhs)

    def smear(self, fat, lng, thin, coeffs, prec=HISQ_F64):
        hisq_smear(self.ctx, fat, lng, thin, coeffs, prec)

    def hisq_links(self, fat, lng, thin, level1, level2, prec=HISQ_F64):
        hisq_hisq_links(self.ctx, fat, lng, thin, level1, level2, prec)

    def apply_A(self, out, in_, mass, prec, nrhs=1, sigma=0.0):
        hisq_apply_A(self.ctx, out, in_, mass, sigma, prec, nrhs)

    def dslash_interleaved(self, out_parity, out, in_, prec, nrhs):
        hisq_dslash_interleaved(self.ctx, out_parity, out, in_, prec, nrhs)

    def apply_A_interleaved(self, out, in_, mass, prec, nrhs, sigma=0.0):
        hisq_apply_A_interleaved(self.ctx, out, in_, mass, sigma, prec, nrhs)

    def cg(self, x, b, mass, rel_tol=1e-10, maxiter=10000, nrhs=1, **opts):
        return hisq_cg(self.ctx, x, b, nrhs, mass, rel_tol, maxiter, make_opts(**opts))

    def multishift_cg(self, x, b, shifts, mass, rel_tol=1e-9, maxiter=10000, **opts):
        return hisq_multishift_cg(self.ctx, x, b, shifts, mass, rel_tol, maxiter, make_opts(**opts))

    def dslash_bytes(self, prec, nrhs=1):
        return hisq_dslash_bytes(self.ctx, prec, nrhs)
