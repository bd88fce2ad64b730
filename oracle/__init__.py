"""ORACLE -- test infrastructure only.

Plain FP64 CPU implementation of what the HISQ even/odd hot path computes: link folding
(staggered phases, antiperiodic time), the Dslash halves D_eo / D_oe, A = 4m^2 - D_eo D_oe,
CG and multi-shift CG. Only tests/, the package smoke check and the CPU-baseline leg of
bench.py may import this module. The CUDA library shares no code with it.

Each function cites the passage it follows:
  * Dslash: the operator the paper's performance section benchmarks, the stencil that
    dominates the CG's cost (Sec. 3); HISQ action
    (Sec. 1, Sec. 2). The paper writes no formula, so the textbook staggered operator with
    fat one-hop and Naik three-hop long links is used (the readings are listed in oracle.c).
  * CG, multi-shift CG, multi-RHS: Sec. 2 (list of modules) and Sec. 3 (CG in RHMC).

Parity pins (tests/test_oracle_*.py): free-field closed-form spectrum, point-source probe on
a non-cubic lattice, gauge covariance, anti-hermiticity, positivity of A, dense brute force
on 4^4, FFT-exact free-field solutions for CG and multi-shift CG. PTC functions live in
oracle/ptc.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

APPLY_PHASES = 1
ANTIPERIODIC_T = 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP over output sites)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i4 = ctypes.POINTER(ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_fold_links.argtypes = [i4, ctypes.c_uint, dp, dp, dp, dp]
        lib.oracle_fold_links.restype = None
        lib.oracle_dslash_full.argtypes = [i4, dp, dp, dp, dp]
        lib.oracle_dslash_full.restype = None
        lib.oracle_dslash.argtypes = [i4, dp, dp, ctypes.c_int, dp, dp]
        lib.oracle_dslash.restype = None
        lib.oracle_dslash_sites.argtypes = [i4, dp, dp, ctypes.c_int, dp, ctypes.c_int64, i64p, dp]
        lib.oracle_dslash_sites.restype = None
        lib.oracle_apply_A.argtypes = [i4, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.oracle_apply_A.restype = None
        lib.oracle_true_residual.argtypes = [i4, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.oracle_true_residual.restype = ctypes.c_double
        lib.oracle_cg.argtypes = [i4, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_double,
                                  ctypes.c_int]
        lib.oracle_cg.restype = ctypes.c_int
        lib.oracle_multishift_cg.argtypes = [i4, dp, dp, ctypes.c_double, ctypes.c_int, dp, dp, dp, dp,
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_multishift_cg.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dims(L):
    return (ctypes.c_int * 4)(*[int(v) for v in L])


def _dp(a):
    if a is None:
        return None
    assert a.dtype in (np.complex128, np.float64) and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.complex128)


def volume(L) -> int:
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def fold_links(L, fat, lng, flags: int = APPLY_PHASES | ANTIPERIODIC_T):
    """Staggered phases and antiperiodic-t signs multiplied into the links."""
    fat, lng = _c(fat), _c(lng)
    fo = np.empty_like(fat) if fat is not None else None
    lo = np.empty_like(lng) if lng is not None else None
    _load().oracle_fold_links(_dims(L), flags, _dp(fat), _dp(lng), _dp(fo), _dp(lo))
    return fo, lo


def dslash_full(L, fat, lng, vec):
    """D on the full lattice; vec shape (V, 3) in lexicographic order."""
    v = _c(vec)
    out = np.empty_like(v)
    _load().oracle_dslash_full(_dims(L), _dp(_c(fat)), _dp(_c(lng)), _dp(v), _dp(out))
    return out


def dslash(L, fat, lng, out_parity: int, vec):
    """out_parity 0: D_eo vec (vec on odd sites); 1: D_oe vec. vec shape (V/2, 3)."""
    v = _c(vec)
    out = np.empty_like(v)
    _load().oracle_dslash(_dims(L), _dp(_c(fat)), _dp(_c(lng)), int(out_parity), _dp(v), _dp(out))
    return out


def dslash_sites(L, fat, lng, out_parity: int, vec, cb_list):
    """The operator at the listed output sites only (cb numbers); returns (n, 3)."""
    v = _c(vec)
    cbs = np.ascontiguousarray(cb_list, dtype=np.int64)
    out = np.empty((len(cbs), 3), np.complex128)
    _load().oracle_dslash_sites(_dims(L), _dp(_c(fat)), _dp(_c(lng)), int(out_parity), _dp(v), len(cbs),
                                cbs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    return out


def apply_A(L, fat, lng, mass: float, vec, sigma: float = 0.0):
    """(4 m^2 + sigma) vec - D_eo D_oe vec on even sites."""
    v = _c(vec)
    out = np.empty_like(v)
    _load().oracle_apply_A(_dims(L), _dp(_c(fat)), _dp(_c(lng)), float(mass), float(sigma), _dp(v), _dp(out))
    return out


def true_residual(L, fat, lng, mass: float, b, x, sigma: float = 0.0) -> float:
    return float(_load().oracle_true_residual(_dims(L), _dp(_c(fat)), _dp(_c(lng)), float(mass), float(sigma),
                                              _dp(_c(b)), _dp(_c(x))))


def cg(L, fat, lng, mass: float, b, tol: float = 1e-10, maxiter: int = 10000, sigma: float = 0.0, x0=None):
    """Textbook CG on (A + sigma) x = b; returns (x, iterations or -1)."""
    b = _c(b)
    x = np.zeros_like(b) if x0 is None else _c(x0).copy()
    it = _load().oracle_cg(_dims(L), _dp(_c(fat)), _dp(_c(lng)), float(mass), float(sigma), _dp(b), _dp(x),
                           float(tol), int(maxiter))
    return x, int(it)


def multishift_cg(L, fat, lng, mass: float, sigmas, b, tol, maxiter: int = 10000):
    """Multi-shift CG; returns (x of shape (ns,)+b.shape, per-shift iterations, base iterations)."""
    b = _c(b)
    sig = np.ascontiguousarray(sigmas, dtype=np.float64)
    ns = len(sig)
    tols = np.ascontiguousarray(np.broadcast_to(np.asarray(tol, np.float64), (ns,)))
    x = np.zeros((ns,) + b.shape, np.complex128)
    its = (ctypes.c_int * ns)()
    base = _load().oracle_multishift_cg(_dims(L), _dp(_c(fat)), _dp(_c(lng)), float(mass), ns, _dp(sig), _dp(b),
                                        _dp(x), _dp(tols), int(maxiter), its)
    return x, [int(v) for v in its], int(base)


# ---------------------------------------------------------------- plain indexing helpers (numpy)

def coords(L, idx):
    idx = np.asarray(idx)
    x = idx % L[0]
    y = (idx // L[0]) % L[1]
    z = (idx // (L[0] * L[1])) % L[2]
    t = idx // (L[0] * L[1] * L[2])
    return x, y, z, t


def parity_sites(L, p: int):
    """Lexicographic indices of the sites of parity p, in cb order."""
    idx = np.arange(volume(L))
    x, y, z, t = coords(L, idx)
    return idx[((x + y + z + t) & 1) == p]


def to_full(L, even=None, odd=None):
    """Embed parity vectors (V/2, 3) into a full-lattice vector (V, 3)."""
    out = np.zeros((volume(L), 3), np.complex128)
    if even is not None:
        out[parity_sites(L, 0)] = even
    if odd is not None:
        out[parity_sites(L, 1)] = odd
    return out


def from_full(L, full, p: int):
    return np.ascontiguousarray(full[parity_sites(L, p)])


def rational_apply(L, fat, lng, mass: float, b, a0: float, coeffs, sigmas, tol=1e-12, maxiter: int = 10000):
    """r(A) b = a0 b + sum_k a_k (A + sigma_k)^-1 b: the rational-function use of the multi-shift CG
    in RHMC (Sec. 2: RHMC for HISQ fermions; Sec. 3: multi-shift CG). Coefficients are inputs."""
    b = _c(b)
    xs, its, _ = multishift_cg(L, fat, lng, mass, sigmas, b, tol, maxiter)
    out = a0 * b
    for a, x in zip(coeffs, xs):
        out = out + a * x
    return out
