"""Seeded synthetic inputs: gauge links and source vectors.

Shared by the CPU oracle's tests and the CUDA library's tests and benchmark. It draws
inputs only and holds none of the operator's arithmetic: staggered phases, boundary
signs and hopping terms are applied by each side on its own.

Recipe (stand-in for thermalised HotQCD gauge ensembles, which are not available):
  thin links  U = exp(i*eps*H), H = sum_a h_a lambda_a/2, h_a ~ N(0,1)
  fat links   F = U + noise*G, G complex Gaussian (Re, Im ~ N(0, 1/2))
  long links  L_mu(x) = -(1/24) U_mu(x) U_mu(x+mu) U_mu(x+2mu)
  sources     complex Gaussian entries (Re, Im ~ N(0, 1/2))
Random numbers come from Philox4x32-10, counter-based, so a slab of t-slices (or a
single link) can be generated on its own.

Array layouts (complex128):
  links    (Lt, Lz, Ly, Lx, 4, 3, 3)   mu = 0..3 = x, y, z, t
  vectors  (nvec, V/2, 3)              sites of one parity, cb = lexicographic index // 2
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libhisq_inputs.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libhisq_inputs.so with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i4 = ctypes.POINTER(ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.hin_gen_links.argtypes = [i4, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, dp, dp]
        lib.hin_gen_thin.argtypes = [i4, ctypes.c_uint64, ctypes.c_double, dp]
        lib.hin_thin_generator.argtypes = [i4, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, dp]
        lib.hin_thin_generator.restype = None
        lib.hin_gen_source.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, dp]
        lib.hin_gen_gauge_xform.argtypes = [i4, ctypes.c_uint64, ctypes.c_double, dp]
        lib.hin_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_int64, dp]
        lib.hin_uniforms.restype = None
        lib.hin_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 2 + [ctypes.POINTER(ctypes.c_uint32)]
        lib.hin_philox4x32_10.restype = None
        _lib = lib
    return _lib


def _dims(dims):
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    return d


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def philox4x32_10(counter, key):
    """One Philox4x32-10 block: four uint32 outputs for a 4-word counter and 2-word key."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*counter)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib.hin_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def gen_links(dims, seed: int, eps: float = 0.3, noise: float = 0.1, t0: int = 0, nt: int | None = None,
              want_fat: bool = True, want_long: bool = True):
    """Fat and long links for t in [t0, t0+nt), shape (nt, Lz, Ly, Lx, 4, 3, 3) complex128."""
    lib = _load()
    Lx, Ly, Lz, Lt = [int(v) for v in dims]
    if nt is None:
        nt = Lt - t0
    shape = (nt, Lz, Ly, Lx, 4, 3, 3)
    fat = np.empty(shape, np.complex128) if want_fat else None
    lng = np.empty(shape, np.complex128) if want_long else None
    rc = lib.hin_gen_links(_dims(dims), seed, eps, noise, t0, nt,
                           _dp(fat.view(np.float64)) if fat is not None else None,
                           _dp(lng.view(np.float64)) if lng is not None else None)
    if rc != 0:
        raise ValueError("bad lattice arguments")
    return fat, lng


def gen_thin(dims, seed: int, eps: float = 0.3):
    lib = _load()
    Lx, Ly, Lz, Lt = [int(v) for v in dims]
    out = np.empty((Lt, Lz, Ly, Lx, 4, 3, 3), np.complex128)
    lib.hin_gen_thin(_dims(dims), seed, eps, _dp(out.view(np.float64)))
    return out


def thin_generator(dims, seed: int, site: int, mu: int):
    """Hermitian traceless H with thin link = exp(i*eps*H)."""
    lib = _load()
    out = np.empty((3, 3), np.complex128)
    lib.hin_thin_generator(_dims(dims), seed, site, mu, _dp(out.view(np.float64)))
    return out


def gen_source(seed: int, n_sites: int, nvec: int = 1):
    """nvec complex Gaussian vectors on one parity, shape (nvec, n_sites, 3)."""
    lib = _load()
    out = np.empty((nvec, n_sites, 3), np.complex128)
    lib.hin_gen_source(seed, n_sites, nvec, _dp(out.view(np.float64)))
    return out


def gen_gauge_xform(dims, seed: int, a: float = 1.0):
    """A random SU(3) matrix per site (lexicographic order), shape (V, 3, 3)."""
    lib = _load()
    V = int(np.prod([int(v) for v in dims]))
    out = np.empty((V, 3, 3), np.complex128)
    lib.hin_gen_gauge_xform(_dims(dims), seed, a, _dp(out.view(np.float64)))
    return out


def uniforms(seed: int, n: int):
    lib = _load()
    out = np.empty(n, np.float64)
    lib.hin_uniforms(seed, n, _dp(out))
    return out


def lattice_mix_64(master_seed: int = 3000):
    """The uneven batch: 64 lattices mixed 32/19/13 across 16^4, 24^3x8, 32^3x8.

    Per lattice: gauge seed, eps ~ U(0.2, 0.4), mass log-uniform in [0.005, 0.1], source seed.
    """
    shapes = [(16, 16, 16, 16)] * 32 + [(24, 24, 24, 8)] * 19 + [(32, 32, 32, 8)] * 13
    u = uniforms(master_seed, 2 * len(shapes))
    out = []
    for i, d in enumerate(shapes):
        eps = 0.2 + 0.2 * u[2 * i]
        mass = float(np.exp(np.log(0.005) + (np.log(0.1) - np.log(0.005)) * u[2 * i + 1]))
        out.append({"dims": d, "gauge_seed": master_seed + 1 + i, "source_seed": master_seed + 101 + i,
                    "eps": float(eps), "mass": mass})
    return out
