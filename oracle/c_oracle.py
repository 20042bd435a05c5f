"""ctypes access to the plain C oracle (``oracle/c/plq_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline leg may use it.  ``build()`` compiles the C file with gcc and OpenMP;
the other functions take canonical-layout complex128 NumPy arrays (see the
``synthetic`` module) and return NumPy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "c", "plq_oracle.c")
LIB = os.path.join(_HERE, "c", "libplq_oracle.so")
_lib = None


def build(force=False):
    """Compile the C oracle into a shared library next to its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        dp = ctypes.c_void_p
        L.plq_oracle_hopping.argtypes = [dp, ctypes.c_int, dp, dp, dp, ctypes.c_int]
        L.plq_oracle_wilson.argtypes = [dp, ctypes.c_int, ctypes.c_double, dp, dp, dp, ctypes.c_int]
        L.plq_oracle_hopping_sites.argtypes = [dp, ctypes.c_int, dp, dp, dp, ctypes.c_long, dp, ctypes.c_int]
        L.plq_oracle_threads.argtypes = [ctypes.c_int]
        L.plq_oracle_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dims_of(phi):
    T, Lz, Ly, Lx = phi.shape[:4]
    return np.array([T, Lx, Ly, Lz], dtype=np.int32)


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.ctypes.data


def threads(nthreads=0):
    """OpenMP threads the oracle runs with (``nthreads <= 0``: the default)."""
    return lib().plq_oracle_threads(int(nthreads))


def hopping(U, phi, t_bc=-1, nthreads=0):
    """psi = H phi (Eq. (1)) over the whole lattice."""
    dims = _dims_of(phi)
    U, pu = _c(U)
    phi, pp = _c(phi)
    out = np.empty_like(phi)
    lib().plq_oracle_hopping(dims.ctypes.data, int(t_bc), pu, pp, out.ctypes.data, int(nthreads))
    return out


def wilson(U, phi, kappa, t_bc=-1, nthreads=0):
    """psi = M phi = phi - kappa H phi over the whole lattice."""
    dims = _dims_of(phi)
    U, pu = _c(U)
    phi, pp = _c(phi)
    out = np.empty_like(phi)
    lib().plq_oracle_wilson(dims.ctypes.data, int(t_bc), float(kappa), pu, pp, out.ctypes.data, int(nthreads))
    return out


def hopping_sites(U, phi, sites, t_bc=-1, nthreads=0):
    """(H phi) at the given lexicographic sites, shape (len(sites), 4, 3)."""
    dims = _dims_of(phi)
    U, pu = _c(U)
    phi, pp = _c(phi)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    lib().plq_oracle_hopping_sites(dims.ctypes.data, int(t_bc), pu, pp, sites.ctypes.data, len(sites),
                                   out.ctypes.data, int(nthreads))
    return out
