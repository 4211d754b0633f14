"""ctypes wrapper of reach_oracle_c.c: the oracle's Jacobi and BiCGStab loops in plain C.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: the CPU baseline of ``bench.py`` times
these loops on the host cores, and the CPU tests check them against the numpy oracle and
the closed forms.  ``build()`` compiles the C file with gcc (OpenMP when the compiler has
it, else single-threaded) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "reach_oracle_c.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libreach_oracle_c.so")
_LIB = None


def build(force: bool = False) -> str:
    """Compile the C oracle; OpenMP if gcc supports it, otherwise a serial build."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no C compiler for the C oracle")
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + ".tmp"
    base = [cc, "-O2", "-std=c11", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:2] + ["-fopenmp"] + base[2:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"C oracle build failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _LIB
    if _LIB is None:
        so = C.CDLL(build())
        P, I64, D = C.c_void_p, C.c_int64, C.c_double
        so.oracle_c_openmp.restype = C.c_int
        so.oracle_c_threads.restype = C.c_int
        so.oracle_c_threads.argtypes = [C.c_int]
        so.oracle_c_jacobi.restype = I64
        so.oracle_c_jacobi.argtypes = [I64, P, P, P, P, D, I64, P, P, C.POINTER(D), C.POINTER(C.c_int)]
        so.oracle_c_bicgstab.restype = C.c_int
        so.oracle_c_bicgstab.argtypes = [I64, P, P, P, P, D, I64, P, P, C.POINTER(I64), C.POINTER(D)]
        _LIB = so
    return _LIB


def set_threads(want: int = 0) -> int:
    """Threads the loops use (0 = every host core); returns the count in effect."""
    return int(lib().oracle_c_threads(int(want)))


def _csr(m):
    m = sp.csr_matrix(m)
    m.sort_indices()
    return (np.ascontiguousarray(m.indptr, np.int64), np.ascontiguousarray(m.indices, np.int32),
            np.ascontiguousarray(m.data, np.float64))


def jacobi(m, b, eps, max_iter, x0=None):
    """Jacobi for M x = b (§3.1); returns (x, sweeps, last max|x - x'|, converged)."""
    rp, ci, v = _csr(m)
    n = rp.size - 1
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64)
    work = np.empty(max(n, 1))
    d, ok = C.c_double(0.0), C.c_int(0)
    it = lib().oracle_c_jacobi(n, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, b.ctypes.data, float(eps),
                               int(max_iter), x.ctypes.data, work.ctypes.data, C.byref(d), C.byref(ok))
    if it < 0:
        raise MemoryError("C oracle: allocation failed")
    return x, int(it), d.value, bool(ok.value)


def bicgstab(m, b, eps, max_iter, x0=None):
    """BiCGStab for M x = b (§3.2); returns (x, iterations, last residual max, status)
    with status 0 = converged, 1 = max_iter reached, 2 = breakdown after a restart."""
    rp, ci, v = _csr(m)
    n = rp.size - 1
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64)
    work = np.empty(max(6 * n, 1))
    it, res = C.c_int64(0), C.c_double(0.0)
    st = lib().oracle_c_bicgstab(n, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, b.ctypes.data, float(eps),
                                 int(max_iter), x.ctypes.data, work.ctypes.data, C.byref(it), C.byref(res))
    return x, int(it.value), res.value, int(st)
