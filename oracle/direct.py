"""ctypes binding of oracle/direct.c (the direct FP64 matvec).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The shared object is compiled on first use with the host C compiler
(``gcc -O2 -fopenmp``) into ``oracle/_build/``; ``build()`` does it eagerly.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle_direct.so")
_lock = threading.Lock()
_lib = None

# phase kinds; the numbering is the interface shared with the product's
# built-in kernels (each side defines it independently)
DFT, FIO, FIOPW, ONES, SEP = 0, 1, 2, 3, 4


def build(force=False):
    """Compile direct.c into oracle/_build/liboracle_direct.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.POINTER(ctypes.c_double)
            for name in ("oracle_direct", "oracle_direct_ld"):
                fn = getattr(lib, name)
                fn.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int64,
                               i64p, ctypes.c_int64, dp, ctypes.c_int64, dp]
                fn.restype = None
            lib.oracle_entries.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int64, i64p, ctypes.c_int64, i64p,
                                           ctypes.c_int64, dp]
            lib.oracle_expphase.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64, i64p, i64p,
                                            ctypes.c_int64, ctypes.c_int, dp]
            lib.oracle_amplitude.argtypes = [ctypes.c_int, ctypes.c_int64, i64p, i64p, ctypes.c_int64, dp]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = None
            _lib = lib
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _call(name, kind, s, amp, N, f, rows):
    lib = _load()
    f = np.asarray(f)
    vec = f.ndim == 1
    f2 = np.ascontiguousarray(f.reshape(N, -1), dtype=np.complex128)
    m = f2.shape[1]
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    g = np.zeros((rows.size, m), dtype=np.complex128)
    getattr(lib, name)(int(kind), float(s), int(amp), int(N), _ptr(rows, ctypes.c_int64),
                       rows.size, _ptr(f2.view(np.float64), ctypes.c_double), m,
                       _ptr(g.view(np.float64), ctypes.c_double))
    return g[:, 0] if vec else g


def direct(kind, N, f, rows=None, s=1.0, amp=0):
    """g[rows] = (K f)[rows] in FP64 (compensated sums, OpenMP over rows).

    ``f`` is (N,) or (N, m) complex; the result has shape (len(rows),) or
    (len(rows), m).  Definition: Sec. 4 potential + Sec. 5 discretisation.
    """
    return _call("oracle_direct", kind, s, amp, N, f, rows)


def direct_ld(kind, N, f, rows=None, s=1.0, amp=0):
    """Same definition evaluated entirely in C long double (brute force)."""
    return _call("oracle_direct_ld", kind, s, amp, N, f, rows)


def entries(kind, N, rows, cols, s=1.0, amp=0):
    """K[rows][:, cols] as a complex128 matrix."""
    lib = _load()
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.zeros((rows.size, cols.size), dtype=np.complex128)
    lib.oracle_entries(int(kind), float(s), int(amp), int(N), _ptr(rows, ctypes.c_int64), rows.size,
                       _ptr(cols, ctypes.c_int64), cols.size, _ptr(out.view(np.float64), ctypes.c_double))
    return out


def expphase(kind, N, i, j, sign=1, s=1.0):
    """exp(sign 2 pi i Phi(x_i, xi_j)) elementwise over broadcast index arrays i, j."""
    lib = _load()
    i, j = np.broadcast_arrays(np.asarray(i, dtype=np.int64), np.asarray(j, dtype=np.int64))
    shape = i.shape
    ii = np.ascontiguousarray(i.ravel()); jj = np.ascontiguousarray(j.ravel())
    out = np.zeros(ii.size, dtype=np.complex128)
    lib.oracle_expphase(int(kind), float(s), int(N), _ptr(ii, ctypes.c_int64), _ptr(jj, ctypes.c_int64),
                        ii.size, int(sign), _ptr(out.view(np.float64), ctypes.c_double))
    return out.reshape(shape)


def amplitude(amp, N, i, j):
    """alpha(x_i, xi_j) elementwise over broadcast index arrays (real)."""
    lib = _load()
    i, j = np.broadcast_arrays(np.asarray(i, dtype=np.int64), np.asarray(j, dtype=np.int64))
    shape = i.shape
    ii = np.ascontiguousarray(i.ravel()); jj = np.ascontiguousarray(j.ravel())
    out = np.zeros(ii.size, dtype=np.float64)
    lib.oracle_amplitude(int(amp), int(N), _ptr(ii, ctypes.c_int64), _ptr(jj, ctypes.c_int64), ii.size,
                         _ptr(out, ctypes.c_double))
    return out.reshape(shape)


def num_threads():
    return int(_load().oracle_num_threads())


def set_threads(n):
    """Host threads of the oracle's parallel loops for later calls from this thread."""
    _load().oracle_set_threads(int(n))
