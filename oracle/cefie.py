"""ctypes wrapper of oracle/cefie.c (the oracle's plain-C EFIE entry used for
ACA rows and columns and block fills of large meshes).  Test infrastructure.

Pinned by: entry-by-entry agreement with the NumPy evaluator of oracle.efie
(relative 1e-12) on self, touching and separated pairs."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cefie.c")
_LIB = None


def lib_path():
    import platform
    return os.path.join(_HERE, f"_cefie_{platform.machine()}.so")


def build():
    out = lib_path()
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-ffp-contract=off",
                               "-o", out, _SRC, "-lm"])
    return out


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build())
        d, q = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)
        _LIB.efie_block_c.argtypes = [d, q, d, d, q, q, q, q, d, d, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_longlong, q, ctypes.c_longlong,
                                      q, d]
        _LIB.efie_block_c.restype = None
    return _LIB


class CBlock:
    """Z[rows][cols] from the C entry; arrays kept contiguous for the calls."""

    def __init__(self, efie):
        r = efie.rwg
        self.arrs = [np.ascontiguousarray(x) for x in (
            r.verts.astype(np.float64), r.tris.astype(np.int64), efie.Q.astype(np.float64),
            r.area.astype(np.float64), r.tri_p.astype(np.int64), r.tri_m.astype(np.int64),
            r.free_p.astype(np.int64), r.free_m.astype(np.int64), r.length.astype(np.float64),
            efie.w.astype(np.float64))]
        self.k = efie.k
        self.eta = efie.eta
        self.lib = _lib()

    def __call__(self, rows, cols):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        out = np.empty((len(rows), len(cols)), np.complex128)
        d = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        q = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
        V, T, Q, A, tp, tm, fp, fm, ln, w = self.arrs
        self.lib.efie_block_c(d(V), q(T), d(Q), d(A), q(tp), q(tm), q(fp), q(fm), d(ln), d(w),
                              self.k, self.eta, len(rows), q(rows), len(cols), q(cols),
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out
