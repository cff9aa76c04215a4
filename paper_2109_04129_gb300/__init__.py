"""Python binding of the GB300 power-series H-matrix EFIE solver (libhmps.so).

Argument marshalling only: every step of the method runs in the native
library behind the C ABI of include/hm.h.  Device buffers are torch tensors
(complex128, shape (nrhs, N) in memory = column-major N x nrhs); the CUDA
stream is torch's current stream.  If the native library is missing this
module raises ImportError: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhmps.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"native library not built: {LIB_PATH} "
                      "(run __graft_entry__.build() or paper_2109_04129_gb300/build_native.py)")
_lib = ctypes.CDLL(LIB_PATH)

HM_OK, HM_ERR_INVALID, HM_ERR_CUDA, HM_ERR_OOM, HM_ERR_SINGULAR = 0, 1, 2, 3, 4
HM_ERR_TIMEOUT, HM_ERR_STATE, HM_ERR_IO, HM_WARN_SERIES_RATIO = 5, 6, 7, 100
HM_FP64, HM_MIXED = 0, 1
HM_MIXED_BF16 = HM_MIXED          # the mixed mode by its operand type (bf16 slice products)
HM_ORDER_DFS, HM_ORDER_ND = 0, 1
HM_FILL_FULL, HM_FILL_NEAR = 0, 1
OPS = {"RT": 0, "R": 1, "DINV": 2, "FAR": 3, "NEAR": 4, "Z": 5}
STATS = ("N", "leaves", "near_blocks", "far_blocks", "alpha_entries", "d_entries",
         "near_entries", "far_entries", "max_rank", "fwd_levels", "bwd_levels", "device_bytes",
         "kernel_launches", "terms_used", "tuned_phases")

# every symbol include/hm.h declares
SYMBOLS = ("hm_default_params", "hm_build", "hm_import", "hm_save", "hm_compute_scaling",
           "hm_power_series_solve", "hm_power_series_solve_host", "hm_apply",
           "hm_plane_wave_rhs", "hm_set_stream", "hm_num_unknowns", "hm_get_diagnostics",
           "hm_get_stats", "hm_get_tree", "hm_destroy", "hm_status_string",
           "hm_profile_enable", "hm_get_profile", "hm_apply_far_noalloc", "hm_solve_grouped")
PROF_CATEGORIES = ("rt_sweep", "r_sweep", "sweep_finalize", "dinv", "far_stage1",
                   "far_stage2", "near", "misc", "mixed_sweep", "mixed_far", "conversion")


class hm_params(ctypes.Structure):
    _fields_ = [("wavelength", ctypes.c_double), ("leaf_max", ctypes.c_int),
                ("ordering", ctypes.c_int), ("aca_tol", ctypes.c_double),
                ("fill", ctypes.c_int), ("n_terms", ctypes.c_int),
                ("precision", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("spin_limit", ctypes.c_longlong), ("tensor_cores", ctypes.c_int),
                ("fp64_emulation", ctypes.c_int), ("term_tol", ctypes.c_double),
                ("autotune", ctypes.c_int), ("tc_split_max", ctypes.c_int),
                ("eta", ctypes.c_double), ("freq_hz", ctypes.c_double),
                ("reserved", ctypes.c_int * 2)]


_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_P = ctypes.POINTER
_lib.hm_default_params.argtypes = [_P(hm_params)]
_lib.hm_default_params.restype = None
_lib.hm_status_string.argtypes = [_i]
_lib.hm_status_string.restype = ctypes.c_char_p
for name, args in {
    "hm_build": [_P(ctypes.c_double), _i, _P(ctypes.c_int), _i, _P(hm_params), _P(_vp)],
    "hm_import": [ctypes.c_char_p, _P(hm_params), _P(_vp)],
    "hm_save": [_vp, ctypes.c_char_p],
    "hm_compute_scaling": [_vp],
    "hm_power_series_solve": [_vp, _vp, _vp, _i],
    "hm_power_series_solve_host": [_vp, _vp, _vp, _i],
    "hm_apply": [_vp, _i, _vp, _vp, _i],
    "hm_plane_wave_rhs": [_vp, _P(_d), _P(_d), _P(_i), _i, _vp],
    "hm_set_stream": [_vp, _vp],
    "hm_num_unknowns": [_vp, _P(_i)],
    "hm_get_diagnostics": [_vp, _P(_d), _P(_d), _i],
    "hm_get_stats": [_vp, _P(ctypes.c_longlong), _i],
    "hm_get_tree": [_vp, _P(ctypes.c_longlong), _P(ctypes.c_longlong)],
    "hm_destroy": [_vp],
    "hm_profile_enable": [_vp, _i],
    "hm_get_profile": [_vp, _P(_d), _i],
    "hm_apply_far_noalloc": [_vp, _vp, _vp, _i],
    "hm_solve_grouped": [_P(_vp), _P(_vp), _P(_vp), _P(_i), _i],
}.items():
    fn = getattr(_lib, name)
    fn.argtypes = args
    fn.restype = ctypes.c_int


class HMError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_lib.hm_status_string(status).decode()} ({status})")


def _check(status, where, allow=(HM_OK,)):
    if status not in allow:
        raise HMError(status, where)
    return status


def default_params(**kw):
    p = hm_params()
    _lib.hm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One H-matrix system on the current CUDA device."""

    def __init__(self, handle, params):
        self._h = ctypes.c_void_p(handle)
        self.params = params
        n = ctypes.c_int()
        _check(_lib.hm_num_unknowns(self._h, ctypes.byref(n)), "hm_num_unknowns")
        self.N = n.value

    # ----------------------------------------------------------- creation
    @classmethod
    def build(cls, verts, tris, **kw):
        p = default_params(**kw)
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(_lib.hm_build(v.ctypes.data_as(_P(ctypes.c_double)), len(v),
                             t.ctypes.data_as(_P(ctypes.c_int)), len(t), ctypes.byref(p),
                             ctypes.byref(h)), "hm_build")
        return cls(h.value, p)

    @classmethod
    def load(cls, path, **kw):
        p = default_params(**kw)
        h = ctypes.c_void_p()
        _check(_lib.hm_import(os.fsencode(path), ctypes.byref(p), ctypes.byref(h)), "hm_import")
        return cls(h.value, p)

    def save(self, path):
        _check(_lib.hm_save(self._h, os.fsencode(path)), "hm_save")

    def compute_scaling(self):
        _check(_lib.hm_compute_scaling(self._h), "hm_compute_scaling")

    def close(self):
        if self._h:
            _lib.hm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- device work
    def _stream(self):
        import torch
        _lib.hm_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

    @staticmethod
    def _panel_ok(t, N):
        import torch
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("expected a contiguous complex128 CUDA tensor of shape (nrhs, N)")
        if t.dim() != 2 or t.shape[1] != N:
            raise ValueError(f"expected shape (nrhs, {N})")

    def solve(self, X, B):
        """X <- power-series solution of Z X = B; tensors (nrhs, N) complex128
        on the device (column-major N x nrhs).  Returns the status (OK or the
        series-ratio warning)."""
        self._panel_ok(X, self.N)
        self._panel_ok(B, self.N)
        self._stream()
        return _check(_lib.hm_power_series_solve(self._h, _ptr(X), _ptr(B), B.shape[0]),
                      "hm_power_series_solve", (HM_OK, HM_WARN_SERIES_RATIO))

    def solve_host(self, X, B):
        """Same solve for host numpy arrays (nrhs, N) complex128 (pinned or not)."""
        assert X.dtype == np.complex128 and B.dtype == np.complex128
        assert X.flags.c_contiguous and B.flags.c_contiguous and X.shape == B.shape
        self._stream()
        return _check(_lib.hm_power_series_solve_host(
            self._h, ctypes.c_void_p(X.ctypes.data), ctypes.c_void_p(B.ctypes.data),
            B.shape[0]), "hm_power_series_solve_host", (HM_OK, HM_WARN_SERIES_RATIO))

    def apply(self, op, Y, X):
        self._panel_ok(X, self.N)
        self._panel_ok(Y, self.N)
        self._stream()
        _check(_lib.hm_apply(self._h, OPS[op], _ptr(Y), _ptr(X), X.shape[0]), "hm_apply")

    def apply_far_noalloc(self, Y, X):
        """Y = Z_F X without any device allocation (fixed library scratch)."""
        self._panel_ok(X, self.N)
        self._panel_ok(Y, self.N)
        self._stream()
        _check(_lib.hm_apply_far_noalloc(self._h, _ptr(Y), _ptr(X), X.shape[0]),
               "hm_apply_far_noalloc")

    def plane_wave(self, B, theta, phi, pol):
        self._panel_ok(B, self.N)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        ph = np.ascontiguousarray(phi, dtype=np.float64)
        po = np.ascontiguousarray(pol, dtype=np.int32)
        self._stream()
        _check(_lib.hm_plane_wave_rhs(self._h, th.ctypes.data_as(_P(_d)),
                                      ph.ctypes.data_as(_P(_d)), po.ctypes.data_as(_P(_i)),
                                      len(th), _ptr(B)), "hm_plane_wave_rhs")

    def diagnostics(self, nrhs):
        r = np.zeros(nrhs)
        s = np.zeros(nrhs)
        _check(_lib.hm_get_diagnostics(self._h, r.ctypes.data_as(_P(_d)),
                                       s.ctypes.data_as(_P(_d)), nrhs),
               "hm_get_diagnostics", (HM_OK, HM_WARN_SERIES_RATIO))
        return r, s

    def stats(self):
        out = (ctypes.c_longlong * len(STATS))()
        _check(_lib.hm_get_stats(self._h, out, len(STATS)), "hm_get_stats")
        return dict(zip(STATS, list(out)))

    def profile_enable(self, on=True):
        _check(_lib.hm_profile_enable(self._h, 1 if on else 0), "hm_profile_enable")

    def profile(self):
        """{category: (launches, ms, algorithmic bytes, algorithmic flops)} since
        the last call."""
        n = len(PROF_CATEGORIES)
        out = np.zeros(4 * n)
        _check(_lib.hm_get_profile(self._h, out.ctypes.data_as(_P(_d)), n), "hm_get_profile")
        return {c: tuple(out[4 * i:4 * i + 4]) for i, c in enumerate(PROF_CATEGORIES)}

    def tree(self):
        st = self.stats()
        perm = np.zeros(st["N"], np.int64)
        off = np.zeros(st["leaves"] + 1, np.int64)
        _check(_lib.hm_get_tree(self._h, perm.ctypes.data_as(_P(ctypes.c_longlong)),
                                off.ctypes.data_as(_P(ctypes.c_longlong))), "hm_get_tree")
        return perm, off


def solve_grouped(solvers, Xs, Bs):
    """Grouped solve of independent problems: Xs[i] <- solve of solvers[i] for
    Bs[i] (tensors as in Solver.solve), recorded once into one CUDA graph with
    a branch per problem and replayed on torch's current stream."""
    n = len(solvers)
    if n == 0 or len(Xs) != n or len(Bs) != n:
        raise ValueError("need one X and one B per solver")
    for s, X, B in zip(solvers, Xs, Bs):
        Solver._panel_ok(X, s.N)
        Solver._panel_ok(B, s.N)
        if X.shape != B.shape:
            raise ValueError("X and B shapes differ")
    solvers[0]._stream()
    hs = (_vp * n)(*[s._h.value for s in solvers])
    xs = (_vp * n)(*[X.data_ptr() for X in Xs])
    bs = (_vp * n)(*[B.data_ptr() for B in Bs])
    nr = (_i * n)(*[B.shape[0] for B in Bs])
    return _check(_lib.hm_solve_grouped(hs, xs, bs, nr, n), "hm_solve_grouped")


def exported_symbols():
    """Names from include/hm.h that the loaded library exports."""
    return [s for s in SYMBOLS if hasattr(_lib, s)]
