"""Power-series solution of the scaled system (Sec. III-A/B, Eq. 30-45).

  b~  = R^T b                       (Eq. 25)
  b_o = Z~_N^{-1} b~                (Eq. 32)   = it_0
  it_n = U it_{n-1},  U = Z~_N^{-1} R^T Z_F R   (Eq. 31, applied, never formed)
  x~  = it_0 - it_1 + it_2 - ...    (Eq. 35-36, 44), truncated after n_terms
  x   = R x~                        (Eq. 26)
The paper truncates after two terms ("converges in two iterations"), so
n_terms = 2 by default: x = R (b_o - U b_o).  The per-RHS ratio
||it_n|| / ||it_{n-1}|| of Eq. 45 is returned (the paper wants it below 0.1).

Mixed-precision comparator (not in the paper): one step of iterative
refinement, r = b - (Z_N + Z_F) x, x += series(r), all in FP64 here.

Pinned by: Z_F = 0 -> x = Z_N^{-1} b (reading A), one leaf -> D^{-1} b =
Z^{-1} b, many terms -> the LU solution of the assembled H-matrix when the
ratio is below one, and R^T Z_N R block diagonal (oracle.scaling).  The
adaptive term count is pinned by the same LU solution: with the ratio below
one its error follows the tolerance (tail of a geometric series).
"""
import numpy as np

from .scaling import apply_R, apply_Rt, apply_Dinv


def _norms(v):
    return np.sqrt(np.sum(np.abs(v) ** 2, axis=0))


def series_solve_perm(H, S, b, n_terms=2, term_tol=None):
    """Series on a leaf-ordered RHS; returns (x leaf order, ratios (terms-1, nrhs)).

    ``term_tol`` (adaptive term count; Sec. III-C, Eq. 44-45): after adding
    it_n (n >= 1), stop when every RHS has ||it_n|| <= term_tol ||it_0|| (the
    terms have shrunk to the tolerance), or when some RHS has ||it_n|| >=
    ||it_{n-1}|| > 0 (its ratio of Eq. 45 is at least one: later terms would
    not shrink); ``n_terms`` stays the cap."""
    off = H.leaf_off
    it = apply_Dinv(S, off, apply_Rt(S, off, b))        # it_0 = b_o
    it0 = it
    xt = it.copy()
    ratios = []
    for n in range(1, n_terms):
        z = H.far_apply(apply_R(S, off, it))
        nxt = apply_Dinv(S, off, apply_Rt(S, off, z))    # it_n = U it_{n-1}
        with np.errstate(divide="ignore", invalid="ignore"):
            ratios.append(_norms(nxt) / _norms(it))
        xt = xt + ((-1) ** n) * nxt
        prev, it = it, nxt
        if term_tol is not None:
            a0, ap, an = _norms(it0), _norms(prev), _norms(nxt)
            if np.all(an <= term_tol * a0) or np.any((an > 0) & (an >= ap)):
                break
    return apply_R(S, off, xt), np.array(ratios)


def series_solve(H, S, B, n_terms=2, term_tol=None):
    """X (original RWG order) for B (N,) or (N, nrhs) in original order."""
    B = np.asarray(B, dtype=np.complex128)
    xp, ratios = series_solve_perm(H, S, B[H.perm], n_terms, term_tol)
    X = np.empty_like(xp)
    X[H.perm] = xp
    return X, ratios


def refine_once(H, S, B, X, n_terms=2, term_tol=None):
    """One refinement step: r = B - (Z_N + Z_F) X, X + series(r)."""
    B = np.asarray(B, dtype=np.complex128)
    xp = X[H.perm]
    r = B[H.perm] - H.apply(xp)
    d, _ = series_solve_perm(H, S, r, n_terms, term_tol)
    out = np.empty_like(xp)
    out[H.perm] = xp + d
    return out


def relative_residual(H, B, X):
    B = np.asarray(B, dtype=np.complex128)
    r = B[H.perm] - H.apply(X[H.perm])
    return _norms(r) / _norms(B[H.perm])


def rel_err(A, B):
    """Per-column relative L2 error ||A - B|| / ||B|| (paper's metric, Sec. V-A)."""
    A = np.asarray(A).reshape(len(A), -1)
    B = np.asarray(B).reshape(len(B), -1)
    return _norms(A - B) / _norms(B)
