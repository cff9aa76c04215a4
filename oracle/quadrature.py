"""Symmetric 7-point triangle quadrature of polynomial degree 5 (Radon's rule,
tabulated by Dunavant).  Used on every triangle by the EFIE fill (Sec. II:
Galerkin testing of RWG functions) and the plane-wave RHS.

Pinned by: exact integration of every monomial x^a y^b, a + b <= 5, on the
reference triangle (closed form a! b! / (a+b+2)!), and failure at degree 6.
"""
import math

import numpy as np


def dunavant7():
    """Barycentric points (7, 3) and weights (7,) summing to 1.

    Points: the centroid, and two orbits (a, a, 1-2a) with a = (6 -+ sqrt 15)/21.
    Weights: 9/40 and (155 -+ sqrt 15)/1200.
    """
    s15 = math.sqrt(15.0)
    a1 = (6.0 - s15) / 21.0
    a2 = (6.0 + s15) / 21.0
    w1 = (155.0 - s15) / 1200.0
    w2 = (155.0 + s15) / 1200.0
    pts = [(1 / 3, 1 / 3, 1 / 3)]
    wts = [9.0 / 40.0]
    for a, w in ((a1, w1), (a2, w2)):
        b = 1.0 - 2.0 * a
        pts += [(a, a, b), (a, b, a), (b, a, a)]
        wts += [w, w, w]
    return np.array(pts, dtype=np.float64), np.array(wts, dtype=np.float64)


def triangle_points(tri_verts):
    """Quadrature points (nt, 7, 3) for triangles given as (nt, 3, 3) vertices."""
    bary, _ = dunavant7()
    return np.einsum("qk,tkc->tqc", bary, tri_verts)
