"""Cached oracle builds shared by the CPU and GPU test modules."""
import functools

import numpy as np

from hm_workloads import get_workload, icosphere, plate
from oracle.efie import EFIE
from oracle.hmatrix import build_hmatrix
from oracle.scaling import compute_scaling


@functools.lru_cache(maxsize=None)
def case(name, leaf_max=None, reading="A", processes=1):
    """(workload, H, S, B) for a named workload; B holds its plane-wave RHS."""
    w = get_workload(name)
    v, f = w.build_mesh()
    lm = leaf_max or w.leaf_max
    H = build_hmatrix(v, f, w.wavelength, lm, w.aca_tol, processes=processes)
    S = compute_scaling(H, reading)
    th, ph, po = w.angles()
    B = EFIE(H.rwg, w.wavelength).plane_wave(th, ph, po)
    return w, H, S, B


@functools.lru_cache(maxsize=None)
def plate_converging():
    """2 lambda plate, leaf cap 128: rho(Z_N^-1 Z_F) ~ 0.38 < 1."""
    v, f = plate(2.0, 20)
    H = build_hmatrix(v, f, 1.0, 128, 1e-4)
    S = compute_scaling(H, "A")
    B = EFIE(H.rwg, 1.0).plane_wave(np.radians([0.0, 60.0]), np.radians([0.0, 30.0]), [0, 1])
    return H, S, B


@functools.lru_cache(maxsize=None)
def dense_sphere_c1():
    """Dense symmetric Z and the x-polarised theta=0 RHS of the 0.5 lambda sphere."""
    v, f = icosphere(3, 0.5)
    from oracle.rwg import build_rwg
    r = build_rwg(v, f)
    E = EFIE(r, 1.0)
    return r, E, E.dense(), E.plane_wave([0.0], [0.0], [0])
