"""Leaves of up to 256 unknowns (leaf cap 256, as the 10 lambda sphere and
part of the scatterer batch use): the library cuts every task of more than
128 output rows into row slices so the tensor-core engine (MMA N <= 256 real
columns) takes the whole launch.  Checked on the 1 lambda sphere (icosphere
level 4, N = 7680, leaves <= 256) against the oracle, with the library's own
nested-dissection scaling: FP64 solve <= 1e-6, operators of the mixed chain
<= 2e-5, mixed chain + refinement <= 1e-4."""
import os

import numpy as np
import pytest

import hm_workloads as hw
from oracle.efie import EFIE
from oracle.hmatrix import build_hmatrix
from oracle.scaling import apply_R, apply_Rt, compute_scaling, nd_order
from oracle.series import refine_once, series_solve
from tests.gpu_util import from_dev, load_case, rand_panel, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wide():
    v, f = hw.icosphere(4, 1.0)
    procs = max(1, min(8, (os.cpu_count() or 2) - 1))
    H = build_hmatrix(v, f, 1.0, 256, 1e-4, processes=procs, use_c=True)
    m = np.diff(H.leaf_off)
    assert m.max() > 128 and len(H.far) > 0
    S = compute_scaling(H, "A", nd_order(H.tree, list(H.near.keys())))
    th = np.radians(np.linspace(0.0, 180.0, 40))
    B = EFIE(H.rwg, 1.0).plane_wave(th, np.zeros(40), np.arange(40) % 2)
    return H, S, B


def test_wide_leaves_fp64_and_mixed(wide):
    import torch
    import paper_2109_04129_gb300 as hp
    H, S, B = wide
    Bd = to_dev(B)
    x2, _ = series_solve(H, S, B, 2)
    sol = load_case(H, None, ordering=hp.HM_ORDER_ND)
    sol.compute_scaling()
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    assert rel(from_dev(X), x2).max() <= 1e-6
    mix = load_case(H, None, ordering=hp.HM_ORDER_ND, precision=hp.HM_MIXED, refine_steps=1)
    mix.compute_scaling()
    x = rand_panel(H.N, 40, 8)
    Xr = to_dev(x)
    Y = torch.empty_like(Xr)
    xp = x[H.perm]
    for op, fn in (("RT", lambda v: apply_Rt(S, H.leaf_off, v)),
                   ("R", lambda v: apply_R(S, H.leaf_off, v)),
                   ("FAR", H.far_apply)):
        mix.apply(op, Y, Xr)
        want = np.empty_like(xp)
        want[H.perm] = fn(xp)
        assert rel(from_dev(Y), want).max() <= 2e-5, op
    Xm = torch.empty_like(Bd)
    mix.solve(Xm, Bd)
    assert rel(from_dev(Xm), refine_once(H, S, B, x2)).max() <= 1e-4
