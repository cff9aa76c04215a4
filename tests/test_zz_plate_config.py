"""Parity on the 8 lambda x 8 lambda plate (80 x 80 cells of lambda/10, 12800
triangles, 19040 unknowns, leaves <= 128, ACA 1e-4; 360 monostatic RHS,
phi = 0..359 deg at theta = 60 deg): an open surface, unlike the spheres.

The oracle builds the H-matrix and the scaling (plain C entries, spawn pool,
nested-dissection order) and the GPU library imports them; all 360 RHS go
through one call of each precision (the tensor-core paths for nrhs >= 32), and
the oracle solves a sample of 5 columns.  Bars: FP64 chain <= 1e-6 against the
oracle's two-term series, mixed chain + refinement <= 1e-4 against the
oracle's series + refinement."""
import os
import tempfile

import numpy as np
import pytest

from hm_workloads import get_workload
from tests.gpu_util import to_dev, from_dev, rel

pytestmark = pytest.mark.gpu

COLS = [0, 90, 180, 270, 359]


@pytest.fixture(scope="module")
def plate_case():
    from oracle.efie import EFIE
    from oracle.hmatrix import build_hmatrix
    from oracle.scaling import compute_scaling, nd_order
    w = get_workload("plate_8l")
    v, f = w.build_mesh()
    procs = max(1, min(16, (os.cpu_count() or 2) - 1))
    H = build_hmatrix(v, f, w.wavelength, w.leaf_max, w.aca_tol, processes=procs, use_c=True)
    S = compute_scaling(H, "A", nd_order(H.tree, list(H.near.keys())))
    th, ph, po = w.angles()
    B = EFIE(H.rwg, w.wavelength).plane_wave(th, ph, po)
    return H, S, B


def _load(H, S, **kw):
    import paper_2109_04129_gb300 as hp
    from oracle.export import write_blocks
    fd, path = tempfile.mkstemp(suffix=".hmps")
    os.close(fd)
    try:
        write_blocks(path, H, S)
        return hp.Solver.load(path, **kw)
    finally:
        os.unlink(path)


def test_plate_fp64_and_mixed(plate_case):
    import torch
    import paper_2109_04129_gb300 as hp
    from oracle.series import series_solve, refine_once
    H, S, B = plate_case
    assert H.N == 19040 and B.shape[1] == 360
    x2, ratio = series_solve(H, S, B[:, COLS], 2)
    xr = refine_once(H, S, B[:, COLS], x2)
    Bd = to_dev(B)
    sol = _load(H, S)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    err64 = rel(from_dev(X)[:, COLS], x2)
    assert err64.max() <= 1e-6, err64
    ratio_gpu, _ = sol.diagnostics(B.shape[1])
    assert np.allclose(np.asarray(ratio_gpu)[COLS], ratio.ravel(), rtol=1e-6)
    del sol
    solm = _load(H, S, precision=hp.HM_MIXED, refine_steps=1)
    Xm = torch.empty_like(Bd)
    solm.solve(Xm, Bd)
    errm = rel(from_dev(Xm)[:, COLS], xr)
    assert errm.max() <= 1e-4, errm
    print(f"plate: FP64 max rel err {err64.max():.2e}, mixed {errm.max():.2e}, "
          f"ratio {ratio.max():.3f}")
