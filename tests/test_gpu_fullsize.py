"""Parity at the benchmark's full size: the 2-lambda sphere (icosphere level 5,
N = 30720, leaves <= 128, ACA 1e-4, nested-dissection elimination order),
all 362 monostatic right-hand sides in one call (the launch configuration
bench.py times: tensor-core mixed chain and FP64-accurate tensor residual for
nrhs >= 32).  The oracle builds its own H-matrix and scaling (plain C entries,
spawn pool).  The GPU imports the H-matrix and either the oracle's scaling
(leaf-level sweeps; the oracle solves a sample of 6 columns) or none, when it
runs its own nested-dissection scaling with supernode sweeps, the schedule
bench.py times (every column compared).

Bars: FP64 chain <= 1e-6, mixed chain + refinement <= 1e-4 (against the
oracle's FP64 series + refinement), per sampled RHS."""
import os
import tempfile

import numpy as np
import pytest

from hm_workloads import get_workload
from tests.gpu_util import to_dev, from_dev, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full_case():
    from oracle.efie import EFIE
    from oracle.hmatrix import build_hmatrix
    from oracle.scaling import compute_scaling, nd_order
    w = get_workload("sphere_r2_L5")
    v, f = w.build_mesh()
    procs = max(1, min(16, (os.cpu_count() or 2) - 1))
    H = build_hmatrix(v, f, w.wavelength, w.leaf_max, w.aca_tol, processes=procs, use_c=True)
    S = compute_scaling(H, "A", nd_order(H.tree, list(H.near.keys())))
    th, ph, po = w.angles()
    B = EFIE(H.rwg, w.wavelength).plane_wave(th, ph, po)
    return w, H, S, B


def _load(H, S, **kw):
    import paper_2109_04129_gb300 as hp
    from oracle.export import write_blocks
    fd, path = tempfile.mkstemp(suffix=".hmps")
    os.close(fd)
    try:
        write_blocks(path, H, S)     # with the leaf centres (nested dissection)
        return hp.Solver.load(path, **kw)
    finally:
        os.unlink(path)


def test_full_size_fp64_and_mixed(full_case):
    import torch
    import paper_2109_04129_gb300 as hp
    from oracle.series import series_solve, refine_once
    w, H, S, B = full_case
    assert H.N == 30720 and B.shape[1] == 362
    cols = [0, 67, 150, 181, 250, 361]
    x2, _ = series_solve(H, S, B[:, cols], 2)
    xr = refine_once(H, S, B[:, cols], x2)
    Bd = to_dev(B)
    sol = _load(H, S)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    err64 = rel(from_dev(X)[:, cols], x2)
    assert err64.max() <= 1e-6, err64
    del sol
    solm = _load(H, S, precision=hp.HM_MIXED, refine_steps=1)
    Xm = torch.empty_like(Bd)
    solm.solve(Xm, Bd)
    st = hp._lib.hm_get_diagnostics(solm._h, None, None, B.shape[1])
    assert st in (hp.HM_OK, hp.HM_WARN_SERIES_RATIO)
    errm = rel(from_dev(Xm)[:, cols], xr)
    assert errm.max() <= 1e-4, errm
    print(f"full size: FP64 max rel err {err64.max():.2e}, mixed {errm.max():.2e}")


def test_full_size_benchmarked_schedule(full_case):
    """The schedule bench.py times, on all 362 RHS: the library orders the
    leaves by nested dissection, groups the ranks into supernodes and builds
    alpha, D^-1 and T_G itself (hm_compute_scaling on the GPU, from the
    oracle's H-matrix and leaf centres); then the FP64 chain and the mixed
    chain (tcgen05 sweeps over the supernodes, tcgen05 far field, FP64-accurate
    residual, split-K up to 2048 rows) solve every RHS, compared with the
    oracle's series and series + refinement on the same H in the same order."""
    import torch
    import paper_2109_04129_gb300 as hp
    from oracle.export import read_blocks
    from oracle.scaling import nd_order, supernode_inverse
    from oracle.series import series_solve, refine_once
    w, H, S, B = full_case
    order, groups = nd_order(H.tree, list(H.near.keys()), with_groups=True)
    assert list(S.order) == order
    sol = _load(H, None, ordering=hp.HM_ORDER_ND)
    sol.compute_scaling()
    fd, path = tempfile.mkstemp(suffix=".hmps")
    os.close(fd)
    try:
        sol.save(path)
        d = read_blocks(path)
    finally:
        os.unlink(path)
    assert d["elim"] == order and d["rows"] == S.rows and d["groups"] == groups
    sa = max(np.abs(a).max() for a in S.alpha.values())
    ea = max(np.abs(d["alpha"][k] - S.alpha[k]).max() for k in S.alpha) / sa
    assert ea < 1e-9, ea
    big = sorted(d["T"], key=lambda g: -d["T"][g].shape[0])[:3]
    for g in big:
        want = supernode_inverse(S, H.leaf_off, groups[g], groups[g + 1])
        assert np.abs(d["T"][g] - want).max() <= 1e-9 * np.abs(want).max(), g
    del d
    x2, _ = series_solve(H, S, B, 2)
    Bd = to_dev(B)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    err64 = rel(from_dev(X), x2)
    assert err64.max() <= 1e-6, err64.max()
    del sol
    xr = refine_once(H, S, B, x2)
    solm = _load(H, None, ordering=hp.HM_ORDER_ND, precision=hp.HM_MIXED, refine_steps=1)
    solm.compute_scaling()
    Xm = torch.empty_like(Bd)
    solm.solve(Xm, Bd)
    errm = rel(from_dev(Xm), xr)
    assert errm.max() <= 1e-4, errm.max()
    print(f"benchmarked schedule, 362 RHS: FP64 max rel err {err64.max():.2e}, "
          f"mixed {errm.max():.2e}")


def test_full_size_native_build_properties(full_case):
    """Native build of the same sphere: tree identical to the oracle's, and
    the scaling identity D^-1 R^T Z_N R v = v (Eq. 23) on random panels."""
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B = full_case
    v, f = w.build_mesh()
    sol = hp.Solver.build(v, f, leaf_max=w.leaf_max, aca_tol=w.aca_tol,
                          ordering=hp.HM_ORDER_ND)
    perm, off = sol.tree()
    assert np.array_equal(perm, H.perm) and np.array_equal(off, H.leaf_off)
    sol.compute_scaling()
    st = sol.stats()
    assert st["alpha_entries"] == S.entries(H.leaf_off)[0]
    rng = np.random.default_rng(9)
    x = rng.standard_normal((H.N, 40)) + 1j * rng.standard_normal((H.N, 40))
    a = torch.empty((40, H.N), dtype=torch.complex128, device="cuda")
    b = torch.empty_like(a)
    sol.apply("R", a, to_dev(x))
    sol.apply("NEAR", b, a)
    sol.apply("RT", a, b)
    sol.apply("DINV", b, a)
    assert rel(from_dev(b), x).max() < 1e-9
