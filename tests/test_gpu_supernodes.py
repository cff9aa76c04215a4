"""The schedule bench.py times, against the oracle, on a small case.

bench.py builds the H-matrix on the GPU, then lets hm_compute_scaling order
the leaves by nested dissection and group the ranks into supernodes whose
sweeps apply T_G = (I - A_G^T)^-1 as one dense product (Eq. 25-26 per group).
Here the library gets the oracle's H-matrix with its leaf cell centres and
runs that same scaling itself, so every step of the benchmarked chain meets
the oracle: the elimination order and groups (exact), alpha, D^-1 and T_G
(<= 1e-9), the operators and the solves (FP64 <= 1e-6, mixed chain + one
refinement <= 1e-4 against the oracle's FP64 series + refinement), with and
without the tensor-core engines (nrhs 40 and 7).  The oracle's own alpha,
D^-1 and T_G imported through the block file run the same schedule (P1)."""
import numpy as np
import pytest

from oracle.efie import EFIE
from oracle.export import read_blocks
from oracle.scaling import (apply_R, apply_Rt, apply_Dinv, compute_scaling, nd_order,
                            supernode_inverse)
from oracle.series import refine_once, series_solve
from tests.gpu_util import from_dev, load_case, rand_panel, rel, to_dev
from tests.oracle_cases import case

pytestmark = pytest.mark.gpu

NAME = "sphere_r0.5_L3"


@pytest.fixture(scope="module")
def nd_case():
    w, H, _, _ = case(NAME)
    order, groups = nd_order(H.tree, list(H.near.keys()), with_groups=True)
    S = compute_scaling(H, "A", order)
    th = np.radians(np.linspace(0.0, 180.0, 40))
    B = EFIE(H.rwg, w.wavelength).plane_wave(th, np.zeros(40), np.arange(40) % 2)
    return w, H, S, B, order, groups


def _gpu_nd(H, tmp_path, **kw):
    import paper_2109_04129_gb300 as hp
    sol = load_case(H, None, ordering=hp.HM_ORDER_ND, **kw)
    sol.compute_scaling()
    p = str(tmp_path / "nd.hmps")
    sol.save(p)
    return sol, read_blocks(p)


def test_gpu_nd_scaling_groups_and_supernodes(nd_case, tmp_path):
    w, H, S, B, order, groups = nd_case
    sol, d = _gpu_nd(H, tmp_path)
    assert d["elim"] == order
    assert d["rows"] == S.rows
    assert d["groups"] == groups
    sa = max(np.abs(a).max() for a in S.alpha.values())
    ea = max(np.abs(d["alpha"][k] - S.alpha[k]).max() for k in S.alpha) / sa
    sd = max(np.abs(a).max() for a in S.Dinv)
    ed = max(np.abs(a - b).max() for a, b in zip(d["Dinv"], S.Dinv)) / sd
    assert ea < 1e-9 and ed < 1e-9, (ea, ed)
    multi = [g for g in range(len(groups) - 1) if groups[g + 1] - groups[g] > 1]
    assert sorted(d["T"]) == multi and len(multi) >= 3
    for g in multi:
        want = supernode_inverse(S, H.leaf_off, groups[g], groups[g + 1])
        err = np.abs(d["T"][g] - want).max() / np.abs(want).max()
        assert err < 1e-9, (g, err)
    # the group schedule is in use: fewer launch phases than leaf levels
    st = sol.stats()
    assert st["fwd_levels"] <= 2 * len(set(groups))


@pytest.mark.parametrize("nrhs", [1, 7, 40])
def test_gpu_nd_operators_fp64(nd_case, tmp_path, nrhs):
    w, H, S, B, order, groups = nd_case
    import torch
    sol, _ = _gpu_nd(H, tmp_path)
    x = rand_panel(H.N, nrhs, 20 + nrhs)
    X = to_dev(x)
    Y = torch.empty_like(X)
    xp = x[H.perm]
    for op, fn in (("RT", lambda v: apply_Rt(S, H.leaf_off, v)),
                   ("R", lambda v: apply_R(S, H.leaf_off, v)),
                   ("DINV", lambda v: apply_Dinv(S, H.leaf_off, v))):
        sol.apply(op, Y, X)
        want = np.empty_like(xp)
        want[H.perm] = fn(xp)
        err = rel(from_dev(Y), want)
        assert err.max() < 1e-8, (op, err.max())


@pytest.mark.parametrize("nrhs", [1, 7, 40])
def test_gpu_nd_solve_fp64(nd_case, tmp_path, nrhs):
    import torch
    w, H, S, B, order, groups = nd_case
    sol, _ = _gpu_nd(H, tmp_path)
    Bc = B[:, :nrhs]
    want, ratios = series_solve(H, S, Bc, 2)
    Bd = to_dev(Bc)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    err = rel(from_dev(X), want)
    assert err.max() <= 1e-6, err.max()
    r, _ = sol.diagnostics(nrhs)
    assert np.allclose(r, ratios[0], rtol=1e-7)


@pytest.mark.parametrize("nrhs", [7, 40])
def test_gpu_nd_solve_mixed(nd_case, tmp_path, nrhs):
    """Mixed chain + one FP64 refinement in the benchmarked configuration
    (nrhs >= 32: tcgen05 sweeps over the supernodes, FP64-accurate residual);
    nrhs = 7 runs the CUDA-core kernels of the same schedule."""
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B, order, groups = nd_case
    sol, _ = _gpu_nd(H, tmp_path, precision=hp.HM_MIXED, refine_steps=1)
    Bc = B[:, :nrhs]
    x2, _ = series_solve(H, S, Bc, 2)
    want = refine_once(H, S, Bc, x2)
    Bd = to_dev(Bc)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    err = rel(from_dev(X), want)
    assert err.max() <= 1e-4, err.max()


def test_imported_supernodes_run_the_same_schedule(nd_case, tmp_path):
    """The oracle's alpha, D^-1 and T_G imported: the library runs the group
    schedule on them (FP64 <= 1e-6, mixed <= 1e-4), and a save / load round
    trip keeps the groups and gives a bit-identical solve."""
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B, order, groups = nd_case
    sol = load_case(H, S, groups=groups)
    st = sol.stats()
    Bd = to_dev(B)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    x2, _ = series_solve(H, S, B, 2)
    assert rel(from_dev(X), x2).max() <= 1e-6
    p = str(tmp_path / "rt.hmps")
    sol.save(p)
    d = read_blocks(p)
    assert d["groups"] == groups
    sol2 = hp.Solver.load(p)
    assert sol2.stats()["fwd_levels"] == st["fwd_levels"]
    X2 = torch.empty_like(Bd)
    sol2.solve(X2, Bd)
    assert torch.equal(X, X2)
    mix = load_case(H, S, groups=groups, precision=hp.HM_MIXED, refine_steps=1)
    Xm = torch.empty_like(Bd)
    mix.solve(Xm, Bd)
    want = refine_once(H, S, B, x2)
    assert rel(from_dev(Xm), want).max() <= 1e-4
