"""Degenerate and unusual H-matrices through the GPU chain, against the oracle.

* One leaf (leaf cap above N): Z_F = 0, no scaling coefficients, and the
  series is exact: x = D^-1 b = Z^-1 b (Sec. III-B, Eq. 32 with U = 0).
  Native build and imported oracle blocks, FP64 and mixed, 1 and 40 RHS.
* Far blocks stored dense and of rank zero (a block the ACA finds to vanish):
  the far product of Eq. 11/13 over such blocks, in every engine."""
import copy

import numpy as np
import pytest

import hm_workloads as hw
from oracle.efie import EFIE
from oracle.hmatrix import build_hmatrix
from oracle.scaling import compute_scaling
from oracle.series import refine_once, series_solve
from tests.gpu_util import from_dev, load_case, rand_panel, rel, to_dev
from tests.oracle_cases import case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def one_leaf():
    v, f = hw.icosphere(2, 0.25)
    H = build_hmatrix(v, f, 1.0, 10 ** 6, 1e-4)
    assert H.n_leaves == 1 and H.far == []
    S = compute_scaling(H, "A")
    th = np.radians(np.linspace(0.0, 180.0, 40))
    B = EFIE(H.rwg, 1.0).plane_wave(th, np.zeros(40), np.arange(40) % 2)
    xl = np.linalg.solve(H.to_dense(), B[H.perm])
    X_lu = np.empty_like(xl)
    X_lu[H.perm] = xl
    return v, f, H, S, B, X_lu


@pytest.mark.parametrize("nrhs", [1, 40])
def test_one_leaf_imported(one_leaf, nrhs):
    import torch
    import paper_2109_04129_gb300 as hp
    v, f, H, S, B, X_lu = one_leaf
    Bd = to_dev(B[:, :nrhs])
    sol = load_case(H, S)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    assert rel(from_dev(X), X_lu[:, :nrhs]).max() <= 1e-9
    r, _ = sol.diagnostics(nrhs)
    assert np.all(r == 0.0)                      # it_1 = D^-1 R^T Z_F R b_o = 0
    mix = load_case(H, S, precision=hp.HM_MIXED, refine_steps=1)
    Xm = torch.empty_like(Bd)
    mix.solve(Xm, Bd)
    x2, _ = series_solve(H, S, B[:, :nrhs], 2)
    want = refine_once(H, S, B[:, :nrhs], x2)
    assert rel(from_dev(Xm), want).max() <= 1e-4
    # no far field: every far product is zero
    Y = torch.full_like(Bd, float("nan"))
    sol.apply("FAR", Y, Bd)
    assert torch.count_nonzero(Y).item() == 0
    Y.fill_(float("nan"))
    sol.apply_far_noalloc(Y, Bd)
    torch.cuda.synchronize()
    assert torch.count_nonzero(Y).item() == 0


def test_one_leaf_native_build(one_leaf):
    import torch
    import paper_2109_04129_gb300 as hp
    v, f, H, S, B, X_lu = one_leaf
    for prec in (hp.HM_FP64, hp.HM_MIXED):
        sol = hp.Solver.build(v, f, leaf_max=10 ** 6, ordering=hp.HM_ORDER_ND, precision=prec,
                              refine_steps=1 if prec == hp.HM_MIXED else 0)
        perm, off = sol.tree()
        assert len(off) == 2 and np.array_equal(perm, H.perm)
        sol.compute_scaling()
        st = sol.stats()
        assert st["far_blocks"] == 0 and st["alpha_entries"] == 0
        th = np.radians(np.linspace(0.0, 180.0, 40))
        Bd = torch.empty((40, sol.N), dtype=torch.complex128, device="cuda")
        sol.plane_wave(Bd, th, np.zeros(40), np.arange(40) % 2)
        X = torch.empty_like(Bd)
        sol.solve(X, Bd)
        # the native near block equals the oracle's to ~1e-10: so does Z^-1 b
        bar = 1e-6 if prec == hp.HM_FP64 else 1e-4
        assert rel(from_dev(X), X_lu).max() <= bar, prec


def _odd_far_blocks():
    """plate_2l with one low-rank far block stored dense (its U V^T) and one
    set to rank zero; the scaling is unchanged (it reads the near field only)."""
    w, H, S, B = case("plate_2l")
    H2 = copy.copy(H)
    far = list(H.far)
    lr = [q for q, b in enumerate(far) if b[0] == "lr" and b[5].shape[1] > 0]
    a, z = lr[0], lr[len(lr) // 2]
    kind, r0, m, c0, n, P, Q = far[a]
    far[a] = ("dense", r0, m, c0, n, P @ Q.T, None)
    kind, r0, m, c0, n, P, Q = far[z]
    far[z] = ("lr", r0, m, c0, n, P[:, :0].copy(), Q[:, :0].copy())
    H2.far = far
    return w, H2, S


@pytest.mark.parametrize("nrhs", [1, 7, 40])
def test_dense_and_rank_zero_far_blocks(nrhs):
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S = _odd_far_blocks()
    x = rand_panel(H.N, nrhs, 77 + nrhs)
    X = to_dev(x)
    Y = torch.empty_like(X)
    want_far = np.empty_like(x)
    want_far[H.perm] = H.far_apply(x[H.perm])
    want_z = np.empty_like(x)
    want_z[H.perm] = H.apply(x[H.perm])
    sol = load_case(H, S)
    sol.apply("FAR", Y, X)
    assert rel(from_dev(Y), want_far).max() <= 1e-12
    sol.apply("Z", Y, X)
    assert rel(from_dev(Y), want_z).max() <= 1e-12
    Y.zero_()
    sol.apply_far_noalloc(Y, X)
    torch.cuda.synchronize()
    assert rel(from_dev(Y), want_far).max() <= 1e-12
    x2, _ = series_solve(H, S, x, 2)
    Xs = torch.empty_like(X)
    sol.solve(Xs, X)
    assert rel(from_dev(Xs), x2).max() <= 1e-6
    mix = load_case(H, S, precision=hp.HM_MIXED, refine_steps=1)
    mix.apply("FAR", Y, X)
    assert rel(from_dev(Y), want_far).max() <= 2e-5
    mix.apply("Z", Y, X)                         # FP64-accurate residual products
    assert rel(from_dev(Y), want_z).max() <= 1e-12
    mix.solve(Xs, X)
    assert rel(from_dev(Xs), refine_once(H, S, x, x2)).max() <= 1e-4
