"""The CFIE (Eq. 8) on the GPU, against the oracle: a non-symmetric system
imported through the block file (its NONSYM01 section: the blocks of both
orders and the left scaling coefficients), solved by the FP64 chain with the
forward sweep over the left coefficients (L, not R^T) and every near and far
block applied one way.  0.25 lambda PEC sphere, 480 unknowns, leaves <= 32,
CFIE alpha = 0.5, the oracle's non-symmetric scaling (reading A).

Operators L, R, D^-1, Z_F, Z (<= 1e-12 against oracle.nonsym, 1, 3 and 40
RHS), the n-term solves against the oracle's series (<= 1e-10, equal Eq. 45
ratios), and the calls a non-symmetric handle refuses (GPU scaling, save,
the mixed chain)."""
import numpy as np
import pytest

import hm_workloads as hw
from oracle.export import write_blocks_nonsym
from oracle.mfie import CFIE
from oracle.nonsym import (apply_L, build_hmatrix_general, compute_scaling_general,
                           series_solve_general)
from oracle.scaling import apply_Dinv, apply_R
from tests.gpu_util import from_dev, rand_panel, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfie():
    v, f = hw.icosphere(2, 0.25)
    H = build_hmatrix_general(v, f, lambda r: CFIE(r, 1.0, 0.5), leaf_max=32, compress="svd")
    S = compute_scaling_general(H, "A")
    th = np.radians(np.linspace(0.0, 180.0, 40))
    B = CFIE(H.rwg, 1.0, 0.5).plane_wave(th, np.zeros(40), np.arange(40) % 2)
    return H, S, B


def _load(H, S, tmp_path, **kw):
    import paper_2109_04129_gb300 as hp
    p = str(tmp_path / "cfie.hmps")
    write_blocks_nonsym(p, H, S)
    return hp.Solver.load(p, **kw)


@pytest.mark.parametrize("nrhs", [1, 3, 40])
def test_cfie_operators(cfie, tmp_path, nrhs):
    import torch
    H, S, B = cfie
    sol = _load(H, S, tmp_path)
    off = H.leaf_off
    x = rand_panel(H.N, nrhs, 31 + nrhs)
    X = to_dev(x)
    Y = torch.empty_like(X)
    xp = x[H.perm]
    for op, fn in (("RT", lambda v: apply_L(S, off, v)), ("R", lambda v: apply_R(S, off, v)),
                   ("DINV", lambda v: apply_Dinv(S, off, v)), ("FAR", H.far_apply),
                   ("NEAR", H.near_apply), ("Z", H.apply)):
        sol.apply(op, Y, X)
        want = np.empty_like(xp)
        want[H.perm] = fn(xp)
        err = rel(from_dev(Y), want)
        assert err.max() <= 1e-12, (op, err.max())


@pytest.mark.parametrize("n_terms", [2, 5])
def test_cfie_solve(cfie, tmp_path, n_terms):
    import torch
    H, S, B = cfie
    sol = _load(H, S, tmp_path, n_terms=n_terms)
    want, ratios = series_solve_general(H, S, B, n_terms)
    Bd = to_dev(B)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    assert rel(from_dev(X), want).max() <= 1e-10
    r, _ = sol.diagnostics(B.shape[1])
    assert np.allclose(r, ratios[0], rtol=1e-9)
    assert ratios[0].max() < 1.0                 # the CFIE series converges here


def test_cfie_handle_refusals(cfie, tmp_path):
    import paper_2109_04129_gb300 as hp
    H, S, B = cfie
    with pytest.raises(hp.HMError) as e:
        _load(H, S, tmp_path, precision=hp.HM_MIXED, refine_steps=1)
    assert e.value.status == hp.HM_ERR_INVALID
    sol = _load(H, S, tmp_path)
    with pytest.raises(hp.HMError) as e:
        sol.compute_scaling()
    assert e.value.status == hp.HM_ERR_STATE
    with pytest.raises(hp.HMError) as e:
        sol.save(str(tmp_path / "again.hmps"))
    assert e.value.status == hp.HM_ERR_STATE
