"""Adaptive term count of the series (Sec. III-C, Eq. 44-45) on the GPU,
against the oracle's n-term loop with the same stopping rule: after term
it_t, stop when every RHS has ||it_t|| <= term_tol ||it_0||, or when some
RHS's terms stop shrinking, with n_terms as the cap.  Same number of terms and
the same solution (FP64 <= 1e-6, mixed + refinement <= 1e-4), on the
converging 2 lambda plate (ratio about 0.4) and on the 0.5 lambda sphere whose
terms eventually grow."""
import numpy as np
import pytest

from oracle.efie import EFIE
from oracle.series import refine_once, series_solve
from tests.gpu_util import from_dev, load_case, rel, to_dev
from tests.oracle_cases import case, plate_converging

pytestmark = pytest.mark.gpu

CAP = 60


def _margin_ok(H, S, B, tol):
    """The oracle's decisions are not borderline: at every term, the largest
    ||it_t|| / (tol ||it_0||) and the largest ratio ||it_t|| / ||it_t-1|| stay
    at least 1 % away from one (so rounding on the GPU takes the same ones)."""
    from oracle.scaling import apply_R, apply_Rt, apply_Dinv
    off = H.leaf_off
    b = np.asarray(B, dtype=np.complex128)[H.perm]
    it = apply_Dinv(S, off, apply_Rt(S, off, b))
    n0 = np.linalg.norm(it, axis=0)
    for _ in range(1, CAP):
        nxt = apply_Dinv(S, off, apply_Rt(S, off, H.far_apply(apply_R(S, off, it))))
        a = np.linalg.norm(nxt, axis=0)
        q1 = np.max(a / (tol * n0))
        q2 = np.max(a / np.linalg.norm(it, axis=0))
        if abs(q1 - 1) < 0.01 or abs(q2 - 1) < 0.01:
            return False
        if q1 <= 1 or q2 >= 1:
            return True
        it = nxt
    return True


def _plate40():
    H, S, _ = plate_converging()
    th = np.radians(np.linspace(0.0, 90.0, 40))
    B = EFIE(H.rwg, 1.0).plane_wave(th, np.full(40, np.radians(30.0)), np.arange(40) % 2)
    return H, S, B


@pytest.mark.parametrize("nrhs", [2, 40])
def test_adaptive_terms_fp64(nrhs):
    import torch
    H, S, B = _plate40() if nrhs == 40 else plate_converging()
    tol = 1e-6
    assert _margin_ok(H, S, B, tol)
    want, ratios = series_solve(H, S, B, CAP, term_tol=tol)
    sol = load_case(H, S, n_terms=CAP, term_tol=tol)
    Bd = to_dev(B)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    assert sol.stats()["terms_used"] == len(ratios) + 1 < CAP
    assert rel(from_dev(X), want).max() <= 1e-6


def test_adaptive_terms_mixed_tensor_cores():
    import torch
    import paper_2109_04129_gb300 as hp
    H, S, B = _plate40()
    tol = 1e-5
    assert _margin_ok(H, S, B, tol)
    x, ratios = series_solve(H, S, B, CAP, term_tol=tol)
    want = refine_once(H, S, B, x, CAP, term_tol=tol)
    sol = load_case(H, S, n_terms=CAP, term_tol=tol, precision=hp.HM_MIXED, refine_steps=1)
    Bd = to_dev(B)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    assert sol.stats()["terms_used"] >= len(ratios) + 1
    assert rel(from_dev(X), want).max() <= 1e-4


def test_adaptive_terms_stop_when_terms_grow():
    import torch
    w, H, S, B = case("sphere_r0.5_L3")
    tol = 1e-8
    assert _margin_ok(H, S, B, tol)
    want, ratios = series_solve(H, S, B, CAP, term_tol=tol)
    assert ratios[-1].max() >= 1.0
    sol = load_case(H, S, n_terms=CAP, term_tol=tol)
    Bd = to_dev(B)
    X = torch.empty_like(Bd)
    sol.solve(X, Bd)
    assert sol.stats()["terms_used"] == len(ratios) + 1
    assert rel(from_dev(X), want).max() <= 1e-6


def test_grouped_solve_refuses_adaptive_handles():
    import torch
    import paper_2109_04129_gb300 as hp
    H, S, B = plate_converging()
    sol = load_case(H, S, n_terms=CAP, term_tol=1e-6)
    Bd = to_dev(B)
    X = torch.empty_like(Bd)
    with pytest.raises(hp.HMError) as e:
        hp.solve_grouped([sol], [X], [Bd])
    assert e.value.status == hp.HM_ERR_STATE
