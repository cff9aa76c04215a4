"""The split-K autotuner of the tensor-core sweeps (hm_params.autotune): on
the first mixed solve with 32 or more RHS every supernode sweep phase is timed
with its candidate split sizes and the fastest lists are kept; the choices are
cached per phase shape for the process.  Checked against the oracle on the
0.5 lambda sphere (the library's own nested-dissection scaling, 40 RHS): tuned
and untuned handles both within the mixed bar, a second handle of the same
case takes the cached choices and reproduces the first handle's result bit for
bit, and a grouped solve of tuned handles equals their single solves."""
import numpy as np
import pytest

from oracle.efie import EFIE
from oracle.scaling import compute_scaling, nd_order
from oracle.series import refine_once, series_solve
from tests.gpu_util import from_dev, load_case, rel, to_dev
from tests.oracle_cases import case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nd():
    w, H, _, _ = case("sphere_r0.5_L3")
    S = compute_scaling(H, "A", nd_order(H.tree, list(H.near.keys())))
    th = np.radians(np.linspace(0.0, 180.0, 40))
    B = EFIE(H.rwg, w.wavelength).plane_wave(th, np.zeros(40), np.arange(40) % 2)
    x2, _ = series_solve(H, S, B, 2)
    return H, S, B, refine_once(H, S, B, x2)


def _mixed(H, tune):
    import paper_2109_04129_gb300 as hp
    sol = load_case(H, None, ordering=hp.HM_ORDER_ND, precision=hp.HM_MIXED, refine_steps=1,
                    autotune=tune)
    sol.compute_scaling()
    return sol


def test_tuned_and_untuned_within_the_bar(nd):
    import torch
    H, S, B, want = nd
    Bd = to_dev(B)
    out = {}
    for tune in (0, 1):
        sol = _mixed(H, tune)
        X = torch.empty_like(Bd)
        sol.solve(X, Bd)
        assert rel(from_dev(X), want).max() <= 1e-4, tune
        st = sol.stats()
        out[tune] = (st["tuned_phases"], st["fwd_levels"] + st["bwd_levels"])
    assert out[0][0] == 0
    assert out[1][0] == out[1][1]              # every phase of both sweeps tuned


def test_cached_choices_and_grouped_solve(nd):
    import torch
    import paper_2109_04129_gb300 as hp
    H, S, B, want = nd
    Bd = to_dev(B)
    a, b = _mixed(H, 1), _mixed(H, 1)
    Xa, Xb = torch.empty_like(Bd), torch.empty_like(Bd)
    a.solve(Xa, Bd)
    b.solve(Xb, Bd)                             # same phase shapes: choices from the cache
    assert torch.equal(Xa, Xb)
    assert b.stats()["tuned_phases"] == a.stats()["tuned_phases"] > 0
    Ga, Gb = torch.empty_like(Bd), torch.empty_like(Bd)
    hp.solve_grouped([a, b], [Ga, Gb], [Bd, Bd])
    torch.cuda.synchronize()
    assert torch.equal(Ga, Xa) and torch.equal(Gb, Xb)
