"""Bounded device waits: a solve whose waits may spin only once gives up, the
host reads HM_ERR_TIMEOUT from hm_get_diagnostics, and the context stays
usable (a second handle with the default limit still solves correctly).

Every mbarrier wait of the tensor-core kernels is bounded by spin_limit; a
CTA that gives up records the timeout, lets its copies and MMAs complete
under a cleanup limit of its own, releases tensor memory and returns.  No
fault, trap or endless loop is involved."""
import numpy as np
import pytest

from hm_workloads.meshes import closed_cylinder

pytestmark = pytest.mark.gpu


def _handle(spin_limit):
    import paper_2109_04129_gb300 as hp
    v, t = closed_cylinder(0.3, 0.6, 0.1)
    s = hp.Solver.build(v, t, wavelength=1.0, leaf_max=64, ordering=hp.HM_ORDER_ND,
                        precision=hp.HM_MIXED, refine_steps=1, spin_limit=spin_limit)
    s.compute_scaling()
    return s


def _rhs(sol, nrhs):
    import torch
    B = torch.empty((nrhs, sol.N), dtype=torch.complex128, device="cuda")
    th = np.radians(np.linspace(0.0, 180.0, nrhs))
    sol.plane_wave(B, th, np.zeros(nrhs), np.zeros(nrhs, np.int32))
    return B


def test_wait_runs_out_and_context_survives():
    import torch
    import paper_2109_04129_gb300 as hp
    good = _handle(1 << 26)
    B = _rhs(good, 64)
    want = torch.empty_like(B)
    good.solve(want, B)
    torch.cuda.synchronize()
    assert hp._lib.hm_get_diagnostics(good._h, None, None, 64) in (hp.HM_OK,
                                                                   hp.HM_WARN_SERIES_RATIO)
    bad = _handle(1)
    X = torch.empty_like(B)
    bad.solve(X, B)                      # waits give up after one try
    torch.cuda.synchronize()             # no fault: the stream completes
    assert hp._lib.hm_get_diagnostics(bad._h, None, None, 64) == hp.HM_ERR_TIMEOUT
    # the context is intact: the good handle reproduces its result bit for bit
    again = torch.empty_like(B)
    good.solve(again, B)
    torch.cuda.synchronize()
    assert torch.equal(again, want)
