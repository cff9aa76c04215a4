"""Grouped solve of a batch of independent scatterers (one CUDA graph with a
branch per problem) against the per-problem solves and the oracle.

The grouped call runs the same kernels on the same data as one
hm_power_series_solve per problem, and every kernel of the chain is
deterministic (no atomics; split-K partial sums are reduced in a fixed
order), so the results must be bit-identical to the single solves.  The two
problems loaded from the oracle's blocks are also held to the FP64 bar
(relative L2 error <= 1e-6 per RHS vs the oracle's two-term series) and the
mixed bar (<= 1e-4 vs the oracle's series plus one refinement step)."""
import numpy as np
import pytest

from hm_workloads.meshes import closed_cylinder, ellipsoid
from oracle.series import series_solve, refine_once
from tests.oracle_cases import case
from tests.gpu_util import load_case, to_dev, from_dev, rel

pytestmark = pytest.mark.gpu

ORACLE_CASES = ["sphere_r0.25_L2", "plate_2l"]


def _batch(precision):
    """Two oracle-loaded problems and two natively built closed bodies with
    uneven leaf caps and RHS counts (14, 12, 40, 91)."""
    import torch
    import paper_2109_04129_gb300 as hp
    kw = dict(precision=precision, refine_steps=1 if precision == hp.HM_MIXED else 0)
    probs = []
    for name in ORACLE_CASES:
        w, H, S, B = case(name)
        probs.append(dict(name=name, sol=load_case(H, S, **kw), B=to_dev(B), H=H, S=S,
                          Bh=B))
    for name, (v, t), leaf, nrhs in (
            ("cylinder", closed_cylinder(0.3, 0.6, 0.1), 32, 40),
            ("ellipsoid", ellipsoid(2, (0.25, 0.25, 0.6)), 64, 91)):
        sol = hp.Solver.build(v, t, wavelength=1.0, leaf_max=leaf, ordering=hp.HM_ORDER_ND, **kw)
        sol.compute_scaling()
        th = np.radians(np.linspace(0.0, 180.0, nrhs))
        B = torch.empty((nrhs, sol.N), dtype=torch.complex128, device="cuda")
        sol.plane_wave(B, th, np.zeros(nrhs), np.zeros(nrhs, np.int32))
        probs.append(dict(name=name, sol=sol, B=B))
    return probs


def _singles(probs):
    import torch
    out = []
    for p in probs:
        X = torch.empty_like(p["B"])
        p["sol"].solve(X, p["B"])
        out.append(X)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grouped_equals_single_solves(precision):
    import torch
    import paper_2109_04129_gb300 as hp
    prec = hp.HM_FP64 if precision == "fp64" else hp.HM_MIXED
    probs = _batch(prec)
    sols = [p["sol"] for p in probs]
    Bs = [p["B"] for p in probs]
    Xs = [torch.full_like(B, complex(7.0, -3.0)) for B in Bs]
    want = _singles(probs)
    hp.solve_grouped(sols, Xs, Bs)          # records the graph, then launches it
    torch.cuda.synchronize()
    for p, X, W in zip(probs, Xs, want):
        assert torch.equal(X, W), p["name"]
    # the oracle bar on the problems loaded from its blocks
    for p, X in zip(probs[:2], Xs[:2]):
        x2, _ = series_solve(p["H"], p["S"], p["Bh"], 2)
        if prec == hp.HM_FP64:
            err = rel(from_dev(X), x2)
            assert err.max() <= 1e-6, (p["name"], err.max())
        else:
            err = rel(from_dev(X), refine_once(p["H"], p["S"], p["Bh"], x2))
            assert err.max() <= 1e-4, (p["name"], err.max())
    # replay: new right-hand sides in the same buffers, graph launched again
    for i, B in enumerate(Bs):
        B.mul_(complex(0.5, 0.25 * (i + 1)))
    want2 = _singles(probs)
    for X in Xs:
        X.fill_(0)
    hp.solve_grouped(sols, Xs, Bs)
    torch.cuda.synchronize()
    for p, X, W in zip(probs, Xs, want2):
        assert torch.equal(X, W), p["name"]
    # per-handle diagnostics after a grouped launch
    for p in probs:
        r, _ = p["sol"].diagnostics(p["B"].shape[0])
        assert np.all(np.isfinite(r)) and np.all(r > 0)


def test_grouped_rebuilds_after_buffer_growth():
    """A handle whose work panels were reallocated (a single solve with more
    RHS) gets a fresh graph: the grouped result stays equal to single solves."""
    import torch
    import paper_2109_04129_gb300 as hp
    probs = _batch(hp.HM_FP64)[2:]
    sols = [p["sol"] for p in probs]
    Bs = [p["B"][:16].contiguous() for p in probs]
    Xs = [torch.empty_like(B) for B in Bs]
    hp.solve_grouped(sols, Xs, Bs)
    torch.cuda.synchronize()
    big = probs[1]["B"]                     # 91 RHS > 16: panels reallocated
    Xb = torch.empty_like(big)
    sols[1].solve(Xb, big)
    for X in Xs:
        X.fill_(0)
    hp.solve_grouped(sols, Xs, Bs)
    torch.cuda.synchronize()
    for s, B, X in zip(sols, Bs, Xs):
        W = torch.empty_like(B)
        s.solve(W, B)
        torch.cuda.synchronize()
        assert torch.equal(X, W)


def test_grouped_rejects_bad_arguments():
    import torch
    import paper_2109_04129_gb300 as hp
    probs = _batch(hp.HM_FP64)[2:]
    s0 = probs[0]["sol"]
    B = probs[0]["B"]
    X = torch.empty_like(B)
    with pytest.raises(hp.HMError):          # the same handle twice
        hp.solve_grouped([s0, s0], [X, torch.empty_like(B)], [B, B])
    s0.profile_enable(True)
    with pytest.raises(hp.HMError):          # profiling events cannot be recorded in a graph
        hp.solve_grouped([s0], [X], [B])
    s0.profile_enable(False)
    hp.solve_grouped([s0], [X], [B])
    torch.cuda.synchronize()
