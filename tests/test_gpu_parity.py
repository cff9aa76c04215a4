"""GPU parity of the FP64 chain against the oracle (block file import: the
GPU consumes the oracle's leaf order, blocks, alpha and D^-1).

Tolerance: relative L2 error per RHS <= 1e-6 for the solve (the FP64 bar);
single operators <= 1e-12 (same products, different summation order)."""
import numpy as np
import pytest

from oracle.scaling import apply_R, apply_Rt, apply_Dinv, compute_scaling
from oracle.series import series_solve
from tests.oracle_cases import case, plate_converging
from tests.gpu_util import load_case, to_dev, from_dev, rand_panel, rel

pytestmark = pytest.mark.gpu

CASES = ["sphere_r0.25_L2", "plate_2l", "sphere_r0.5_L3"]


def _oracle_op(H, S, op, X):
    p = H.perm
    xp = X[p]
    if op == "RT":
        y = apply_Rt(S, H.leaf_off, xp)
    elif op == "R":
        y = apply_R(S, H.leaf_off, xp)
    elif op == "DINV":
        y = apply_Dinv(S, H.leaf_off, xp)
    elif op == "FAR":
        y = H.far_apply(xp)
    elif op == "NEAR":
        y = H.near_apply(xp)
    else:
        y = H.apply(xp)
    out = np.empty_like(y)
    out[p] = y
    return out


@pytest.fixture(scope="module", params=CASES)
def loaded(request):
    import torch
    assert torch.cuda.is_available()
    w, H, S, B = case(request.param)
    return request.param, H, S, B, load_case(H, S)


@pytest.mark.parametrize("op", ["RT", "R", "DINV", "FAR", "NEAR", "Z"])
@pytest.mark.parametrize("nrhs", [1, 3, 7, 40])
def test_operator_parity(loaded, op, nrhs):
    import torch
    name, H, S, B, sol = loaded
    X = rand_panel(H.N, nrhs, 11 + nrhs)
    Y = torch.empty((nrhs, H.N), dtype=torch.complex128, device="cuda")
    sol.apply(op, Y, to_dev(X))
    want = _oracle_op(H, S, op, X)
    err = rel(from_dev(Y), want)
    assert err.max() < 1e-12, (name, op, nrhs, err.max())


def test_solve_parity_fp64(loaded):
    import torch
    name, H, S, B, sol = loaded
    X = torch.empty((B.shape[1], H.N), dtype=torch.complex128, device="cuda")
    sol.solve(X, to_dev(B))
    want, ratio = series_solve(H, S, B, 2)
    err = rel(from_dev(X), want)
    assert err.max() <= 1e-6, (name, err)
    import paper_2109_04129_gb300 as hp
    st = hp._lib.hm_get_diagnostics(sol._h, None, None, B.shape[1])
    r, _ = sol.diagnostics(B.shape[1])
    assert np.allclose(r, ratio[0], rtol=1e-9)
    assert (st == hp.HM_WARN_SERIES_RATIO) == bool(np.any(ratio[0] > 0.1))


def test_solve_host_buffers_equal_device(loaded):
    import torch
    name, H, S, B, sol = loaded
    Bh = np.ascontiguousarray(B.T)
    Xh = np.zeros_like(Bh)
    sol.solve_host(Xh, Bh)
    X = torch.empty((B.shape[1], H.N), dtype=torch.complex128, device="cuda")
    sol.solve(X, to_dev(B))
    assert np.array_equal(Xh, X.cpu().numpy())


def test_more_terms_and_reading_B():
    import torch
    H, S, B = plate_converging()
    for nt in (1, 3, 6):
        sol = load_case(H, S, n_terms=nt)
        X = torch.empty((B.shape[1], H.N), dtype=torch.complex128, device="cuda")
        sol.solve(X, to_dev(B))
        want, _ = series_solve(H, S, B, nt)
        assert rel(from_dev(X), want).max() <= 1e-6
    w, Hs, _, Bs = case("sphere_r0.25_L2")
    SB = compute_scaling(Hs, "B")
    sol = load_case(Hs, SB)
    X = torch.empty((Bs.shape[1], Hs.N), dtype=torch.complex128, device="cuda")
    sol.solve(X, to_dev(Bs))
    want, _ = series_solve(Hs, SB, Bs, 2)
    assert rel(from_dev(X), want).max() <= 1e-6


def test_state_and_argument_errors():
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B = case("sphere_r0.25_L2")
    sol = load_case(H, None)                 # no scaling in the file
    X = torch.empty((1, H.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(hp.HMError) as e:
        sol.solve(X, to_dev(B[:, :1]))
    assert e.value.status == hp.HM_ERR_STATE
    # Z_F and Z_N products do not need the scaling
    sol.apply("FAR", X, to_dev(B[:, :1]))
    sol2 = load_case(H, S)
    assert hp._lib.hm_power_series_solve(sol2._h, hp._ptr(X), hp._ptr(X), 0) == hp.HM_ERR_INVALID


def test_save_load_round_trip(tmp_path):
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B = case("plate_2l")
    sol = load_case(H, S)
    p = str(tmp_path / "c.hmps")
    sol.save(p)
    sol2 = hp.Solver.load(p)
    X1 = torch.empty((B.shape[1], H.N), dtype=torch.complex128, device="cuda")
    X2 = torch.empty_like(X1)
    sol.solve(X1, to_dev(B))
    sol2.solve(X2, to_dev(B))
    assert torch.equal(X1, X2)


@pytest.mark.parametrize("name", CASES)
def test_mixed_solve_parity(name):
    """Mixed chain (complex64 alpha / far factors, FP64 D^-1) plus one FP64
    residual refinement vs the oracle's FP64 series plus the same refinement:
    relative L2 error <= 1e-4 per RHS."""
    import torch
    import paper_2109_04129_gb300 as hp
    from oracle.series import refine_once
    w, H, S, B = case(name)
    sol = load_case(H, S, precision=hp.HM_MIXED, refine_steps=1)
    X = torch.empty((B.shape[1], H.N), dtype=torch.complex128, device="cuda")
    sol.solve(X, to_dev(B))
    x2, _ = series_solve(H, S, B, 2)
    want = refine_once(H, S, B, x2)
    err = rel(from_dev(X), want)
    assert err.max() <= 1e-4, (name, err.max())
    r, resid = sol.diagnostics(B.shape[1])
    assert np.all(resid > 0)


@pytest.mark.parametrize("op", ["RT", "R", "DINV", "FAR"])
def test_mixed_operator_parity(op):
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B = case("plate_2l")
    sol = load_case(H, S, precision=hp.HM_MIXED, refine_steps=1)
    for nrhs in (1, 5, 40):
        X = rand_panel(H.N, nrhs, 3 + nrhs)
        Y = torch.empty((nrhs, H.N), dtype=torch.complex128, device="cuda")
        sol.apply(op, Y, to_dev(X))
        err = rel(from_dev(Y), _oracle_op(H, S, op, X))
        assert err.max() < 2e-5, (op, nrhs, err.max())


@pytest.mark.parametrize("name", ["sphere_r0.25_L2", "plate_2l"])
def test_mixed_tensor_core_solve(name):
    """nrhs >= 32 runs the mixed products on tcgen05 (three-way bf16 split,
    FP32 accumulation): same 1e-4 bar against the oracle's FP64 series plus
    refinement, and close to the CUDA-core FP32 path."""
    import torch
    import paper_2109_04129_gb300 as hp
    from oracle.series import refine_once
    w, H, S, B = case(name)
    Bw = np.concatenate([B, rand_panel(H.N, 40, 77) * np.abs(B).max()], axis=1)   # 52+ RHS
    x2, _ = series_solve(H, S, Bw, 2)
    want = refine_once(H, S, Bw, x2)
    out = {}
    for tc in (1, 0):
        sol = load_case(H, S, precision=hp.HM_MIXED, refine_steps=1, tensor_cores=tc)
        X = torch.empty((Bw.shape[1], H.N), dtype=torch.complex128, device="cuda")
        sol.solve(X, to_dev(Bw))
        assert hp._lib.hm_get_diagnostics(sol._h, None, None, Bw.shape[1]) in (0, 100)
        out[tc] = from_dev(X)
        err = rel(out[tc], want)
        assert err.max() <= 1e-4, (name, tc, err.max())
    assert rel(out[1], out[0]).max() <= 1e-4


@pytest.mark.parametrize("name", ["sphere_r0.25_L2", "plate_2l", "sphere_r0.5_L3"])
@pytest.mark.parametrize("op", ["NEAR", "Z"])
def test_fp64_emulated_products(name, op):
    """Refinement-residual products of a mixed handle (nrhs >= 32: bf16 tensor
    cores with exact 7-bit integer slicing of the FP64 operands) against the
    oracle's FP64 products: relative error <= 1e-12 per RHS."""
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B = case(name)
    sol = load_case(H, S, precision=hp.HM_MIXED, refine_steps=1)
    for nrhs, seed in ((33, 5), (130, 6)):
        X = rand_panel(H.N, nrhs, seed)
        X[:, 0] *= 1e-6            # a column far below the others' scale
        Y = torch.empty((nrhs, H.N), dtype=torch.complex128, device="cuda")
        sol.apply(op, Y, to_dev(X))
        err = rel(from_dev(Y), _oracle_op(H, S, op, X))
        assert err.max() < 1e-12, (name, op, nrhs, err.max())
    assert hp._lib.hm_get_diagnostics(sol._h, None, None, 1) != hp.HM_ERR_TIMEOUT


def test_fp64_refinement_parity():
    """FP64 chain with one refinement step vs the oracle's FP64 series plus
    the same refinement (the like-for-like comparator of the mixed chain)."""
    import torch
    from oracle.series import refine_once
    for name in ("sphere_r0.25_L2", "plate_2l"):
        w, H, S, B = case(name)
        sol = load_case(H, S, refine_steps=1)
        X = torch.empty((B.shape[1], H.N), dtype=torch.complex128, device="cuda")
        sol.solve(X, to_dev(B))
        x2, _ = series_solve(H, S, B, 2)
        want = refine_once(H, S, B, x2)
        assert rel(from_dev(X), want).max() <= 1e-6
        r, resid = sol.diagnostics(B.shape[1])
        assert np.all(resid > 0)
