"""The far-field product entry point that allocates no device memory, for
callers that cannot allocate (a pre-sized pool or arena owns the device
memory, an allocator forbids raw cudaMalloc).  Checked through the C ABI
against the oracle's far-field product and against the ordinary
hm_apply(HM_OP_FAR) product, twice in a row (the fixed scratch array keeps the
previous call's contents), at the largest batch its scratch holds, and its
size limit one RHS above that.

Collected last on purpose: the other GPU tests run first."""
import numpy as np
import pytest

from tests.oracle_cases import case
from tests.gpu_util import load_case, to_dev, from_dev, rand_panel, rel

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20          # HM_NOALLOC_SCRATCH_BYTES of include/hm.h


def _oracle_far(H, x):
    y = np.empty_like(x)
    y[H.perm] = H.far_apply(x[H.perm])
    return y


def test_far_noalloc_matches_oracle_and_apply_far_twice():
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B = case("plate_2l")
    sol = load_case(H, S)
    for call, nrhs in enumerate((3, 7)):
        x = rand_panel(H.N, nrhs, 100 + call)
        X = to_dev(x)
        Yref = torch.empty((nrhs, H.N), dtype=torch.complex128, device="cuda")
        sol.apply("FAR", Yref, X)
        Y = torch.full((nrhs, H.N), float("nan"), dtype=torch.complex128, device="cuda")
        st = hp._lib.hm_apply_far_noalloc(sol._h, hp._ptr(Y), hp._ptr(X), nrhs)
        assert st == hp.HM_OK
        torch.cuda.synchronize()
        y = from_dev(Y)
        assert rel(y, _oracle_far(H, x)).max() < 1e-12, call
        assert rel(y, from_dev(Yref)).max() < 1e-12, call


def test_far_noalloc_size_limit():
    """The largest nrhs whose stage-1 panels (2 * sum of ranks rows) fit the
    scratch array works; one more is rejected; so is an absurd size."""
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B = case("plate_2l")
    sol = load_case(H, S)
    t_rows = 2 * sum(b[5].shape[1] for b in H.far if b[0] == "lr")
    nmax = SCRATCH_BYTES // 16 // t_rows
    x = rand_panel(H.N, nmax, 5)
    X = to_dev(x)
    Y = torch.empty_like(X)
    assert hp._lib.hm_apply_far_noalloc(sol._h, hp._ptr(Y), hp._ptr(X), nmax) == hp.HM_OK
    torch.cuda.synchronize()
    cols = [0, nmax // 2, nmax - 1]
    assert rel(from_dev(Y)[:, cols], _oracle_far(H, x[:, cols])).max() < 1e-12
    X1 = torch.zeros((nmax + 1, H.N), dtype=torch.complex128, device="cuda")
    Y1 = torch.empty_like(X1)
    st = hp._lib.hm_apply_far_noalloc(sol._h, hp._ptr(Y1), hp._ptr(X1), nmax + 1)
    assert st == hp.HM_ERR_INVALID
    st = hp._lib.hm_apply_far_noalloc(sol._h, hp._ptr(Y1), hp._ptr(X1), 1 << 30)
    assert st == hp.HM_ERR_INVALID
