"""The far-field product entry point that allocates no device memory, for
callers that cannot allocate (a pre-sized pool or arena owns the device
memory, an allocator forbids raw cudaMalloc).  Checked through the C ABI
against the ordinary hm_apply(HM_OP_FAR) product, twice in a row (the fixed
scratch array keeps the previous call's contents), and its size limit.

Collected last on purpose: the other GPU tests run first."""
import ctypes

import numpy as np
import pytest

from tests.oracle_cases import case
from tests.gpu_util import load_case, to_dev, from_dev, rand_panel, rel

pytestmark = pytest.mark.gpu


def test_far_noalloc_matches_apply_far_twice():
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B = case("plate_2l")
    sol = load_case(H, S)
    for call, nrhs in enumerate((3, 7)):
        X = to_dev(rand_panel(H.N, nrhs, 100 + call))
        Yref = torch.empty((nrhs, H.N), dtype=torch.complex128, device="cuda")
        sol.apply("FAR", Yref, X)
        Y = torch.full((nrhs, H.N), float("nan"), dtype=torch.complex128, device="cuda")
        st = hp._lib.hm_apply_far_noalloc(sol._h, hp._ptr(Y), hp._ptr(X), nrhs)
        assert st == hp.HM_OK
        torch.cuda.synchronize()
        err = rel(from_dev(Y), from_dev(Yref))
        assert err.max() < 1e-12, (call, err.max())


def test_far_noalloc_rejects_oversize():
    import torch
    import paper_2109_04129_gb300 as hp
    w, H, S, B = case("plate_2l")
    sol = load_case(H, S)
    X = torch.zeros((1, H.N), dtype=torch.complex128, device="cuda")
    huge = 1 << 30
    st = hp._lib.hm_apply_far_noalloc(sol._h, hp._ptr(X), hp._ptr(X), huge)
    assert st == hp.HM_ERR_INVALID
