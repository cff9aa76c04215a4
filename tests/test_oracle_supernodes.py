"""Supernodes of the nested-dissection order (CPU, oracle only).

The GPU sweeps apply the forward substitution of Eq. 25 group by group: a
group G of consecutive elimination ranks (one bottom set or one separator of
the dissection) first gathers its sources outside G, then applies
T_G = (I - A_G^T)^-1 as one dense product.  These tests pin the oracle's
statement of both pieces: the groups (a partition of the ranks into
consecutive runs) and T_G (against the leaf-by-leaf forward substitution,
which Eq. 23 pins), and show that the group schedule reproduces R^T b."""
import os
import tempfile

import numpy as np

from oracle.export import read_blocks, write_blocks, leaf_centres
from oracle.scaling import (apply_Rt, apply_R, compute_scaling, nd_order,
                            supernode_inverse)
from tests.oracle_cases import case


def _nd_case():
    w, H, _, _ = case("sphere_r0.5_L3")
    order, groups = nd_order(H.tree, list(H.near.keys()), with_groups=True)
    S = compute_scaling(H, "A", order)
    return H, S, order, groups


def test_nd_groups_partition_the_ranks():
    H, S, order, groups = _nd_case()
    assert order == nd_order(H.tree, list(H.near.keys()))
    assert groups[0] == 0 and groups[-1] == H.n_leaves
    assert all(b > a for a, b in zip(groups, groups[1:]))
    # several groups of more than one leaf (what the supernode sweeps use)
    sizes = np.diff(groups)
    assert (sizes > 1).sum() >= 3


def test_supernode_inverse_equals_restricted_forward_substitution():
    """T_G b_G = (R^T b)_G for b supported on G: every path of the forward
    substitution between two ranks of G runs through ranks of G only, because
    the ranks of G are consecutive."""
    H, S, order, groups = _nd_case()
    m = np.diff(H.leaf_off)[order]
    off = np.concatenate([[0], np.cumsum(m)])
    rng = np.random.default_rng(3)
    checked = 0
    for g in range(len(groups) - 1):
        g0, g1 = groups[g], groups[g + 1]
        if g1 - g0 < 2:
            continue
        T = supernode_inverse(S, H.leaf_off, g0, g1)
        b_rank = np.zeros((H.N, 2), np.complex128)          # rank-ordered panel
        bG = rng.standard_normal((off[g1] - off[g0], 2)) + 1j * rng.standard_normal(
            (off[g1] - off[g0], 2))
        b_rank[off[g0]:off[g1]] = bG
        # to leaf order for apply_Rt
        b = np.zeros_like(b_rank)
        for q, leaf in enumerate(order):
            b[H.leaf_slice(leaf)] = b_rank[off[q]:off[q + 1]]
        y = apply_Rt(S, H.leaf_off, b)
        yG = np.concatenate([y[H.leaf_slice(order[q])] for q in range(g0, g1)])
        assert np.abs(T @ bG - yG).max() <= 1e-12 * np.abs(yG).max()
        checked += 1
    assert checked >= 3


def _group_sweep(H, S, groups, b, forward=True):
    """R^T b (forward) or R b (backward) by the supernode schedule: group
    levels; per level, every target adds its sources outside its group, then
    each group applies T_G (forward) or T_G^T (backward)."""
    order = S.order
    n = S.n
    sl = [H.leaf_slice(order[q]) for q in range(n)]
    gid = np.zeros(n, int)
    for g in range(len(groups) - 1):
        gid[groups[g]:groups[g + 1]] = g
    ng = len(groups) - 1
    src = [[] for _ in range(n)]
    for k in range(n):
        for j in S.rows[k]:
            if forward:
                src[j].append(k)
            else:
                src[k].append(j)
    lev = [0] * ng
    seq = range(ng) if forward else range(ng - 1, -1, -1)
    for g in seq:
        for t in range(groups[g], groups[g + 1]):
            for s in src[t]:
                if gid[s] != g:
                    lev[g] = max(lev[g], lev[gid[s]] + 1)
    out = np.array(b, dtype=np.complex128, copy=True)
    for L in range(max(lev) + 1):
        gs = [g for g in range(ng) if lev[g] == L]
        add = {}
        for g in gs:
            for t in range(groups[g], groups[g + 1]):
                acc = np.zeros_like(out[sl[t]])
                for s in src[t]:
                    if gid[s] == g:
                        continue
                    A = S.alpha[(s, t)] if forward else S.alpha[(t, s)]
                    acc += (A.T if forward else A) @ out[sl[s]]
                add[t] = acc
        for t, a in add.items():
            out[sl[t]] += a
        for g in gs:
            g0, g1 = groups[g], groups[g + 1]
            if g1 - g0 < 2:
                continue
            T = supernode_inverse(S, H.leaf_off, g0, g1)
            v = np.concatenate([out[sl[q]] for q in range(g0, g1)])
            v = (T if forward else T.T) @ v
            p = 0
            for q in range(g0, g1):
                mq = sl[q].stop - sl[q].start
                out[sl[q]] = v[p:p + mq]
                p += mq
    return out


def test_group_schedule_reproduces_both_sweeps():
    H, S, order, groups = _nd_case()
    rng = np.random.default_rng(11)
    b = rng.standard_normal((H.N, 3)) + 1j * rng.standard_normal((H.N, 3))
    for fwd, ref in ((True, apply_Rt(S, H.leaf_off, b)), (False, apply_R(S, H.leaf_off, b))):
        got = _group_sweep(H, S, groups, b, fwd)
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), fwd


def test_block_file_sections_round_trip():
    H, S, order, groups = _nd_case()
    fd, path = tempfile.mkstemp(suffix=".hmps")
    os.close(fd)
    try:
        write_blocks(path, H, S, groups=groups)
        d = read_blocks(path)
    finally:
        os.unlink(path)
    assert np.array_equal(d["leaf_cen"], leaf_centres(H))
    assert d["groups"] == groups and d["elim"] == order
    for g, T in d["T"].items():
        assert np.array_equal(T, supernode_inverse(S, H.leaf_off, groups[g], groups[g + 1]))
    assert len(d["T"]) == int((np.diff(groups) > 1).sum())


def test_load_blocks_gives_the_same_series():
    """The oracle's loader of block files (used to check the library on its
    own blocks) reproduces the series of the H-matrix and scaling it was
    written from."""
    from oracle.export import load_blocks
    from oracle.series import series_solve
    H, S, order, groups = _nd_case()
    fd, path = tempfile.mkstemp(suffix=".hmps")
    os.close(fd)
    try:
        write_blocks(path, H, S)
        H2, S2 = load_blocks(path)
        rng = np.random.default_rng(2)
        b = rng.standard_normal((H.N, 2)) + 1j * rng.standard_normal((H.N, 2))
        x1, r1 = series_solve(H, S, b, 3)
        x2, r2 = series_solve(H2, S2, b, 3)
        assert np.array_equal(x1, x2) and np.array_equal(r1, r2)
    finally:
        os.unlink(path)
