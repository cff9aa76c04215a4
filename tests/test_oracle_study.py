"""The oracle's study scripts on small cases: the leaf-size study (Sec. V-A,
Fig. 4) and its admissibility option, the memory study's counts against the
numerical scaling, and the mixed-precision error model."""
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_leaf_size_study_runs():
    r = subprocess.run([sys.executable, "-m", "oracle.study_leaf_size", "--level", "2",
                        "--radius", "0.25", "--caps", "16", "1000", "--terms", "2", "3",
                        "--processes", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    rows = [ln.split() for ln in r.stdout.splitlines() if not ln.startswith("#")]
    assert [int(x[0]) for x in rows] == [16, 1000]
    small, one_leaf = rows
    assert int(small[1]) > int(one_leaf[1]) == 1
    # a single leaf: no far field, the series is exact
    assert float(one_leaf[6]) < 1e-10 and float(one_leaf[7]) < 1e-10


def test_eta_admissibility_reduces_to_non_touching():
    """Non-touching cells are at least one smaller-cell edge apart, so the
    paper-form admissibility min(diam) <= eta dist with eta >= sqrt(3) gives
    the same block tree; a stricter eta only moves pairs from far to near."""
    import math
    import numpy as np
    from hm_workloads import icosphere
    from oracle.octree import Octree
    from oracle.rwg import build_rwg
    from oracle.study_leaf_size import eta_octree
    v, f = icosphere(3, 0.5)
    pts = build_rwg(v, f).centre
    near0, far0 = Octree(pts, 32).blocks()
    near1, far1 = eta_octree(math.sqrt(3.0) * (1 + 1e-12))(pts, 32).blocks()
    assert sorted(near0) == sorted(near1) and sorted(far0) == sorted(far1)
    T = eta_octree(1.0)(pts, 32)
    near2, far2 = T.blocks()
    assert set(near0) < set(near2)
    cover = np.zeros((len(pts), len(pts)), np.int8)
    for i, j in near2:
        cover[T.leaf_off[i]:T.leaf_off[i + 1], T.leaf_off[j]:T.leaf_off[j + 1]] += 1
    for s, t in far2:
        a, b = T.nodes[s], T.nodes[t]
        cover[a.start:a.start + a.count, b.start:b.start + b.count] += 1
    assert cover.min() == 1 and cover.max() == 1


def test_fill_study_counts_equal_the_scaling():
    """The symbolic counts of the memory study equal the entries of the
    numerical scaling (readings A in both orders, B) and of the near field."""
    from oracle.scaling import compute_scaling, nd_order
    from oracle.study_fill import counts
    from tests.oracle_cases import case
    _, H, SA, _ = case("sphere_r0.5_L3")
    N, nl, zn, d, ad, an, ab = counts(H.rwg.centre, H.meta["leaf_max"])
    assert (N, nl) == (H.N, H.n_leaves)
    assert zn == sum(b.size for b in H.near.values())
    assert (ad, d) == SA.entries(H.leaf_off)
    SN = compute_scaling(H, "A", nd_order(H.tree, list(H.near.keys())))
    assert an == SN.entries(H.leaf_off)[0]
    assert ab == compute_scaling(H, "B").entries(H.leaf_off)[0]
    assert ab < zn < ad                     # reading B below the near field, A above


def test_mixed_error_model_small_case():
    """The mixed-precision model runs on a small case: the chain's complex64
    storage alone moves the refined solution by FP32-level amounts, complex64
    arithmetic by more, both far below the mixed bar of 1e-4."""
    from oracle.series import rel_err
    from oracle.study_mixed_error import mixed_model
    from tests.oracle_cases import case
    _, H, S, B = case("sphere_r0.25_L2")
    xs, x64 = mixed_model(H, S, B[:, :4], arithmetic=False)
    xa, _ = mixed_model(H, S, B[:, :4], arithmetic=True)
    es, ea = rel_err(xs, x64), rel_err(xa, x64)
    assert np.all(es > 0) and np.all(es < 1e-5)
    assert np.all(ea < 1e-4) and ea.max() > es.max()


def test_binary_tree_partition():
    """The paper's binary tree (study reading): leaves tile the points, every
    leaf's longest edge lies in [leaf size, 2 leaf size), near and far blocks
    tile the index square once, and every far pair meets Eq. 10 (checked on
    the cell geometry, not with the tree's own test)."""
    from hm_workloads import icosphere
    from oracle.rwg import build_rwg
    from oracle.study_leaf_size import BinaryTree, leaf_edges
    v, f = icosphere(3, 1.0)
    pts = build_rwg(v, f).centre
    for size, eta in ((0.25, 1.0), (0.5, 1.0), (0.5, 2.0)):
        T = BinaryTree(pts, size, eta)
        assert sorted(T.perm.tolist()) == list(range(len(pts)))
        e = leaf_edges(T, 1.0)
        assert np.all(e >= size) and np.all(e < 2 * size)
        for n in T.leaves:
            nd = T.nodes[n]
            p = pts[T.perm[nd.start:nd.start + nd.count]]
            assert np.all(p >= nd.lo - 1e-12) and np.all(p <= nd.hi + 1e-12)
        near, far = T.blocks()
        cover = np.zeros((len(pts), len(pts)), np.int8)
        for i, j in near:
            cover[T.leaf_off[i]:T.leaf_off[i + 1], T.leaf_off[j]:T.leaf_off[j + 1]] += 1
        for s, t in far:
            a, b = T.nodes[s], T.nodes[t]
            cover[a.start:a.start + a.count, b.start:b.start + b.count] += 1
            # Eq. 10 on the cells: min diagonal <= eta * (distance between cells)
            lo = np.maximum(a.lo, b.lo)
            hi = np.minimum(a.hi, b.hi)
            dist = np.linalg.norm(np.maximum(0.0, lo - hi))
            dmin = min(np.linalg.norm(a.hi - a.lo), np.linalg.norm(b.hi - b.lo))
            assert dist > 0 and dmin <= eta * dist + 1e-12
        assert cover.min() == 1 and cover.max() == 1


def test_leaf_size_study_binary_tree_runs():
    r = subprocess.run([sys.executable, "-m", "oracle.study_leaf_size", "--level", "2",
                        "--radius", "0.25", "--binary", "0.1", "1.0", "--terms", "2",
                        "--processes", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    rows = [ln.split() for ln in r.stdout.splitlines() if not ln.startswith("#")]
    assert len(rows) == 2 and int(rows[0][1]) > int(rows[1][1])
