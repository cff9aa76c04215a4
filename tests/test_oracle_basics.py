"""Pins of the oracle's building blocks: quadrature, closed-form potentials,
RWG basis, meshes, octree and ACA (Sec. II, Eq. 10-12)."""
import math
import os

import numpy as np
import pytest

from hm_workloads import icosphere, plate, mesh_stats, closed_cylinder, ellipsoid
from oracle.quadrature import dunavant7
from oracle.potentials import static_potentials, duffy_brute
from oracle.rwg import build_rwg
from oracle.octree import Octree
from oracle.aca import aca, recompress
from oracle.efie import EFIE

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_dunavant_matches_published_table():
    pts, w = dunavant7()
    tab = _golden("dunavant7.txt")
    got = sorted({(round(float(p.min()), 15), round(float(wt), 15)) for p, wt in zip(pts, w)})
    want = sorted((round(float(a), 15), round(float(b), 15)) for a, b in tab)
    # orbit (a, a, 1-2a): the smallest barycentric coordinate of the
    # 0.47 orbit is 1 - 2a, of the others a itself
    got_a = sorted(round(x, 12) for x, _ in got)
    want_a = sorted(round(min(a, 1 - 2 * a), 12) for a, _ in want)
    assert got_a == want_a
    assert sorted(round(b, 12) for _, b in got) == sorted(round(b, 12) for _, b in want)
    assert abs(w.sum() - 1.0) < 1e-15


def test_dunavant_degree5_exact_degree6_not():
    pts, w = dunavant7()
    # reference triangle (0,0),(1,0),(0,1): x = l2, y = l3, area 1/2
    x, y = pts[:, 1], pts[:, 2]
    for a in range(7):
        for b in range(7 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = 0.5 * np.sum(w * x ** a * y ** b)
            if a + b <= 5:
                assert abs(got - exact) < 1e-15, (a, b)
    worst = max(abs(0.5 * np.sum(w * x ** a * y ** (6 - a)) -
                    math.factorial(a) * math.factorial(6 - a) / math.factorial(8))
                for a in range(7))
    assert worst > 1e-6


@pytest.mark.parametrize("obs", [
    (0.4, 0.3, 0.0),          # inside, in plane (self-term singularity)
    (0.4, 0.3, 0.05),         # just above
    (1.3, 0.9, 0.02),         # outside, near an edge extension
    (-0.4, -0.02, 0.0),       # in plane, beyond a vertex
    (3.0, -2.0, 1.0),         # far
])
def test_static_potentials_vs_duffy(obs):
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.0]])
    Is, Iv, _ = static_potentials(np.array([obs]), tri[None])
    bs, bv = duffy_brute(np.array(obs), tri, order=64)
    assert abs(Is[0] - bs) < 1e-10 * max(1.0, abs(bs))
    assert np.abs(Iv[0] - bv).max() < 1e-10


def test_static_potential_far_limit():
    tri = np.array([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0], [0.0, 0.01, 0.0]])
    c = tri.mean(0)
    obs = np.array([[5.0, 3.0, 2.0]])
    Is, _, _ = static_potentials(obs, tri[None])
    area = 0.5e-4
    # next term of the multipole expansion is O((size / distance)^2) ~ 1e-6
    assert abs(Is[0] - area / np.linalg.norm(obs[0] - c)) < 1e-5 * Is[0]


def test_workload_counts_golden():
    for name, nt, nu in _golden("workload_counts.txt"):
        if name.startswith("icosphere"):
            L = int(name[-1])
            if L > 5:
                assert 20 * 4 ** L == int(nt) and 30 * 4 ** L == int(nu)
                continue
            v, f = icosphere(L, 1.0)
        else:
            v, f = plate(8.0, 80)
        r = build_rwg(v, f)
        assert len(f) == int(nt) and r.n == int(nu)


def test_meshes_closed_and_oriented():
    for v, f in (icosphere(2, 0.5), closed_cylinder(0.3, 0.8, 0.1), ellipsoid(2, (0.3, 0.3, 0.9))):
        st = mesh_stats(v, f)
        assert st["boundary"] == 0 and st["nonmanifold"] == 0 and st["euler"] == 2
        assert st["volume"] > 0
    v, f = icosphere(3, 0.5)
    assert np.allclose(np.linalg.norm(v, axis=1), 0.5)
    st = mesh_stats(*plate(2.0, 20))
    assert st["boundary"] == 80 and st["euler"] == 1


def test_rwg_charge_neutral_and_normal_continuity():
    v, f = icosphere(2, 0.5)
    r = build_rwg(v, f)
    assert r.n == 3 * len(f) // 2
    # total charge: (l/A+) A+ - (l/A-) A- = 0 exactly by construction; check the
    # flux of f through the common edge from both sides equals l
    for n in range(0, r.n, 37):
        a, b = r.edge[n]
        for tri, free, sgn in ((r.tri_p[n], r.free_p[n], 1.0), (r.tri_m[n], r.free_m[n], -1.0)):
            vf = v[f[tri, free]]
            mid = 0.5 * (v[a] + v[b])
            fval = sgn * r.length[n] / (2 * r.area[tri]) * (mid - vf)
            # in-plane normal of the edge pointing away from the free vertex
            e = v[b] - v[a]
            nrm = np.cross(v[f[tri, 1]] - v[f[tri, 0]], v[f[tri, 2]] - v[f[tri, 0]])
            u = np.cross(e, nrm)
            u /= np.linalg.norm(u)
            if np.dot(u, mid - vf) < 0:
                u = -u
            flux = np.dot(fval, u) * r.length[n]
            assert abs(abs(flux) - r.length[n]) < 1e-12   # f.u = 1 on the edge
            assert np.sign(flux) == sgn


def far_pairs_separated(T, far):
    """Every far pair's cells (boxes from the octree cube) leave a gap of at
    least the smaller cell's edge on some axis (non-touching admissibility)."""
    for s, t in far:
        a, b = T.nodes[s], T.nodes[t]
        ca, cb = T.size / 2 ** a.level, T.size / 2 ** b.level
        lo_a = T.origin + np.array(a.ijk) * ca
        lo_b = T.origin + np.array(b.ijk) * cb
        gap = np.maximum(lo_b - (lo_a + ca), lo_a - (lo_b + cb))
        if not gap.max() >= min(ca, cb) * (1 - 1e-9):
            return False
    return True


def test_octree_tiling_and_admissibility():
    v, f = icosphere(3, 0.5)
    r = build_rwg(v, f)
    T = Octree(r.centre, 64)
    near, far = T.blocks()
    N = r.n
    cover = np.zeros((N, N), np.int8)
    m = np.diff(T.leaf_off)
    for i, j in near:
        cover[T.leaf_off[i]:T.leaf_off[i + 1], T.leaf_off[j]:T.leaf_off[j + 1]] += 1
        assert T.touching(T.leaves[i], T.leaves[j])
    for s, t in far:
        a, b = T.nodes[s], T.nodes[t]
        cover[a.start:a.start + a.count, b.start:b.start + b.count] += 1
        assert not T.touching(s, t)
    # admissibility checked independently of touching(): the cell boxes of a
    # far pair, from the cube's origin and size, are apart on some axis by at
    # least the smaller cell, so the point sets are separated too
    assert far_pairs_separated(T, far)
    assert cover.min() == 1 and cover.max() == 1
    assert sorted(T.perm.tolist()) == list(range(N))
    assert m.max() <= 64
    # points lie inside their leaf cells
    for li, nid in enumerate(T.leaves):
        nd = T.nodes[nid]
        cell = T.size / 2 ** nd.level
        lo = T.origin + np.array(nd.ijk) * cell
        pts = r.centre[T.perm[nd.start:nd.start + nd.count]]
        assert np.all(pts >= lo - 1e-12) and np.all(pts <= lo + cell + 1e-12)


def test_eta_admissibility_closed_forms():
    """Eq. 10 with constant eta, min(diam) <= eta dist, on cells whose
    diagonals and gaps are known in closed form (diam = sqrt 3 edge):
    * two cells of edge c one cell apart diagonally: dist = sqrt 3 c = diam,
      far exactly when eta >= 1 (the tie at eta = 1 is far);
    * a face-neighbour of the neighbour (gap c along one axis): dist = c,
      far exactly when eta >= sqrt 3;
    * a cell of edge c one cell away from a cell of edge 2c: min diam is the
      small one's; touching cells are near for every eta."""
    import math
    from oracle.octree import MAX_DEPTH, Node

    def pair(cells, eta):
        T = Octree.__new__(Octree)
        T.eta = eta
        T.nodes = [Node(level, ijk, 0, 1) for level, ijk in cells]
        return not T.near_pair(0, 1)            # True = far

    diag = [(3, (0, 0, 0)), (3, (2, 2, 2))]
    assert pair(diag, 1.0) and not pair(diag, 1.0 - 1e-9)
    axis = [(3, (0, 0, 0)), (3, (2, 0, 0))]
    r3 = math.sqrt(3.0)
    assert pair(axis, r3 * (1 + 1e-12)) and not pair(axis, r3 * (1 - 1e-12))
    mixed = [(2, (0, 0, 0)), (3, (3, 0, 0))]     # big cell [0,2), small [3,4): gap 1 small edge
    assert pair(mixed, 2.0) and not pair(mixed, 1.7)
    touch = [(3, (0, 0, 0)), (3, (1, 1, 1))]
    assert not pair(touch, 1e6) and not pair(touch, 0.0)
    # eta = 0 is the plain non-touching test
    assert pair(axis, 0.0) and pair(diag, 0.0)
    assert MAX_DEPTH >= 3


def test_aca_bounds_and_exact_rank():
    rng = np.random.default_rng(3)
    # explicit rank-5 complex matrix is recovered to rounding
    A = rng.standard_normal((40, 5)) + 1j * rng.standard_normal((40, 5))
    Bm = rng.standard_normal((30, 5)) + 1j * rng.standard_normal((30, 5))
    M = A @ Bm.T
    U, V = aca(lambda i: M[i], lambda j: M[:, j], 40, 30, 1e-12)
    # the step after the exact rank adds a rounding-level term, then stops
    assert U.shape[1] in (5, 6)
    assert np.linalg.norm(M - U @ V.T) < 1e-10 * np.linalg.norm(M)
    U2, V2 = recompress(U, V, 1e-12)
    assert U2.shape[1] == 5 and np.linalg.norm(M - U2 @ V2.T) < 1e-10 * np.linalg.norm(M)
    # zero block -> rank 0
    Z = np.zeros((7, 9), np.complex128)
    U, V = aca(lambda i: Z[i], lambda j: Z[:, j], 7, 9, 1e-4)
    assert U.shape[1] == 0
    # EFIE far blocks: brute-force Frobenius error against the filled block
    v, f = icosphere(3, 0.5)
    r = build_rwg(v, f)
    E = EFIE(r)
    T = Octree(r.centre, 64)
    _, far = T.upper_blocks()
    P = T.perm
    for bi in (0, len(far) // 3, len(far) - 1):
        s, t = far[bi]
        rows = P[T.nodes[s].start:T.nodes[s].start + T.nodes[s].count]
        cols = P[T.nodes[t].start:T.nodes[t].start + T.nodes[t].count]
        U, V = aca(lambda i: E.block(rows[i:i + 1], cols)[0],
                   lambda j: E.block(rows, cols[j:j + 1])[:, 0], len(rows), len(cols), 1e-4)
        U, V = recompress(U, V, 1e-4)
        Zb = E.block(rows, cols)
        assert np.linalg.norm(Zb - U @ V.T) <= 3e-4 * np.linalg.norm(Zb)


def test_block_file_round_trip(tmp_path):
    from tests.oracle_cases import case
    from oracle.export import write_blocks, read_blocks
    _, H, S, _ = case("sphere_r0.25_L2")
    p = tmp_path / "h.hmps"
    write_blocks(str(p), H, S)
    d = read_blocks(str(p))
    assert d["N"] == H.N and np.array_equal(d["perm"], H.perm)
    assert all(np.array_equal(d["near"][k], H.near[k]) for k in H.near)
    assert len(d["far"]) == len(H.far)
    for a, b in zip(d["far"], H.far):
        assert a[:5] == b[:5] and np.array_equal(a[5], b[5])
    assert d["rows"] == S.rows
    assert all(np.array_equal(d["alpha"][k], S.alpha[k]) for k in S.alpha)


def test_c_entries_match_numpy():
    """oracle/cefie.c states the same EFIE entry as oracle/efie.py."""
    from oracle.cefie import CBlock
    v, f = icosphere(2, 0.5)
    r = build_rwg(v, f)
    E = EFIE(r)
    C = CBlock(E)
    rows = np.arange(0, r.n, 7)
    cols = np.arange(r.n)
    a = E.block(rows, cols)
    b = C(rows, cols)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    vp, fp = plate(1.0, 8)
    rp = build_rwg(vp, fp)
    Ep = EFIE(rp)
    a = Ep.block(np.arange(rp.n), np.arange(rp.n))
    assert np.abs(a - CBlock(Ep)(np.arange(rp.n), np.arange(rp.n))).max() < 1e-12 * np.abs(a).max()
