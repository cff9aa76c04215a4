"""MFIE / CFIE (Sec. II, Eq. 4-8) and the non-symmetric scaling and series
(Sec. III without Z = Z^T) in the oracle, CPU only.

Pins: the closed-form static kernel of the MFIE against brute force and
against the gradient of the 1/R potential; the MFIE of a plane equal to half
the Gram matrix of an independent exact rule (K vanishes between coplanar
triangles); outward normals; MFIE and CFIE currents of a PEC sphere against
the Mie series; the CFIE free of the interior resonance that makes the EFIE
and MFIE matrices nearly singular; the non-symmetric scaling equal to the
symmetric one on a symmetric matrix, block-diagonalising the CFIE near field,
and its series reaching Z_N^-1 b, Z^-1 b and the LU solution in the limits
where the method is exact."""
import functools
import math

import numpy as np

import hm_workloads as hw
from oracle.efie import EFIE
from oracle.mfie import CFIE, MFIE
from oracle.nonsym import (apply_L, build_hmatrix_general, compute_scaling_general, dense_L,
                           from_symmetric, series_solve_general)
from oracle.potentials import gradient_brute, static_gradient, static_potentials
from oracle.rcs import mie_bistatic, rcs
from oracle.rwg import build_rwg
from oracle.scaling import compute_scaling, dense_R
from oracle.series import series_solve
from tests.oracle_cases import case


def test_static_gradient_closed_form():
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.9, 0.0]])
    pts = [[0.4, 0.3, 0.5], [0.4, 0.3, -0.2], [1.5, 1.2, 0.3], [0.2, -0.5, 0.05],
           [2.0, 2.0, 0.0], [0.5, 0.05, 0.02]]
    for p in pts:
        got = static_gradient(np.array([p]), tri[None])[0]
        ref = gradient_brute(p, tri, order=300)
        assert np.abs(got - ref).max() <= 1e-7 * np.abs(ref).max(), (p, got, ref)
        # minus the gradient of int 1/R (central differences)
        h = 1e-5
        fd = np.zeros(3)
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            ip = static_potentials(np.array([np.add(p, e)]), tri[None])[0][0]
            im = static_potentials(np.array([np.subtract(p, e)]), tri[None])[0][0]
            fd[c] = -(ip - im) / (2 * h)
        assert np.abs(got - fd).max() <= 1e-6 * np.abs(got).max(), (p, got, fd)


def _gram_midpoint(rwg):
    """<f_m, f_n> by the three-edge-midpoint rule (exact for quadratics)."""
    N = rwg.n
    G = np.zeros((N, N))
    parts = []
    for s, tr, fr in ((1.0, rwg.tri_p, rwg.free_p), (-1.0, rwg.tri_m, rwg.free_m)):
        parts.append((s, tr, rwg.verts[rwg.tris[tr, fr]]))
    for sa, ta, va in parts:
        for sb, tb, vb in parts:
            for m in range(N):
                same = np.nonzero(tb == ta[m])[0]
                for n in same:
                    T = rwg.verts[rwg.tris[ta[m]]]
                    mids = 0.5 * (T + np.roll(T, -1, axis=0))
                    A = rwg.area[ta[m]]
                    val = sum(np.dot(q - va[m], q - vb[n]) for q in mids) * A / 3.0
                    G[m, n] += (sa * sb * rwg.length[m] * rwg.length[n]
                                / (4.0 * A * A)) * val
    return G


def test_mfie_of_a_plane_is_half_the_gram_matrix():
    v, f = hw.plate(1.0, 5)
    r = build_rwg(v, f)
    M = MFIE(r, 1.0).dense()
    G = _gram_midpoint(r)
    assert np.abs(M - 0.5 * G).max() <= 1e-12 * np.abs(G).max()


def test_closed_meshes_have_outward_normals():
    meshes = [hw.icosphere(3, 0.5), hw.ellipsoid(3, (1.0, 0.6, 0.4)),
              hw.closed_cylinder(0.5, 1.0, 0.1)]
    for v, f in meshes:
        M = MFIE(build_rwg(v, f), 1.0)
        c = M.tv.mean(axis=1)
        inside = v.mean(axis=0)
        assert np.all(np.einsum("tc,tc->t", M.nrm, c - inside) > 0)


@functools.lru_cache(maxsize=None)
def _sphere05():
    v, f = hw.icosphere(3, 0.5)
    r = build_rwg(v, f)
    E, M = EFIE(r, 1.0), MFIE(r, 1.0)
    return r, E, M, E.dense(), M.dense()


def test_mfie_and_cfie_currents_match_mie():
    """0.5 lambda sphere, 1920 unknowns, waves from theta = 0: bistatic RCS of
    the MFIE and CFIE (alpha = 0.5) currents within 0.5 dB of the Mie series
    (as the EFIE's), x-polarised in its E-plane and y-polarised in its
    H-plane; the MFIE is not symmetric."""
    r, E, M, Ze, Zm = _sphere05()
    assert np.abs(Zm - Zm.T).max() > 1e-4 * np.abs(Zm).max()
    th = np.radians(np.arange(0.0, 181.0, 5.0))
    mie = mie_bistatic(0.5, E.k, np.pi - th, "E")
    bm = M.plane_wave([0.0], [0.0], [0])
    be = E.plane_wave([0.0], [0.0], [0])
    for Z, b in ((Zm, bm), (0.5 * Ze + 0.5 * M.eta * Zm, 0.5 * be + 0.5 * M.eta * bm)):
        x = np.linalg.solve(Z, b)
        db = 10 * np.log10(rcs(r, E.k, x, th, 0.0, "theta")[:, 0] / mie)
        assert np.abs(db).max() < 0.5, db
    # the phi-polarised (y) wave: the xz-plane is its H-plane (Mie S1 pattern)
    mie_h = mie_bistatic(0.5, E.k, np.pi - th, "H")
    bm1 = M.plane_wave([0.0], [0.0], [1])
    be1 = E.plane_wave([0.0], [0.0], [1])
    for Z, b in ((Zm, bm1), (0.5 * Ze + 0.5 * M.eta * Zm, 0.5 * be1 + 0.5 * M.eta * bm1)):
        x = np.linalg.solve(Z, b)
        db = 10 * np.log10(rcs(r, E.k, x, th, 0.0, "phi")[:, 0] / mie_h)
        assert np.abs(db).max() < 0.5, db
    # the CFIE class assembles the same system
    C = CFIE(r, 1.0, 0.5)
    rows = np.arange(0, r.n, 97)
    Zc = 0.5 * Ze + 0.5 * M.eta * Zm
    blk = C.block(rows, np.arange(r.n))
    assert np.abs(blk - Zc[rows]).max() <= 1e-12 * np.abs(Zc).max() * 10
    assert np.allclose(C.plane_wave([0.0], [0.0], [0]), 0.5 * be + 0.5 * M.eta * bm)


def test_cfie_has_no_interior_resonance():
    """Sphere of 480 unknowns near its first interior resonance (ka = 2.744;
    the faceted mesh resonates at ka = 2.79): the smallest singular value of
    the EFIE and MFIE matrices (relative to the largest) falls 4x and 10x
    below its value at ka = 2.2, the CFIE's does not fall."""
    out = {}
    for ka in (2.2, 2.79):
        v, f = hw.icosphere(2, 0.5)
        r = build_rwg(v, f)
        wl = 2 * math.pi * 0.5 / ka
        E, M = EFIE(r, wl), MFIE(r, wl)
        Ze, Zm = E.dense(), M.eta * M.dense()
        q = []
        for Z in (Ze, Zm, 0.5 * Ze + 0.5 * Zm):
            sv = np.linalg.svd(Z, compute_uv=False)
            q.append(sv[-1] / sv[0])
        out[ka] = q
    (e0, m0, c0), (e1, m1, c1) = out[2.2], out[2.79]
    assert e1 < e0 / 4 and m1 < m0 / 10, out
    assert c1 > 0.8 * c0 and c1 > 0.2, out


def test_general_scaling_reduces_to_the_symmetric_one():
    w, H, S, B = case("sphere_r0.5_L3")
    G = from_symmetric(H)
    SG = compute_scaling_general(G, "A")
    sa = max(np.abs(a).max() for a in S.alpha.values())
    assert max(np.abs(SG.alphaL[kj] - S.alpha[kj].T).max() for kj in S.alpha) <= 1e-12 * sa
    assert max(np.abs(SG.alpha[kj] - S.alpha[kj]).max() for kj in S.alpha) <= 1e-12 * sa
    sd = max(np.abs(d).max() for d in S.D)
    assert max(np.abs(a - b).max() for a, b in zip(SG.D, S.D)) <= 1e-12 * sd
    x1, r1 = series_solve(H, S, B, 3)
    x2, r2 = series_solve_general(G, SG, B, 3)
    assert np.abs(x1 - x2).max() <= 1e-12 * np.abs(x1).max()
    assert np.allclose(r1, r2, rtol=1e-12)
    # reading B (fill kept to the near pattern) reduces the same way
    SB = compute_scaling(H, "B")
    SGB = compute_scaling_general(G, "B")
    assert SGB.rows == SB.rows
    sb = max(np.abs(a).max() for a in SB.alpha.values())
    assert max(np.abs(SGB.alphaL[kj] - SB.alpha[kj].T).max() for kj in SB.alpha) <= 1e-12 * sb
    assert max(np.abs(a - b).max() for a, b in zip(SGB.D, SB.D)) <= 1e-12 * sd


@functools.lru_cache(maxsize=None)
def _cfie_small():
    v, f = hw.icosphere(2, 0.25)
    H = build_hmatrix_general(v, f, lambda r: CFIE(r, 1.0, 0.5), leaf_max=32, compress="svd")
    S = compute_scaling_general(H, "A")
    b = CFIE(H.rwg, 1.0, 0.5).plane_wave([0.0, 1.0], [0.0, 0.5], [0, 1])
    return v, f, H, S, b


def test_cfie_scaling_block_diagonalises_the_near_field():
    v, f, H, S, b = _cfie_small()
    L, R = dense_L(S, H.leaf_off), dense_R(S, H.leaf_off)
    m = np.diff(H.leaf_off)[S.order]
    idx = np.concatenate([np.arange(H.leaf_off[l], H.leaf_off[l + 1]) for l in S.order])
    Dm = (L @ H.to_dense(far=False) @ R)[np.ix_(idx, idx)]
    o = np.concatenate([[0], np.cumsum(m)])
    scale = np.abs(Dm).max()
    for k in range(S.n):
        blk = Dm[o[k]:o[k + 1], o[k]:o[k + 1]]
        assert np.abs(blk - S.D[k]).max() <= 1e-12 * scale
        Dm[o[k]:o[k + 1], o[k]:o[k + 1]] = 0.0
    assert np.abs(Dm).max() <= 1e-12 * scale
    # the left factor is not the transpose of the right one here: a plausible
    # mistake (L = R^T, the symmetric shortcut) leaves the near field coupled
    Dbad = (R.T @ H.to_dense(far=False) @ R)[np.ix_(idx, idx)]
    for k in range(S.n):
        Dbad[o[k]:o[k + 1], o[k]:o[k + 1]] = 0.0
    assert np.abs(Dbad).max() > 1e-3 * scale
    # forward substitution equals the dense factor
    assert np.abs(apply_L(S, H.leaf_off, b[H.perm]) - L @ b[H.perm]).max() <= \
        1e-12 * np.abs(L @ b[H.perm]).max()


def test_cfie_series_limits():
    """Z_F = 0 -> the two-term series is Z_N^-1 b; many terms -> the LU
    solution of the assembled CFIE H-matrix (the ratio of Eq. 45 is below
    one here); one leaf -> D^-1 b = Z^-1 b."""
    import copy
    v, f, H, S, b = _cfie_small()
    H0 = copy.copy(H)
    H0.far = []
    x0, _ = series_solve_general(H0, S, b, 2)
    xn = np.linalg.solve(H.to_dense(far=False), b[H.perm])
    X = np.empty_like(xn)
    X[H.perm] = xn
    assert np.abs(x0 - X).max() <= 1e-10 * np.abs(X).max()
    xl = np.linalg.solve(H.to_dense(), b[H.perm])
    XL = np.empty_like(xl)
    XL[H.perm] = xl
    xs, ratios = series_solve_general(H, S, b, 40)
    assert ratios[0].max() < 1.0
    assert np.linalg.norm(xs - XL) <= 1e-9 * np.linalg.norm(XL)
    x2, _ = series_solve_general(H, S, b, 2)
    assert np.linalg.norm(x2 - XL) > 1e-3 * np.linalg.norm(XL)     # truncation visible
    H1 = build_hmatrix_general(v, f, lambda r: CFIE(r, 1.0, 0.5), leaf_max=10 ** 6)
    assert H1.n_leaves == 1 and H1.far == []
    S1 = compute_scaling_general(H1, "A")
    x1, r1 = series_solve_general(H1, S1, b, 2)
    xl1 = np.linalg.solve(H1.to_dense(), b[H1.perm])
    X1 = np.empty_like(xl1)
    X1[H1.perm] = xl1
    assert np.abs(x1 - X1).max() <= 1e-10 * np.abs(X1).max() and np.all(r1 == 0.0)


def test_dense_fill_and_hmatrix_from_dense():
    """The study path (one dense CFIE fill, by a spawned pool or serially,
    then each cap's H-matrix cut from it) gives the same matrix and blocks
    as the block-by-block build."""
    from oracle.nonsym import dense_cfie, hmatrix_from_dense
    v, f = hw.icosphere(2, 0.25)
    r, Z1 = dense_cfie(v, f, 1.0, 0.5, processes=1)
    _, Z2 = dense_cfie(v, f, 1.0, 0.5, processes=2)
    scale = np.abs(Z1).max()
    assert np.abs(Z1 - Z2).max() <= 1e-13 * scale
    H = hmatrix_from_dense(Z1, r, 32)
    _, _, Hb, _, _ = _cfie_small()
    assert sorted(H.near) == sorted(Hb.near)
    assert max(np.abs(H.near[k] - Hb.near[k]).max() for k in H.near) <= 1e-12 * scale
    assert [x[:5] for x in H.far] == [x[:5] for x in Hb.far]
    assert np.abs(H.to_dense() - Hb.to_dense()).max() <= 1e-12 * scale
    # the far blocks keep the SVD tolerance against the full matrix
    Zp = Z1[np.ix_(H.perm, H.perm)]
    assert np.linalg.norm(H.to_dense() - Zp) <= 1e-4 * np.linalg.norm(Zp)


def test_nonsym_block_file_round_trip():
    """The block file of a non-symmetric system (NONSYM01 section) gives back
    every ordered near and far block and both sets of coefficients."""
    import os
    import tempfile
    from oracle.export import read_blocks, write_blocks_nonsym
    v, f, H, S, b = _cfie_small()
    fd, path = tempfile.mkstemp(suffix=".hmps")
    os.close(fd)
    try:
        write_blocks_nonsym(path, H, S)
        d = read_blocks(path)
        assert d.get("nonsym") and sorted(d["near"]) == sorted(H.near)
        assert all(np.array_equal(d["near"][k], H.near[k]) for k in H.near)
        key = lambda x: (x[1], x[3])
        fa, fb = sorted(d["far"], key=key), sorted(H.far, key=key)
        assert [x[:5] for x in fa] == [x[:5] for x in fb]
        assert all(np.array_equal(x[5], y[5]) for x, y in zip(fa, fb))
        assert d["rows"] == S.rows and d["elim"] == S.order
        assert all(np.array_equal(d["alpha"][kj], S.alpha[kj]) for kj in S.alpha)
        assert all(np.array_equal(d["alphaL"][kj], S.alphaL[kj]) for kj in S.alphaL)
    finally:
        os.unlink(path)
