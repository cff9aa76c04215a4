"""Pins of the oracle's method: Schur-complement scaling (Eq. 14-23), the
power series (Eq. 30-36), the H-matrix against the dense matrix, and the EFIE
solution against the Mie series (Sec. V)."""
import numpy as np
import pytest

from oracle.hmatrix import HMatrix
from oracle.scaling import (compute_scaling, dense_R, symbolic_fill,
                            symbolic_fill_naive, near_pattern, apply_R, apply_Rt)
from oracle.series import series_solve, rel_err, refine_once, relative_residual
from oracle.rcs import (rcs, mie_bistatic, mie_backscatter, mie_amplitudes)
from tests.oracle_cases import case, plate_converging, dense_sphere_c1


def _sym_blocks(rng, m, pattern):
    """Random complex-symmetric block matrix with the given (i <= j) pattern;
    diagonal blocks made dominant so every Schur complement is invertible."""
    near = {}
    for (i, j) in pattern:
        Bk = rng.standard_normal((m[i], m[j])) + 1j * rng.standard_normal((m[i], m[j]))
        if i == j:
            Bk = 0.5 * (Bk + Bk.T) + 4 * m[i] * np.eye(m[i])
        near[(i, j)] = Bk
    return near


def _fake_h(m, near):
    off = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    return HMatrix(N=int(off[-1]), perm=np.arange(off[-1]), leaf_off=off, near=near, far=[])


def _dense_near(H):
    Z = np.zeros((H.N, H.N), np.complex128)
    for (i, j), Bk in H.near.items():
        si, sj = H.leaf_slice(i), H.leaf_slice(j)
        Z[si, sj] = Bk
        Z[sj, si] = Bk.T
    return Z


def test_four_block_example_eq14_21():
    """Fig. 1 / Eq. 14: blocks 1 and 4 far apart (Z_14 = 0)."""
    rng = np.random.default_rng(14)
    m = [3, 4, 2, 5]
    pat = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
    H = _fake_h(m, _sym_blocks(rng, m, pat))
    Z = {k: v for k, v in H.near.items()}
    T = lambda i, j: Z[(i, j)] if i <= j else Z[(j, i)].T
    S = compute_scaling(H, "A")
    assert S.rows == [[1, 2], [2, 3], [3], []]
    # Eq. 16: alpha_1j = -Z_11^{-1} Z_1j
    for j in (1, 2):
        assert np.allclose(S.alpha[(0, j)], -np.linalg.solve(T(0, 0), T(0, j)), atol=1e-13)
    # Eq. 21: Schur complement of block 1; rows/cols of block 4 untouched
    Z22 = T(1, 1) - T(1, 0) @ np.linalg.solve(T(0, 0), T(0, 1))
    Z23 = T(1, 2) - T(1, 0) @ np.linalg.solve(T(0, 0), T(0, 2))
    assert np.allclose(S.D[1], Z22, atol=1e-12)
    assert np.allclose(S.alpha[(1, 2)], -np.linalg.solve(Z22, Z23), atol=1e-12)
    assert np.allclose(S.alpha[(1, 3)], -np.linalg.solve(Z22, T(1, 3)), atol=1e-12)
    # Eq. 19-20 with the dense alpha_1 and alpha'_1 = alpha_1^T (Eq. 15-18)
    ZN = _dense_near(H)
    A1 = np.eye(H.N, dtype=complex)
    A1[0:3, 3:7] = S.alpha[(0, 1)]
    A1[0:3, 7:9] = S.alpha[(0, 2)]
    Z1 = A1.T @ ZN @ A1
    assert np.abs(Z1[0:3, 3:]).max() < 1e-12 and np.abs(Z1[3:, 0:3]).max() < 1e-12
    assert np.allclose(Z1[0:3, 0:3], T(0, 0))
    assert np.array_equal(Z1[9:, 9:], ZN[9:, 9:])
    assert np.allclose(Z1[3:7, 3:7], Z22, atol=1e-12)
    # Eq. 22-23: full sequence is block diagonal
    R = dense_R(S, H.leaf_off)
    M = R.T @ ZN @ R
    D = np.zeros_like(M)
    for k in range(4):
        D[H.leaf_slice(k), H.leaf_slice(k)] = S.D[k]
    assert np.abs(M - D).max() < 1e-12 * np.abs(M).max()


def test_sweeps_equal_dense_R():
    rng = np.random.default_rng(5)
    m = [2, 3, 1, 4, 2, 3]
    pat = [(i, i) for i in range(6)] + [(0, 2), (0, 4), (1, 3), (2, 5), (3, 4), (1, 5)]
    H = _fake_h(m, _sym_blocks(rng, m, pat))
    S = compute_scaling(H, "A")
    R = dense_R(S, H.leaf_off)
    x = rng.standard_normal((H.N, 3)) + 1j * rng.standard_normal((H.N, 3))
    assert np.allclose(apply_R(S, H.leaf_off, x), R @ x, atol=1e-12)
    assert np.allclose(apply_Rt(S, H.leaf_off, x), R.T @ x, atol=1e-12)


def test_symbolic_fill_etree_equals_naive():
    _, H, _, _ = case("sphere_r0.5_L3")
    pairs = list(H.near.keys())
    assert symbolic_fill(H.n_leaves, pairs) == symbolic_fill_naive(H.n_leaves, pairs)


def test_reading_A_block_diagonal_and_reading_B_pattern():
    _, H, S, _ = case("sphere_r0.25_L2")
    ZN = _dense_near(H)
    R = dense_R(S, H.leaf_off)
    M = R.T @ ZN @ R
    D = np.zeros_like(M)
    for k in range(S.n):
        D[H.leaf_slice(k), H.leaf_slice(k)] = S.D[k]
    assert np.abs(M - D).max() < 1e-11 * np.abs(M).max()
    SB = compute_scaling(H, "B")
    assert SB.rows == [sorted(r) for r in near_pattern(H.n_leaves, H.near.keys())]
    RB = dense_R(SB, H.leaf_off)
    MB = RB.T @ ZN @ RB
    assert np.abs(MB - D).max() > 1e-6 * np.abs(M).max()     # dropped fill shows


def test_series_special_cases():
    rng = np.random.default_rng(7)
    m = [4, 3, 5]
    H = _fake_h(m, _sym_blocks(rng, m, [(0, 0), (0, 1), (1, 1), (1, 2), (2, 2)]))
    S = compute_scaling(H, "A")
    b = rng.standard_normal((H.N, 2)) + 1j * rng.standard_normal((H.N, 2))
    x, _ = series_solve(H, S, b, 2)                      # Z_F = 0 -> exact
    assert np.allclose(x, np.linalg.solve(_dense_near(H), b), atol=1e-12, rtol=0)
    # a single leaf: D^{-1} b = Z^{-1} b
    H1 = _fake_h([6], _sym_blocks(rng, [6], [(0, 0)]))
    S1 = compute_scaling(H1, "A")
    b1 = rng.standard_normal(6) + 0j
    assert np.allclose(S1.Dinv[0] @ b1, np.linalg.solve(H1.near[(0, 0)], b1), atol=1e-13)


def test_series_many_terms_converges_to_lu():
    H, S, B = plate_converging()
    Zh = H.to_dense()
    x_lu = np.linalg.solve(Zh, B[H.perm])
    X = np.empty_like(x_lu)
    X[H.perm] = x_lu
    x2, r2 = series_solve(H, S, B, 2)
    x40, r40 = series_solve(H, S, B, 40)
    assert np.all(rel_err(x40, X) < 1e-10)
    assert np.all(rel_err(x2, X) < 0.5)
    assert np.all(r2[0] < 1.0)
    # one FP64 refinement step lowers the error of the two-term result
    xr = refine_once(H, S, B, x2)
    assert np.all(rel_err(xr, X) < rel_err(x2, X))
    assert np.all(relative_residual(H, B, xr) < relative_residual(H, B, x2))


def test_hmatrix_vs_dense_and_symmetry():
    r, E, Zd, B = dense_sphere_c1()
    _, H, _, _ = case("sphere_r0.5_L3")
    Zh = H.to_dense()
    Zp = Zd[np.ix_(H.perm, H.perm)]
    assert np.array_equal(Zh, Zh.T)
    err = np.linalg.norm(Zh - Zp) / np.linalg.norm(Zp)
    assert err < 3e-4
    # near blocks are the EFIE entries themselves
    for (i, j) in list(H.near.keys())[::17]:
        si, sj = H.leaf_slice(i), H.leaf_slice(j)
        assert np.allclose(H.near[(i, j)], Zp[si, sj], rtol=0, atol=1e-12 * np.abs(Zp).max())


def test_mie_limits_and_optical_theorem():
    a = 0.5
    for x in (1e-3, 1e-2):
        k = x / a
        assert abs(mie_backscatter(a, k) / (9 * np.pi * a * a * x ** 4) - 1) < 1e-3
    assert abs(mie_backscatter(a, 400.0) / (np.pi * a * a) - 1) < 1e-3
    k = 2 * np.pi
    g = np.linspace(0, np.pi, 6001)
    S1, S2 = mie_amplitudes(k * a, g)
    sca = np.pi / k ** 2 * np.trapezoid((abs(S1) ** 2 + abs(S2) ** 2) * np.sin(g), g)
    S10, _ = mie_amplitudes(k * a, np.array([0.0]))
    assert abs(sca / (4 * np.pi / k ** 2 * S10.real[0]) - 1) < 1e-5
    assert np.isclose(mie_bistatic(a, k, np.pi, "E"), mie_backscatter(a, k))


def test_efie_lu_solution_matches_mie():
    """0.5 lambda PEC sphere, 1920 RWG unknowns: dense LU currents give the
    bistatic E-plane RCS of the Mie series within 0.5 dB (incidence theta=0)."""
    r, E, Zd, B = dense_sphere_c1()
    x = np.linalg.solve(Zd, B)
    th = np.radians(np.arange(0.0, 181.0, 5.0))
    s = rcs(r, E.k, x, th, 0.0, "theta")[:, 0]
    m = mie_bistatic(0.5, E.k, np.pi - th, "E")
    db = 10 * np.log10(s / m)
    assert np.abs(db).max() < 0.5, db


def test_two_term_error_reported_config1():
    """Paper's error metric ||x_LU - x_ps|| / ||x_LU|| (Sec. V-A) on the
    0.5 lambda sphere with leaves <= 64 unknowns; the value is reported, not
    pinned (the paper prints none); the ratio of Eq. 45 is above 0.1 there."""
    r, E, Zd, B = dense_sphere_c1()
    _, H, S, Bw = case("sphere_r0.5_L3")
    x_lu = np.linalg.solve(Zd, B)
    x2, ratio = series_solve(H, S, Bw, 2)
    err = float(rel_err(x2, x_lu)[0])
    # series residual against the dense matrix, ||Z x - b|| / ||b||
    res = float(np.linalg.norm(Zd @ x2[:, 0] - B[:, 0]) / np.linalg.norm(B[:, 0]))
    print(f"two-term error vs LU {err:.3f}, residual {res:.3f}, ratio {float(ratio[0, 0]):.3f}")
    assert np.isfinite(err) and np.isfinite(res) and ratio.shape == (1, 1)
    # the LU solution itself leaves a rounding-level residual
    assert np.linalg.norm(Zd @ x_lu[:, 0] - B[:, 0]) < 1e-10 * np.linalg.norm(B[:, 0])


def test_nested_dissection_order_same_solution():
    """Reading A makes x = Z_N^-1 b - Z_N^-1 Z_F Z_N^-1 b independent of the
    elimination order (R D^-1 R^T = Z_N^-1); nested dissection reduces fill."""
    from oracle.scaling import nd_order
    w, H, S, B = case("sphere_r0.5_L3")
    order = nd_order(H.tree, list(H.near.keys()))
    assert sorted(order) == list(range(H.n_leaves))
    S2 = compute_scaling(H, "A", order)
    x1, r1 = series_solve(H, S, B, 2)
    x2, r2 = series_solve(H, S2, B, 2)
    assert np.all(rel_err(x2, x1) < 1e-11)
    assert S2.entries(H.leaf_off)[0] < S.entries(H.leaf_off)[0]
    ZN = _dense_near(H)
    R = dense_R(S2, H.leaf_off)
    M = R.T @ ZN @ R
    for k, sk in enumerate(S2.slices(H.leaf_off)):
        assert np.allclose(M[sk, sk], S2.D[k], atol=1e-11 * np.abs(M).max())


def test_phi_polarised_wave_matches_mie_h_plane():
    """The phi-polarised wave from theta = 0, phi = 0 is y-polarised, so the
    xz-plane is its H-plane: the phi component of the bistatic RCS there
    follows the Mie series' S1 pattern (0.5 dB)."""
    r, E, Zd, _ = dense_sphere_c1()
    b = E.plane_wave([0.0], [0.0], [1])
    x = np.linalg.solve(Zd, b)
    th = np.radians(np.arange(0.0, 181.0, 5.0))
    s = rcs(r, E.k, x, th, 0.0, "phi")[:, 0]
    m = mie_bistatic(0.5, E.k, np.pi - th, "H")
    db = 10 * np.log10(s / m)
    assert np.abs(db).max() < 0.5, db


def test_adaptive_term_count_follows_tolerance():
    """Adaptive term count (Sec. III-C, Eq. 44-45) on the converging plate
    (ratio about 0.4): the error against the LU solution of the assembled
    H-matrix follows the tolerance, with more terms for a tighter one; on
    the 0.5 lambda sphere, where the terms eventually grow (spectral radius
    above one), the series stops at the first growing term, long before the cap."""
    H, S, B = plate_converging()
    x_lu = np.linalg.solve(H.to_dense(), B[H.perm])
    X = np.empty_like(x_lu)
    X[H.perm] = x_lu
    terms = []
    for tol in (1e-3, 1e-6, 1e-10):
        x, ratios = series_solve(H, S, B, 60, term_tol=tol)
        terms.append(len(ratios) + 1)
        assert np.all(rel_err(x, X) < 10 * tol), (tol, rel_err(x, X))
        assert np.all(ratios < 1.0)
    assert terms[0] < terms[1] < terms[2] < 60
    w, Hs, Ss, Bs = case("sphere_r0.5_L3")
    with np.errstate(all="ignore"):
        x, ratios = series_solve(Hs, Ss, Bs, 60, term_tol=1e-8)
    assert len(ratios) + 1 < 60
    assert np.any(ratios[-1] >= 1.0) and np.all(ratios[:-1] < 1.0)
