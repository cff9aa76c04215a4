"""Mutation checks of the oracle's pins.

Each case copies the source of one oracle module, plants one plausible mistake
in the copy (a wrong sign, a dropped term, a transposed or conjugated operand,
a stale operand, a swapped constant, an off-by-one comparison), loads the copy
as a module of its own and shows that the pin written for that part of the
method rejects it, while the unmodified module passes the same check.  The
committed oracle is never changed; the mutants live only in this process.
"""
import math
import os
import sys
import types

import numpy as np
import pytest

import oracle
from oracle.hmatrix import HMatrix
from tests.oracle_cases import plate_converging, dense_sphere_c1
from tests.test_oracle_basics import far_pairs_separated

ORACLE_DIR = os.path.dirname(oracle.__file__)


def load(modname, old=None, new=None):
    """oracle.<modname> executed from its source, with `old` replaced by `new`
    (exactly one occurrence) when given."""
    path = os.path.join(ORACLE_DIR, modname + ".py")
    with open(path) as f:
        src = f.read()
    tag = "orig"
    if old is not None:
        assert src.count(old) == 1, (modname, old)
        src = src.replace(old, new)
        tag = f"mut{abs(hash((old, new))) % 10 ** 8}"
    name = f"oracle._{tag}_{modname}"
    mod = types.ModuleType(name)
    mod.__package__ = "oracle"
    mod.__file__ = path
    sys.modules[name] = mod          # dataclasses look their module up
    exec(compile(src, f"{path} ({tag})", "exec"), mod.__dict__)
    return mod


# ----------------------------------------------------------------- the pins
def pin_quadrature(q):
    """Degree-5 exactness on the reference triangle, weights summing to 1."""
    pts, w = q.dunavant7()
    x, y = pts[:, 1], pts[:, 2]
    for a in range(6):
        for b in range(6 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            if abs(0.5 * np.sum(w * x ** a * y ** b) - exact) >= 1e-15:
                return False
    return abs(w.sum() - 1.0) < 1e-15


def pin_potentials(pm):
    """Closed-form static potentials against Duffy-transformed brute force."""
    from oracle.potentials import duffy_brute
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.0]])
    for obs in ((0.4, 0.3, 0.05), (1.3, 0.9, 0.02), (-0.4, -0.02, 0.0), (3.0, -2.0, 1.0)):
        Is, Iv, _ = pm.static_potentials(np.array([obs]), tri[None])
        bs, bv = duffy_brute(np.array(obs), tri, order=64)
        if not (abs(Is[0] - bs) < 1e-10 * max(1.0, abs(bs)) and np.abs(Iv[0] - bv).max() < 1e-10):
            return False
    return True


def _mie_db(r, k, x):
    from oracle.rcs import rcs, mie_bistatic
    th = np.radians(np.arange(0.0, 181.0, 5.0))
    s = rcs(r, k, x, th, 0.0, "theta")[:, 0]
    return 10 * np.log10(s / mie_bistatic(0.5, k, np.pi - th, "E"))


def pin_efie(ef):
    """Dense-LU currents of the 0.5 lambda sphere against the Mie series (0.5 dB)."""
    r, E0, Zd, B = dense_sphere_c1()
    if ef is None:
        Z, b = Zd, B
    else:
        E = ef.EFIE(r, 1.0)
        Z, b = E.dense(), E.plane_wave([0.0], [0.0], [0])
    return bool(np.abs(_mie_db(r, E0.k, np.linalg.solve(Z, b))).max() < 0.5)


def pin_plane_wave(ef):
    """The same Mie comparison with the filled Z and the module's excitation."""
    r, E0, Zd, _ = dense_sphere_c1()
    b = ef.EFIE(r, 1.0).plane_wave([0.0], [0.0], [0])
    return bool(np.abs(_mie_db(r, E0.k, np.linalg.solve(Zd, b))).max() < 0.5)


def pin_phi_polarisation(ef):
    """The phi-polarised wave from theta = 0 (y-polarised) against the Mie
    series' H-plane pattern in the xz-plane."""
    from oracle.rcs import rcs, mie_bistatic
    r, E0, Zd, _ = dense_sphere_c1()
    b = ef.EFIE(r, 1.0).plane_wave([0.0], [0.0], [1])
    th = np.radians(np.arange(0.0, 181.0, 5.0))
    s = rcs(r, E0.k, np.linalg.solve(Zd, b), th, 0.0, "phi")[:, 0]
    return bool(np.abs(10 * np.log10(s / mie_bistatic(0.5, E0.k, np.pi - th, "H"))).max() < 0.5)


def pin_rcs(rc):
    """Monostatic sweep RCS of the LU currents against the Mie series."""
    r, E0, Zd, B = dense_sphere_c1()
    x = np.linalg.solve(Zd, B)
    th = np.radians(np.arange(0.0, 181.0, 5.0))
    s = rc.rcs(r, E0.k, x, th, 0.0, "theta")[:, 0]
    from oracle.rcs import mie_bistatic
    return bool(np.abs(10 * np.log10(s / mie_bistatic(0.5, E0.k, np.pi - th, "E"))).max() < 0.5)


def pin_mie(rc):
    """Rayleigh limit, optical limit and the optical theorem."""
    a = 0.5
    for x in (1e-3, 1e-2):
        k = x / a
        if not abs(rc.mie_backscatter(a, k) / (9 * np.pi * a * a * x ** 4) - 1) < 1e-3:
            return False
    if not abs(rc.mie_backscatter(a, 400.0) / (np.pi * a * a) - 1) < 1e-3:
        return False
    k = 2 * np.pi
    g = np.linspace(0, np.pi, 6001)
    S1, S2 = rc.mie_amplitudes(k * a, g)
    sca = np.pi / k ** 2 * np.trapezoid((abs(S1) ** 2 + abs(S2) ** 2) * np.sin(g), g)
    S10, _ = rc.mie_amplitudes(k * a, np.array([0.0]))
    return abs(sca / (4 * np.pi / k ** 2 * S10.real[0]) - 1) < 1e-5


def pin_octree(oc):
    """Near and far blocks tile N x N once; far pairs geometrically separated."""
    from hm_workloads import icosphere
    from oracle.rwg import build_rwg
    v, f = icosphere(3, 0.5)
    r = build_rwg(v, f)
    T = oc.Octree(r.centre, 64)
    near, far = T.blocks()
    cover = np.zeros((r.n, r.n), np.int8)
    for i, j in near:
        cover[T.leaf_off[i]:T.leaf_off[i + 1], T.leaf_off[j]:T.leaf_off[j + 1]] += 1
    for s, t in far:
        a, b = T.nodes[s], T.nodes[t]
        cover[a.start:a.start + a.count, b.start:b.start + b.count] += 1
    return bool(cover.min() == 1 and cover.max() == 1 and far_pairs_separated(T, far))


def pin_aca(ac):
    """Exact recovery of a rank-5 complex matrix, before and after recompression."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 5)) + 1j * rng.standard_normal((40, 5))
    Bm = rng.standard_normal((30, 5)) + 1j * rng.standard_normal((30, 5))
    M = A @ Bm.T
    U, V = ac.aca(lambda i: M[i], lambda j: M[:, j], 40, 30, 1e-12)
    if not np.linalg.norm(M - U @ V.T) < 1e-10 * np.linalg.norm(M):
        return False
    U2, V2 = ac.recompress(U, V, 1e-12)
    return U2.shape[1] == 5 and np.linalg.norm(M - U2 @ V2.T) < 1e-10 * np.linalg.norm(M)


def _sym_case(seed, m, pattern):
    rng = np.random.default_rng(seed)
    near = {}
    for (i, j) in pattern:
        Bk = rng.standard_normal((m[i], m[j])) + 1j * rng.standard_normal((m[i], m[j]))
        if i == j:
            Bk = 0.5 * (Bk + Bk.T) + 4 * m[i] * np.eye(m[i])
        near[(i, j)] = Bk
    off = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    H = HMatrix(N=int(off[-1]), perm=np.arange(off[-1]), leaf_off=off, near=near, far=[])
    Z = np.zeros((H.N, H.N), np.complex128)
    for (i, j), Bk in near.items():
        si, sj = H.leaf_slice(i), H.leaf_slice(j)
        Z[si, sj] = Bk
        Z[sj, si] = Bk.T
    return rng, H, Z


def pin_scaling(sc):
    """R^T Z_N R = blockdiag(D) (Eq. 23) on the four-block example of Eq. 14."""
    pat = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
    _, H, Z = _sym_case(14, [3, 4, 2, 5], pat)
    S = sc.compute_scaling(H, "A")
    R = sc.dense_R(S, H.leaf_off)
    M = R.T @ Z @ R
    D = np.zeros_like(M)
    for k in range(S.n):
        D[H.leaf_slice(k), H.leaf_slice(k)] = S.D[k]
    return bool(np.abs(M - D).max() < 1e-12 * np.abs(M).max())


def pin_sweeps(sc):
    """Block substitutions equal the dense R and R^T (Eq. 25-26)."""
    pat = [(i, i) for i in range(6)] + [(0, 2), (0, 4), (1, 3), (2, 5), (3, 4), (1, 5)]
    rng, H, _ = _sym_case(5, [2, 3, 1, 4, 2, 3], pat)
    S = sc.compute_scaling(H, "A")
    R = sc.dense_R(S, H.leaf_off)
    x = rng.standard_normal((H.N, 3)) + 1j * rng.standard_normal((H.N, 3))
    return bool(np.allclose(sc.apply_R(S, H.leaf_off, x), R @ x, atol=1e-12) and
                np.allclose(sc.apply_Rt(S, H.leaf_off, x), R.T @ x, atol=1e-12))


def pin_supernodes(sc):
    """T_G b_G equals the forward substitution (Eq. 25) of b supported on the
    consecutive ranks G, restricted to G."""
    pat = [(i, i) for i in range(6)] + [(0, 2), (0, 4), (1, 3), (2, 5), (3, 4), (1, 5)]
    rng, H, _ = _sym_case(7, [2, 3, 1, 4, 2, 3], pat)
    S = sc.compute_scaling(H, "A")
    g0, g1 = 1, 5
    T = sc.supernode_inverse(S, H.leaf_off, g0, g1)
    s0, s1 = int(H.leaf_off[g0]), int(H.leaf_off[g1])
    b = np.zeros((H.N, 2), np.complex128)
    b[s0:s1] = rng.standard_normal((s1 - s0, 2)) + 1j * rng.standard_normal((s1 - s0, 2))
    y = sc.apply_Rt(S, H.leaf_off, b)
    return bool(np.allclose(T @ b[s0:s1], y[s0:s1], atol=1e-12))


_LU = {}


def pin_series(se):
    """Many terms reach the LU solution of the assembled H-matrix (rho < 1);
    one refinement step lowers the two-term error and residual."""
    H, S, B = plate_converging()
    if "X" not in _LU:
        x_lu = np.linalg.solve(H.to_dense(), B[H.perm])
        X = np.empty_like(x_lu)
        X[H.perm] = x_lu
        _LU["X"] = X
    X = _LU["X"]
    with np.errstate(all="ignore"):
        x40, _ = se.series_solve(H, S, B, 40)
        x2, _ = se.series_solve(H, S, B, 2)
        xr = se.refine_once(H, S, B, x2)
    from oracle.series import rel_err, relative_residual
    return bool(np.all(rel_err(x40, X) < 1e-10) and
                np.all(rel_err(xr, X) < rel_err(x2, X)) and
                np.all(relative_residual(H, B, xr) < relative_residual(H, B, x2)))


def pin_rwg(rw):
    """Interior-edge count 3F/2 on a closed mesh; the flux of every basis
    function through its edge is l from T+ and -l into T- (normal continuity)."""
    from hm_workloads import icosphere
    v, f = icosphere(2, 0.5)
    r = rw.build_rwg(v, f)
    if r.n != 3 * len(f) // 2:
        return False
    for n in range(0, r.n, 7):
        a, b = r.edge[n]
        for tri, free, sgn in ((r.tri_p[n], r.free_p[n], 1.0), (r.tri_m[n], r.free_m[n], -1.0)):
            vf = v[f[tri, free]]
            mid = 0.5 * (v[a] + v[b])
            fval = sgn * r.length[n] / (2 * r.area[tri]) * (mid - vf)
            e = v[b] - v[a]
            nrm = np.cross(v[f[tri, 1]] - v[f[tri, 0]], v[f[tri, 2]] - v[f[tri, 0]])
            u = np.cross(e, nrm)
            u /= np.linalg.norm(u)
            if np.dot(u, mid - vf) < 0:
                u = -u
            flux = np.dot(fval, u) * np.linalg.norm(e)
            if not (abs(abs(flux) - np.linalg.norm(e)) < 1e-12 and np.sign(flux) == sgn):
                return False
    return True


def pin_hmatrix(hm):
    """The assembled H-matrix is symmetric and within 3 eps of the EFIE
    entries (0.5 lambda sphere); its products agree with the assembled matrix
    through the many-terms series (LU limit) and the refinement residual."""
    from tests.oracle_cases import case
    from oracle.series import series_solve, refine_once, rel_err, relative_residual
    rebuild = lambda H0: hm.HMatrix(N=H0.N, perm=H0.perm, leaf_off=H0.leaf_off,
                                    near=H0.near, far=H0.far, k=H0.k, meta=H0.meta)
    _, Zd, _ = dense_sphere_c1()[1:]
    H1 = rebuild(case("sphere_r0.5_L3")[1])
    Zh = H1.to_dense()
    Zp = Zd[np.ix_(H1.perm, H1.perm)]
    if not (np.array_equal(Zh, Zh.T) and
            np.linalg.norm(Zh - Zp) / np.linalg.norm(Zp) < 3e-4):
        return False
    H0, S, B = plate_converging()
    H = rebuild(H0)
    x_lu = np.linalg.solve(H.to_dense(), B[H.perm])
    X = np.empty_like(x_lu)
    X[H.perm] = x_lu
    with np.errstate(all="ignore"):
        x40, _ = series_solve(H, S, B, 40)
        x2, _ = series_solve(H, S, B, 2)
        xr = refine_once(H, S, B, x2)
    return bool(np.all(rel_err(x40, X) < 1e-10) and
                np.all(rel_err(xr, X) < rel_err(x2, X)) and
                np.all(relative_residual(H, B, xr) < relative_residual(H, B, x2)))


# -------------------------------------------------------------- the mutants
MUTANTS = [
    # (id, module, pin, original text, planted mistake)
    ("quadrature_weight_sign", "quadrature", pin_quadrature,
     "w1 = (155.0 - s15) / 1200.0", "w1 = (155.0 + s15) / 1200.0"),
    ("quadrature_point", "quadrature", pin_quadrature,
     "a1 = (6.0 - s15) / 21.0", "a1 = (6.0 - s15) / 12.0"),
    ("potential_dropped_solid_angle", "potentials", pin_potentials,
     "I_s += t * f - ah * beta", "I_s += t * f"),
    ("potential_vector_sign", "potentials", pin_potentials,
     "(R0sq * f + lp * Rp - lm * Rm)", "(R0sq * f + lp * Rp + lm * Rm)"),
    ("efie_scalar_potential_sign", "efie", pin_efie,
     "((k / 4.0) * A - s0 / k)", "((k / 4.0) * A + s0 / k)"),
    ("efie_vector_potential_dropped", "efie", pin_efie,
     "((k / 4.0) * A - s0 / k)", "(- s0 / k)"),
    ("plane_wave_direction", "efie", pin_plane_wave,
     "khat = -np.stack([st * cp, st * sp, ct], axis=1)",
     "khat = np.stack([st * cp, st * sp, ct], axis=1)"),
    ("phi_polarisation_uses_theta_hat", "efie", pin_phi_polarisation,
     "phat = np.where((pol == 0)[:, None], th_hat, ph_hat)",
     "phat = np.where((pol == 0)[:, None], th_hat, th_hat)"),
    ("rcs_constant", "rcs", pin_rcs,
     "(k * k * ETA0 * ETA0 / (4 * math.pi))", "(k * k * ETA0 * ETA0 / (2 * math.pi))"),
    ("mie_hankel_kind", "rcs", pin_mie,
     "xi = x * (jn + 1j * yn)", "xi = x * (jn - 1j * yn)"),
    ("octree_touching_off_by_one", "octree", pin_octree,
     "if lo_a > hi_b or lo_b > hi_a:", "if lo_a >= hi_b or lo_b >= hi_a:"),
    ("rwg_edge_opposite_wrong_vertex", "rwg", pin_rwg,
     "a, b = int(tv[(k + 1) % 3]), int(tv[(k + 2) % 3])",
     "a, b = int(tv[k]), int(tv[(k + 1) % 3])"),
    ("rwg_area_without_half", "rwg", pin_rwg,
     "area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)",
     "area = np.linalg.norm(np.cross(b - a, c - a), axis=1)"),
    ("far_product_conjugated_lower_block", "hmatrix", pin_hmatrix,
     "y[cs] += Q @ (P.T @ x[rs])", "y[cs] += Q.conj() @ (P.conj().T @ x[rs])"),
    ("near_product_conjugated_lower_block", "hmatrix", pin_hmatrix,
     "y[sj] += Bk.T @ x[si]", "y[sj] += Bk.conj().T @ x[si]"),
    ("assembled_lower_far_block_hermitian", "hmatrix", pin_hmatrix,
     "Z[c0:c0 + n, r0:r0 + m] = Bk.T", "Z[c0:c0 + n, r0:r0 + m] = Bk.conj().T"),
    ("aca_residual_sign", "aca", pin_aca,
     "row -= u[i] * v", "row += u[i] * v"),
    ("recompress_conjugate", "aca", pin_aca,
     "V2 = Qv @ Yh[:keep, :].T", "V2 = Qv @ Yh[:keep, :].conj().T"),
    ("alpha_sign", "scaling", pin_scaling,
     "apanel = -Dk_inv @ panel", "apanel = Dk_inv @ panel"),
    ("schur_update_sign", "scaling", pin_scaling,
     "tgt += upd[cuts[a]:cuts[a + 1], cuts[b]:cuts[b + 1]]",
     "tgt -= upd[cuts[a]:cuts[a + 1], cuts[b]:cuts[b + 1]]"),
    ("forward_sweep_stale_operand", "scaling", pin_sweeps,
     "out[sl[j]] += S.alpha[(k, j)].T @ out[sl[k]]",
     "out[sl[j]] += S.alpha[(k, j)].T @ b[sl[k]]"),
    ("back_sweep_sign", "scaling", pin_sweeps,
     "out[sl[k]] += S.alpha[(k, j)] @ out[sl[j]]",
     "out[sl[k]] -= S.alpha[(k, j)] @ out[sl[j]]"),
    ("supernode_not_transposed", "scaling", pin_supernodes,
     "return np.linalg.inv(np.eye(nG) - A.T)", "return np.linalg.inv(np.eye(nG) - A)"),
    ("supernode_sign", "scaling", pin_supernodes,
     "return np.linalg.inv(np.eye(nG) - A.T)", "return np.linalg.inv(np.eye(nG) + A.T)"),
    ("series_alternating_sign", "series", pin_series,
     "xt = xt + ((-1) ** n) * nxt", "xt = xt + nxt"),
    ("series_dropped_dinv", "series", pin_series,
     "nxt = apply_Dinv(S, off, apply_Rt(S, off, z))", "nxt = apply_Rt(S, off, z)"),
    ("series_dropped_right_scaling", "series", pin_series,
     "z = H.far_apply(apply_R(S, off, it))", "z = H.far_apply(it)"),
    ("refinement_residual_sign", "series", pin_series,
     "r = B[H.perm] - H.apply(xp)", "r = B[H.perm] + H.apply(xp)"),
]


@pytest.mark.parametrize("pin,modname", sorted({(m[2], m[1]) for m in MUTANTS},
                                               key=lambda t: t[0].__name__),
                         ids=lambda v: getattr(v, "__name__", v))
def test_pins_accept_the_oracle(pin, modname):
    if pin is pin_efie:
        assert pin(None)                 # the filled Z of the committed EFIE
    else:
        assert pin(load(modname))


@pytest.mark.parametrize("case", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(case):
    _, modname, pin, old, new = case
    assert not pin(load(modname, old, new))


# ------------------------------------------- the plain-C entry (oracle/cefie.c)
def pin_cefie(cm):
    """The C entry equals the NumPy EFIE entry (relative 1e-12) on self,
    touching and separated pairs of a small sphere."""
    from hm_workloads import icosphere
    from oracle.efie import EFIE
    from oracle.rwg import build_rwg
    v, f = icosphere(2, 0.5)
    r = build_rwg(v, f)
    E = EFIE(r)
    rows, cols = np.arange(0, r.n, 7), np.arange(r.n)
    a = E.block(rows, cols)
    return bool(np.abs(a - cm.CBlock(E)(rows, cols)).max() < 1e-12 * np.abs(a).max())


C_MUTANTS = [
    ("green_phase_sign", "gi = -s * inv4pi / R;", "gi = s * inv4pi / R;"),
    ("singular_part_not_subtracted", "gr = (touch ? c - 1.0 : c) * inv4pi / R;",
     "gr = c * inv4pi / R;"),
    ("solid_angle_dropped", "*Is += t * f - ah * beta;", "*Is += t * f;"),
    ("scalar_potential_sign", "((M->k / 4.0) * A - S[0][c] / M->k)",
     "((M->k / 4.0) * A + S[0][c] / M->k)"),
]


def load_c(tmp_path, old=None, new=None):
    """oracle.cefie bound to a copy of cefie.c (with `old` replaced by `new`)
    compiled into tmp_path."""
    import subprocess
    with open(os.path.join(ORACLE_DIR, "cefie.c")) as f:
        src = f.read()
    if old is not None:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    c = tmp_path / "cefie.c"
    so = tmp_path / "cefie.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-ffp-contract=off",
                           "-o", str(so), str(c), "-lm"])
    mod = load("cefie")
    mod._SRC, mod._LIB = str(c), None
    mod.lib_path = lambda: str(so)
    return mod


def test_c_pin_accepts_the_oracle(tmp_path):
    assert pin_cefie(load_c(tmp_path))


@pytest.mark.parametrize("case", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_c_pin_rejects_planted_mistake(case, tmp_path):
    _, old, new = case
    assert not pin_cefie(load_c(tmp_path, old, new))
