"""Non-symmetric H-matrix, near-field scaling and power series for the CFIE
(Sec. II, Eq. 8; Sec. III-A/B, Eq. 14-36 without Z = Z^T).  Test and study
infrastructure.

The CFIE matrix is not symmetric, so the left scaling coefficients are no
longer the transposes of the right ones (that remark after Eq. 29 rests on
Z = Z^T).  With the leaves in elimination order, for k = 1..n:
  D_k       = Z~_kk
  alpha_kj  = -D_k^{-1} Z~_kj   for j in row k      (right coefficients, Eq. 16)
  alphaL_kj = -Z~_jk D_k^{-1}   for j in row k      (left coefficients, Eq. 18)
  Z~_ij    += Z~_ik alpha_kj = Z~_ij - Z~_ik D_k^{-1} Z~_kj, all i, j in row k (Eq. 21)
Each step is a column operation (right factor R_k = I + sum_j e_k alpha_kj e_j^T)
and the matching row operation (left factor L_k = I + sum_j e_j alphaL_kj e_k^T),
so with L = L_n ... L_1 and R = R_1 ... R_n
  L Z_N R = diag(D_1..D_n)                          (Eq. 22-23, reading A),
b~ = L b is the forward substitution b~_j = b_j + sum_{k<j} alphaL_kj b~_k and
x = R x~ the back substitution of the symmetric case.  For Z = Z^T the left
coefficients are alpha_kj^T and everything reduces to oracle.scaling.  The
series is that of oracle.series with R^T replaced by L:
  it_0 = D^{-1} L b,  it_n = D^{-1} L Z_F R it_{n-1},  x = R sum_n (-1)^n it_n.

Storage (HMatrixGen, leaf order): near[(i, j)] for every ordered near pair of
leaves, far blocks for every ordered far pair of clusters (s, t):
("lr", r0, m, c0, n, U, V) with Z[s, t] ~ U V^T, or ("dense", r0, m, c0, n, B,
None).  Same octree, admissibility and ACA as oracle.hmatrix.

Pinned by: a symmetric H-matrix through these functions gives the symmetric
scaling and series (alphaL = alpha^T, same D, same x); L Z_N R block diagonal
with diagonal D on the CFIE (reading A); Z_F = 0 -> x = Z_N^{-1} b; one leaf
-> x = Z^{-1} b; many terms -> the LU solution when the ratio of Eq. 45 is
below one.
"""
from dataclasses import dataclass, field

import numpy as np

from .aca import aca, recompress
from .octree import Octree
from .rwg import build_rwg
from .scaling import Scaling, apply_R, apply_Dinv, near_pattern, symbolic_fill


@dataclass
class HMatrixGen:
    N: int
    perm: np.ndarray
    leaf_off: np.ndarray
    near: dict                  # (i, j) -> block, every ordered near pair
    far: list                   # every ordered far pair
    k: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n_leaves(self):
        return len(self.leaf_off) - 1

    def leaf_slice(self, i):
        return slice(int(self.leaf_off[i]), int(self.leaf_off[i + 1]))

    def near_apply(self, x):
        y = np.zeros_like(x, dtype=np.complex128)
        for (i, j), Bk in self.near.items():
            y[self.leaf_slice(i)] += Bk @ x[self.leaf_slice(j)]
        return y

    def far_apply(self, x):
        y = np.zeros_like(x, dtype=np.complex128)
        for kind, r0, m, c0, n, P, Q in self.far:
            if kind == "lr":
                y[r0:r0 + m] += P @ (Q.T @ x[c0:c0 + n])
            else:
                y[r0:r0 + m] += P @ x[c0:c0 + n]
        return y

    def apply(self, x):
        return self.near_apply(x) + self.far_apply(x)

    def to_dense(self, far=True):
        Z = np.zeros((self.N, self.N), np.complex128)
        for (i, j), Bk in self.near.items():
            Z[self.leaf_slice(i), self.leaf_slice(j)] = Bk
        if far:
            for kind, r0, m, c0, n, P, Q in self.far:
                Z[r0:r0 + m, c0:c0 + n] = P @ Q.T if kind == "lr" else P
        return Z


def from_symmetric(H):
    """The symmetric H-matrix of oracle.hmatrix with its implied lower half
    stored explicitly (for checks against the symmetric scaling)."""
    near = {}
    for (i, j), Bk in H.near.items():
        near[(i, j)] = Bk
        if i != j:
            near[(j, i)] = Bk.T
    far = []
    for kind, r0, m, c0, n, P, Q in H.far:
        far.append((kind, r0, m, c0, n, P, Q))
        if kind == "lr":
            far.append((kind, c0, n, r0, m, Q, P))
        else:
            far.append((kind, c0, n, r0, m, P.T, None))
    G = HMatrixGen(N=H.N, perm=H.perm, leaf_off=H.leaf_off, near=near, far=far, k=H.k,
                   meta=dict(H.meta))
    G.tree = H.tree
    return G


def _svd_compress(Bk, eps):
    """U, V with U V^T the truncated SVD of Bk: singular values below eps
    times the largest dropped (the best approximation of the rank ACA aims
    at; Eq. 11-12)."""
    u, sv, vh = np.linalg.svd(Bk, full_matrices=False)
    r = int(np.sum(sv > eps * sv[0])) if sv.size and sv[0] > 0 else 0
    return u[:, :r] * sv[:r], vh[:r].T


def build_hmatrix_general(verts, tris, op_factory, leaf_max=64, aca_tol=1e-4, eta=0.0,
                          compress="aca"):
    """H-matrix of a non-symmetric operator: op_factory(rwg) returns an object
    with block(rows, cols) (e.g. lambda r: CFIE(r, wavelength, 0.5)).  Every
    ordered near pair filled densely, every ordered far pair by ACA with
    recompression (``compress="aca"``), or filled densely and cut to its
    truncated SVD (``compress="svd"``, the faster choice for studies); dense
    when the factors would be larger."""
    rwg = build_rwg(verts, tris)
    op = op_factory(rwg)
    tree = Octree(rwg.centre, leaf_max) if not eta else Octree(rwg.centre, leaf_max, eta)
    near_pairs, far_pairs = tree.blocks()
    P, off = tree.perm, tree.leaf_off
    near = {}
    for (i, j) in sorted(set(near_pairs)):
        near[(i, j)] = op.block(P[off[i]:off[i + 1]], P[off[j]:off[j + 1]])
    far = []
    for (s, t) in sorted(set(far_pairs), key=lambda st: (tree.nodes[st[0]].start,
                                                         tree.nodes[st[1]].start)):
        ns, nt = tree.nodes[s], tree.nodes[t]
        rows = P[ns.start:ns.start + ns.count]
        cols = P[nt.start:nt.start + nt.count]
        m, n = len(rows), len(cols)
        Bk = None
        if compress == "svd":
            Bk = op.block(rows, cols)
            U, V = _svd_compress(Bk, aca_tol)
        else:
            U, V = aca(lambda a: op.block(rows[a:a + 1], cols)[0],
                       lambda b: op.block(rows, cols[b:b + 1])[:, 0],
                       m, n, aca_tol)
            U, V = recompress(U, V, aca_tol)
        if U.shape[1] * (m + n) >= m * n:
            far.append(("dense", ns.start, m, nt.start, n,
                        Bk if Bk is not None else op.block(rows, cols), None))
        else:
            far.append(("lr", ns.start, m, nt.start, n, U, V))
    H = HMatrixGen(N=rwg.n, perm=P, leaf_off=off, near=near, far=far, k=getattr(op, "k", 0.0),
                   meta={"leaf_max": leaf_max, "aca_tol": aca_tol, "eta": eta})
    H.tree = tree
    H.rwg = rwg
    return H


_WG = {}


def _dense_init(verts, tris, wavelength, alpha):
    from .mfie import CFIE
    _WG["op"] = CFIE(build_rwg(verts, tris), wavelength, alpha)


def _dense_rows(rows):
    op = _WG["op"]
    return op.block(rows, np.arange(op.rwg.n))


def dense_cfie(verts, tris, wavelength=1.0, alpha=0.5, processes=1, chunk=64):
    """The full CFIE matrix (original RWG order), row chunks filled by a
    spawn-started process pool (same arithmetic as CFIE.block).  Studies."""
    rwg = build_rwg(verts, tris)
    N = rwg.n
    chunks = [np.arange(s, min(N, s + chunk)) for s in range(0, N, chunk)]
    Z = np.empty((N, N), np.complex128)
    if processes > 1:
        import multiprocessing as mp
        import os
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            with mp.get_context("spawn").Pool(processes, initializer=_dense_init,
                                              initargs=(np.asarray(verts), np.asarray(tris),
                                                        wavelength, alpha)) as pool:
                for rows, blk in zip(chunks, pool.imap(_dense_rows, chunks)):
                    Z[rows] = blk
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    else:
        _dense_init(verts, tris, wavelength, alpha)
        for rows in chunks:
            Z[rows] = _dense_rows(rows)
    return rwg, Z


def hmatrix_from_dense(Zd, rwg, leaf_max, aca_tol=1e-4, eta=0.0, tree=None):
    """HMatrixGen of a dense matrix (original order) on the octree of the
    mesh (or a given tree with the same interface, e.g. the binary tree of
    oracle.study_leaf_size): near blocks sliced, far blocks cut to their
    truncated SVD.  Studies (one fill serves every leaf cap)."""
    if tree is None:
        tree = Octree(rwg.centre, leaf_max) if not eta else Octree(rwg.centre, leaf_max, eta)
    near_pairs, far_pairs = tree.blocks()
    P, off = tree.perm, tree.leaf_off
    near = {(i, j): Zd[np.ix_(P[off[i]:off[i + 1]], P[off[j]:off[j + 1]])]
            for (i, j) in sorted(set(near_pairs))}
    far = []
    for (s, t) in sorted(set(far_pairs), key=lambda st: (tree.nodes[st[0]].start,
                                                         tree.nodes[st[1]].start)):
        ns, nt = tree.nodes[s], tree.nodes[t]
        Bk = Zd[np.ix_(P[ns.start:ns.start + ns.count], P[nt.start:nt.start + nt.count])]
        U, V = _svd_compress(Bk, aca_tol)
        m, n = Bk.shape
        if U.shape[1] * (m + n) >= m * n:
            far.append(("dense", ns.start, m, nt.start, n, Bk, None))
        else:
            far.append(("lr", ns.start, m, nt.start, n, U, V))
    H = HMatrixGen(N=rwg.n, perm=P, leaf_off=off, near=near, far=far,
                   meta={"leaf_max": leaf_max, "aca_tol": aca_tol, "eta": eta})
    H.tree = tree
    H.rwg = rwg
    return H


@dataclass
class ScalingGen(Scaling):
    alphaL: dict = field(default_factory=dict)   # (k, j) -> m_j x m_k


def compute_scaling_general(H, reading="A", order=None):
    """Left and right scaling coefficients of a non-symmetric near field (see
    the module docstring); same patterns and readings as oracle.scaling."""
    n = H.n_leaves
    if order is None:
        order = list(range(n))
    order = [int(x) for x in order]
    assert sorted(order) == list(range(n))
    pos = {leaf: q for q, leaf in enumerate(order)}
    pairs = [(pos[i], pos[j]) for (i, j) in H.near.keys()]
    if reading == "A":
        rows = symbolic_fill(n, pairs)
    elif reading == "B":
        rows = [sorted(r) for r in near_pattern(n, pairs)]
    else:
        raise ValueError(reading)
    m = np.diff(H.leaf_off)[order]

    def blk(a, b):
        B = H.near.get((order[a], order[b]))
        return B.copy() if B is not None else np.zeros((m[a], m[b]), np.complex128)

    Zt = {}
    for k in range(n):
        Zt[(k, k)] = blk(k, k)
        for j in rows[k]:
            Zt[(k, j)] = blk(k, j)
            Zt[(j, k)] = blk(j, k)
    alpha, alphaL, D, Dinv = {}, {}, [], []
    for k in range(n):
        Dk = Zt.pop((k, k))
        Dk_inv = np.linalg.inv(Dk)
        D.append(Dk)
        Dinv.append(Dk_inv)
        row = rows[k]
        if not row:
            continue
        cuts = np.concatenate([[0], np.cumsum([m[j] for j in row])])
        right = np.concatenate([Zt.pop((k, j)) for j in row], axis=1)     # Z~_kj
        left = np.concatenate([Zt.pop((j, k)) for j in row], axis=0)      # Z~_jk
        aR = -Dk_inv @ right
        aL = -left @ Dk_inv
        upd = left @ aR                                                   # Z~_ik alpha_kj
        for a, j in enumerate(row):
            alpha[(k, j)] = aR[:, cuts[a]:cuts[a + 1]]
            alphaL[(k, j)] = aL[cuts[a]:cuts[a + 1], :]
        for a, i in enumerate(row):
            for b, j in enumerate(row):
                tgt = Zt.get((i, j))
                if tgt is None:
                    continue                                              # reading B
                tgt += upd[cuts[a]:cuts[a + 1], cuts[b]:cuts[b + 1]]
    return ScalingGen(n=n, rows=rows, alpha=alpha, D=D, Dinv=Dinv, reading=reading,
                      order=order, alphaL=alphaL)


def apply_L(S, leaf_off, b):
    """b~ = L b by forward block substitution (module docstring), leaf order."""
    out = np.array(b, dtype=np.complex128, copy=True)
    sl = S.slices(leaf_off)
    for k in range(S.n):
        for j in S.rows[k]:
            out[sl[j]] += S.alphaL[(k, j)] @ out[sl[k]]
    return out


def dense_L(S, leaf_off):
    """L = L_n ... L_1 as a dense matrix (small N only; tests)."""
    N = int(leaf_off[-1])
    sl = S.slices(leaf_off)
    L = np.eye(N, dtype=np.complex128)
    for k in range(S.n):
        Lk = np.eye(N, dtype=np.complex128)
        for j in S.rows[k]:
            Lk[sl[j], sl[k]] = S.alphaL[(k, j)]
        L = Lk @ L
    return L


def _norms(v):
    return np.sqrt(np.sum(np.abs(v) ** 2, axis=0))


def series_solve_general(H, S, B, n_terms=2):
    """X (original RWG order) and the Eq. 45 ratios for B in original order."""
    B = np.asarray(B, dtype=np.complex128)
    off = H.leaf_off
    it = apply_Dinv(S, off, apply_L(S, off, B[H.perm]))
    xt = it.copy()
    ratios = []
    for t in range(1, n_terms):
        nxt = apply_Dinv(S, off, apply_L(S, off, H.far_apply(apply_R(S, off, it))))
        with np.errstate(divide="ignore", invalid="ignore"):
            ratios.append(_norms(nxt) / _norms(it))
        xt = xt + ((-1) ** t) * nxt
        it = nxt
    xp = apply_R(S, off, xt)
    X = np.empty_like(xp)
    X[H.perm] = xp
    return X, np.array(ratios)
