"""Schur-complement scaling of the symmetric near field (Sec. III-A,
Eq. 14-29).

For leaves k = 1..n in elimination order (the depth-first leaf order):
  D_k      = Z~_kk                                   (the scaled diagonal block)
  alpha_kj = -D_k^{-1} Z~_kj     for j > k in row k   (right coefficients, Eq. 16)
  Z~_ij   += alpha_ki^T Z~_kj    for i <= j in row k  (Schur complement, Eq. 21:
            = Z~_ij - Z~_ik D_k^{-1} Z~_kj, using Z~_ik = Z~_ki^T)
The left coefficients are alpha' = alpha^T (Eq. 18 and the symmetry remark
after Eq. 29) and are never stored.  After all n steps
  R^T Z_N R = diag(D_1..D_n)  (Eq. 22-23),  R = alpha_1 alpha_2 ... alpha_n,
R = (I - E)^{-1} with E_kj = alpha_kj (k < j), so x = R x~ is the block back
substitution x_k = x~_k + sum_{j>k} alpha_kj x_j and b~ = R^T b is the forward
substitution b~_j = b_j + sum_{k<j} alpha_kj^T b~_k (Eq. 25-26).

The elimination order is a permutation of the leaves (``order[q]`` is the
leaf eliminated q-th); rows, alpha, D are indexed by elimination rank.  The
default is the depth-first leaf order; nested dissection (nd_order) is the
fill-reducing alternative (the paper uses Sloan's ordering for the same
purpose, Sec. III-A).

Readings:
  * "A" (default): the scaling considers every fill-in block (the block row of
    k reaches all leaves that elimination connects to k), so Eq. 23 holds
    exactly.  The pattern is the symbolic block Cholesky structure, computed
    with the elimination tree (parent = first leaf in the row).
  * "B": fill restricted to the near-field pattern; updates that land outside
    it are dropped (the storage of the complexity analysis, Sec. IV).
  * D_k^{-1} is LU with partial pivoting followed by the explicit inverse
    (numpy.linalg.inv), FP64.

Pinned by: the 4-block example of Eq. 14-21 (alpha_1 and the first Schur step
block by block, blocks outside row/column 1 untouched), R^T Z_N R block
diagonal with diagonal D (reading A), and the elimination-tree pattern equal
to the naive all-pairs symbolic elimination.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Scaling:
    n: int
    rows: list           # rows[k] = sorted list of ranks j > k with alpha_kj stored
    alpha: dict          # (k, j) -> m_k x m_j   (ranks)
    D: list              # D_k   (rank k)
    Dinv: list           # D_k^{-1}
    reading: str
    order: list          # order[k] = leaf eliminated k-th

    def entries(self, leaf_off):
        m = np.diff(leaf_off)[self.order]
        a = sum(int(m[k] * m[j]) for (k, j) in self.alpha)
        d = int(np.sum(m * m))
        return a, d

    def slices(self, leaf_off):
        return [slice(int(leaf_off[l]), int(leaf_off[l + 1])) for l in self.order]


def near_pattern(n, near_pairs):
    rows = [set() for _ in range(n)]
    for (i, j) in near_pairs:
        if i < j:
            rows[i].add(j)
        elif j < i:
            rows[j].add(i)
    return rows


def symbolic_fill(n, near_pairs):
    """Block Cholesky structure: row(parent) |= row(k) - {parent}, parent =
    min row(k), visiting k in order."""
    rows = near_pattern(n, near_pairs)
    for k in range(n):
        if rows[k]:
            p = min(rows[k])
            rows[p] |= rows[k] - {p}
    return [sorted(r) for r in rows]


def symbolic_fill_naive(n, near_pairs):
    """All-pairs elimination: eliminating k connects every pair of its row."""
    rows = near_pattern(n, near_pairs)
    for k in range(n):
        lst = sorted(rows[k])
        for a, i in enumerate(lst):
            rows[i].update(lst[a + 1:])
    return [sorted(r) for r in rows]


def nd_order(tree, near_pairs, min_size=4, with_groups=False):
    """Geometric nested dissection of the leaf graph (near pairs = edges):
    split the leaves at the median (ties by leaf number) of the widest axis of
    their cell centres; the separator is the part of the first half adjacent
    to the second; order = ND(first - separator), ND(second), separator.

    ``with_groups``: also return the supernode boundaries in ranks, a list
    g_0 = 0 < g_1 < ... = n where every group [g_i, g_i+1) is one bottom set
    of at most ``min_size`` leaves or one separator (ranks of a group are
    consecutive)."""
    n = tree.n_leaves
    adj = [set() for _ in range(n)]
    for (i, j) in near_pairs:
        if i != j:
            adj[i].add(j)
            adj[j].add(i)
    cen = []
    for nid in tree.leaves:
        nd = tree.nodes[nid]
        cen.append([(nd.ijk[a] + 0.5) / (1 << nd.level) for a in range(3)])
    cen = np.array(cen)
    order, groups = [], []

    def rec(ids):
        if len(ids) <= min_size:
            if ids:
                groups.append(len(order))
            order.extend(sorted(ids))
            return
        ext = [cen[ids, a].max() - cen[ids, a].min() for a in range(3)]
        ax = int(np.argmax(ext))        # first axis among equal extents
        srt = sorted(ids, key=lambda i: (cen[i, ax], i))
        h = len(srt) // 2
        second = set(srt[h:])
        first = srt[:h]
        sep = sorted(i for i in first if adj[i] & second)
        sset = set(sep)
        rec(sorted(i for i in first if i not in sset))
        rec(sorted(second))
        if sep:
            groups.append(len(order))
        order.extend(sep)

    rec(list(range(n)))
    if with_groups:
        return order, groups + [n]
    return order


def compute_scaling(H, reading="A", order=None):
    """Scaling coefficients of the H-matrix's near field (see module doc).
    ``order``: leaves in elimination order (default: depth-first)."""
    n = H.n_leaves
    if order is None:
        order = list(range(n))
    order = [int(x) for x in order]
    assert sorted(order) == list(range(n))
    pos = {leaf: q for q, leaf in enumerate(order)}

    def near_blk(a, b):          # near block between ranks a <= b, or None
        la, lb = order[a], order[b]
        if la <= lb:
            blk = H.near.get((la, lb))
            return None if blk is None else blk
        blk = H.near.get((lb, la))
        return None if blk is None else blk.T

    near_pairs = [(pos[i], pos[j]) for (i, j) in H.near.keys()]
    if reading == "A":
        rows = symbolic_fill(n, near_pairs)
    elif reading == "B":
        rows = [sorted(r) for r in near_pattern(n, near_pairs)]
    else:
        raise ValueError(reading)
    m = np.diff(H.leaf_off)[order]
    Zt = {}
    for k in range(n):
        Zt[(k, k)] = near_blk(k, k).copy()
        for j in rows[k]:
            blk = near_blk(k, j)
            Zt[(k, j)] = blk.copy() if blk is not None else \
                np.zeros((m[k], m[j]), np.complex128)
    alpha, D, Dinv = {}, [], []
    for k in range(n):
        Dk = Zt.pop((k, k))
        Dk_inv = np.linalg.inv(Dk)
        D.append(Dk)
        Dinv.append(Dk_inv)
        row = rows[k]
        if not row:
            continue
        # the block row k as one panel [Z~_kj, j in row]: alpha row = -D_k^-1 panel
        # (Eq. 16); all Schur updates alpha_ki^T Z~_kj as one panel product (Eq. 21)
        cuts = np.concatenate([[0], np.cumsum([m[j] for j in row])])
        panel = np.concatenate([Zt[(k, j)] for j in row], axis=1)
        apanel = -Dk_inv @ panel
        upd = apanel.T @ panel
        for a, i in enumerate(row):
            alpha[(k, i)] = apanel[:, cuts[a]:cuts[a + 1]]
        for a, i in enumerate(row):
            for b in range(a, len(row)):
                tgt = Zt.get((i, row[b]))
                if tgt is None:
                    continue                      # reading B: outside the pattern
                tgt += upd[cuts[a]:cuts[a + 1], cuts[b]:cuts[b + 1]]
        for j in row:
            del Zt[(k, j)]
    return Scaling(n=n, rows=rows, alpha=alpha, D=D, Dinv=Dinv, reading=reading,
                   order=order)


def supernode_inverse(S, leaf_off, g0, g1):
    """T_G = (I - A_G^T)^{-1} of the consecutive ranks G = g0 .. g1-1, where
    A_G holds the blocks alpha_kj (k < j, both in G).  Restricted to the rows
    of G, the forward substitution of Eq. 25 reads b~_G = b_G + A_G^T b~_G +
    (terms from ranks before g0), so T_G maps the right-hand side of G, with
    its outside contributions added, to b~_G.  Row-major n_G x n_G, rows and
    columns in rank order (block of rank k at the sum of the sizes of ranks
    g0 .. k-1).  Dense inverse (numpy.linalg.inv); tests and the block file
    only."""
    m = np.diff(leaf_off)[S.order]
    off = np.concatenate([[0], np.cumsum(m[g0:g1])])
    nG = int(off[-1])
    A = np.zeros((nG, nG), np.complex128)
    for k in range(g0, g1):
        for j in S.rows[k]:
            if j < g1:
                a, b = k - g0, j - g0
                A[off[a]:off[a + 1], off[b]:off[b + 1]] = S.alpha[(k, j)]
    return np.linalg.inv(np.eye(nG) - A.T)


# ------------------------------------------------------------ applications
def apply_Rt(S, leaf_off, b):
    """b~ = R^T b (Eq. 25) by forward block substitution, leaf order."""
    out = np.array(b, dtype=np.complex128, copy=True)
    sl = S.slices(leaf_off)
    for k in range(S.n):
        for j in S.rows[k]:
            out[sl[j]] += S.alpha[(k, j)].T @ out[sl[k]]
    return out


def apply_R(S, leaf_off, x_t):
    """x = R x~ (Eq. 26) by back block substitution, leaf order."""
    out = np.array(x_t, dtype=np.complex128, copy=True)
    sl = S.slices(leaf_off)
    for k in range(S.n - 1, -1, -1):
        for j in S.rows[k]:
            out[sl[k]] += S.alpha[(k, j)] @ out[sl[j]]
    return out


def apply_Dinv(S, leaf_off, v):
    """Z~_N^{-1} v, block by block (Eq. 32)."""
    out = np.empty_like(v, dtype=np.complex128)
    for k, s in enumerate(S.slices(leaf_off)):
        out[s] = S.Dinv[k] @ v[s]
    return out


def dense_R(S, leaf_off):
    """R = alpha_1 alpha_2 ... alpha_n as a dense matrix, multiplying the
    dense alpha_k of Eq. 15-16 in order (small N only; tests)."""
    N = int(leaf_off[-1])
    sl = S.slices(leaf_off)
    R = np.eye(N, dtype=np.complex128)
    for k in range(S.n):
        Ak = np.eye(N, dtype=np.complex128)
        for j in S.rows[k]:
            Ak[sl[k], sl[j]] = S.alpha[(k, j)]
        R = R @ Ak
    return R
