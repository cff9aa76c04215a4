"""H-matrix store Z = Z_N + Z_F (Eq. 13) built from the EFIE entries, the
octree block tree and ACA, and its products.

Storage (all in leaf / permuted order, see oracle.octree):
  near[(i, j)]  i <= j leaves: dense m_i x m_j block Z[leaf i, leaf j]; the
                (j, i) block is its transpose (Z_N = Z_N^T exactly); a diagonal
                block is symmetrised (B + B^T)/2;
  far[b]        upper far block (row cluster s before column cluster t):
                ("lr", r0, m, c0, n, U, V) with Z[s, t] ~ U V^T, or
                ("dense", r0, m, c0, n, B, None); the (t, s) block is the
                transpose, so Z_F = Z_F^T exactly.

Pinned by: the H-matrix product against the dense matrix on small meshes
(relative error of order the ACA tolerance), exact symmetry, and tiling of the
index square (oracle.octree).
"""
import os
from dataclasses import dataclass, field

import numpy as np

from .aca import aca, recompress
from .efie import EFIE
from .octree import Octree
from .rwg import build_rwg


@dataclass
class HMatrix:
    N: int
    perm: np.ndarray            # leaf position -> original RWG index
    leaf_off: np.ndarray        # (n_leaves + 1,)
    near: dict                  # (i, j) -> block
    far: list                   # see module docstring
    k: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n_leaves(self):
        return len(self.leaf_off) - 1

    def leaf_slice(self, i):
        return slice(int(self.leaf_off[i]), int(self.leaf_off[i + 1]))

    # --------------------------------------------------------------- products
    def near_apply(self, x):
        """Z_N x for x in leaf order, (N,) or (N, nrhs)."""
        y = np.zeros_like(x, dtype=np.complex128)
        for (i, j), Bk in self.near.items():
            si, sj = self.leaf_slice(i), self.leaf_slice(j)
            y[si] += Bk @ x[sj]
            if i != j:
                y[sj] += Bk.T @ x[si]
        return y

    def far_apply(self, x):
        """Z_F x for x in leaf order."""
        y = np.zeros_like(x, dtype=np.complex128)
        for kind, r0, m, c0, n, P, Q in self.far:
            rs, cs = slice(r0, r0 + m), slice(c0, c0 + n)
            if kind == "lr":
                y[rs] += P @ (Q.T @ x[cs])
                y[cs] += Q @ (P.T @ x[rs])
            else:
                y[rs] += P @ x[cs]
                y[cs] += P.T @ x[rs]
        return y

    def apply(self, x):
        return self.near_apply(x) + self.far_apply(x)

    def to_dense(self):
        """Assembled N x N matrix in leaf order (small N only)."""
        Z = np.zeros((self.N, self.N), np.complex128)
        for (i, j), Bk in self.near.items():
            si, sj = self.leaf_slice(i), self.leaf_slice(j)
            Z[si, sj] = Bk
            Z[sj, si] = Bk.T
        for kind, r0, m, c0, n, P, Q in self.far:
            Bk = P @ Q.T if kind == "lr" else P
            Z[r0:r0 + m, c0:c0 + n] = Bk
            Z[c0:c0 + n, r0:r0 + m] = Bk.T
        return Z

    def stats(self):
        near_e = sum(b.size for b in self.near.values())
        lr = [f for f in self.far if f[0] == "lr"]
        far_e = sum(f[5].size + f[6].size for f in lr) + \
            sum(f[5].size for f in self.far if f[0] != "lr")
        return {"N": self.N, "leaves": self.n_leaves, "near_blocks": len(self.near),
                "near_entries_upper": near_e, "far_blocks": len(self.far),
                "far_lowrank": len(lr), "far_entries": far_e,
                "max_rank": max([f[5].shape[1] for f in lr], default=0)}


# ------------------------------------------------------------------- build
_W = {}


def _worker_init(verts, tris, wavelength, use_c=False):
    rwg = build_rwg(verts, tris)
    E = EFIE(rwg, wavelength)
    _W["efie"] = E
    if use_c:
        from .cefie import CBlock
        _W["block"] = CBlock(E)          # same entries, plain C (oracle/cefie.c)
    else:
        _W["block"] = E.block


def _near_task(args):
    rows, cols, diag = args
    Bk = _W["block"](rows, cols)
    if diag:
        Bk = 0.5 * (Bk + Bk.T)
    return Bk


def _far_task(args):
    rows, cols, eps = args
    blk = _W["block"]
    U, V = aca(lambda i: blk(rows[i:i + 1], cols)[0],
               lambda j: blk(rows, cols[j:j + 1])[:, 0],
               len(rows), len(cols), eps)
    U, V = recompress(U, V, eps)
    m, n = len(rows), len(cols)
    if U.shape[1] * (m + n) >= m * n:
        return ("dense", blk(rows, cols), None)
    return ("lr", U, V)


def build_hmatrix(verts, tris, wavelength=1.0, leaf_max=64, aca_tol=1e-4,
                  processes=None, use_c=False, eta=0.0):
    """Fill the H-matrix of a mesh.  ``eta`` > 0 adds the paper's form of the
    admissibility (Eq. 10, see oracle.octree) to the non-touching test.
    ``processes`` > 1 runs the block fills in
    a spawn-started process pool (same arithmetic, block by block);
    ``use_c`` evaluates the entries with the plain-C statement of the same
    formulas (oracle/cefie.c) instead of NumPy."""
    rwg = build_rwg(verts, tris)
    tree = Octree(rwg.centre, leaf_max) if not eta else Octree(rwg.centre, leaf_max, eta)
    near_u, far_u = tree.upper_blocks()
    P = tree.perm
    off = tree.leaf_off
    near_jobs = []
    for (i, j) in near_u:
        near_jobs.append((P[off[i]:off[i + 1]], P[off[j]:off[j + 1]], i == j))
    far_jobs, far_geom = [], []
    for (s, t) in far_u:
        ns, nt = tree.nodes[s], tree.nodes[t]
        far_jobs.append((P[ns.start:ns.start + ns.count],
                         P[nt.start:nt.start + nt.count], aca_tol))
        far_geom.append((ns.start, ns.count, nt.start, nt.count))
    if processes is None:
        processes = 1
    if processes > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        if use_c:
            from .cefie import build as _build_c
            _build_c()
        # one BLAS thread per worker process (the pool already fills the cores)
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            with ctx.Pool(processes, initializer=_worker_init,
                          initargs=(np.asarray(verts), np.asarray(tris), wavelength,
                                    use_c)) as pool:
                near_res = pool.map(_near_task, near_jobs, chunksize=16)
                far_res = pool.map(_far_task, far_jobs, chunksize=16)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    else:
        _worker_init(verts, tris, wavelength, use_c)
        near_res = [_near_task(a) for a in near_jobs]
        far_res = [_far_task(a) for a in far_jobs]
    near = {key: Bk for key, Bk in zip(near_u, near_res)}
    far = [(kind, r0, m, c0, n, A, B) for (kind, A, B), (r0, m, c0, n)
           in zip(far_res, far_geom)]
    H = HMatrix(N=rwg.n, perm=P, leaf_off=off, near=near, far=far,
                k=2 * np.pi / wavelength,
                meta={"leaf_max": leaf_max, "aca_tol": aca_tol,
                      "wavelength": wavelength})
    H.tree = tree
    H.rwg = rwg
    return H


def default_processes():
    return max(1, min(16, os.cpu_count() or 1))
