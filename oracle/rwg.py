"""RWG basis functions on a triangle mesh (Sec. II: current and charge are
expanded in RWG functions, Galerkin tested).

Conventions (a reading; the paper does not fix them):
  * one unknown per interior edge (an edge shared by exactly two triangles);
  * unknowns numbered by the sorted edge key (min vertex, max vertex);
  * T+ is the lower-index triangle of the pair, T- the higher;
  * on T+-, f = +-(l / 2A+-) (r - v+-) with v+- the vertex opposite the edge,
    so the divergence is +-l / A+-.

Pinned by: interior-edge counts (3F/2 on closed meshes, 19040 on the 80x80
plate), zero total charge per basis function, and continuity of the normal
component across the edge (flux l out of T+ equals flux into T-).
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class RWG:
    verts: np.ndarray        # (nv, 3)
    tris: np.ndarray         # (nt, 3)
    edge: np.ndarray         # (N, 2) vertex indices, sorted
    tri_p: np.ndarray        # (N,) T+ index
    tri_m: np.ndarray        # (N,) T- index
    free_p: np.ndarray       # (N,) local index 0..2 of the free vertex in T+
    free_m: np.ndarray       # (N,) local index 0..2 of the free vertex in T-
    length: np.ndarray       # (N,)
    area: np.ndarray         # (nt,)
    centre: np.ndarray       # (N, 3) edge midpoints (octree points)

    @property
    def n(self):
        return len(self.edge)


def build_rwg(verts, tris) -> RWG:
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    owners = {}
    for t, tv in enumerate(tris):
        for k in range(3):
            a, b = int(tv[(k + 1) % 3]), int(tv[(k + 2) % 3])   # edge opposite local k
            key = (a, b) if a < b else (b, a)
            owners.setdefault(key, []).append((t, k))
    keys = sorted(k for k, v in owners.items() if len(v) == 2)
    N = len(keys)
    edge = np.array(keys, dtype=np.int64).reshape(N, 2)
    tri_p = np.empty(N, np.int64)
    tri_m = np.empty(N, np.int64)
    free_p = np.empty(N, np.int64)
    free_m = np.empty(N, np.int64)
    for i, key in enumerate(keys):
        (t0, k0), (t1, k1) = sorted(owners[key])
        tri_p[i], free_p[i] = t0, k0
        tri_m[i], free_m[i] = t1, k1
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    length = np.linalg.norm(verts[edge[:, 0]] - verts[edge[:, 1]], axis=1)
    centre = 0.5 * (verts[edge[:, 0]] + verts[edge[:, 1]])
    return RWG(verts, tris, edge, tri_p, tri_m, free_p, free_m, length, area, centre)
