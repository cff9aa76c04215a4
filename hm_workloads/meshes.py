"""Deterministic surface-mesh generators (float64 vertices, int64 triangles).

Every generator returns ``(verts, tris)``: ``verts`` is (nv, 3) float64 in metres,
``tris`` is (nt, 3) int64 with counter-clockwise vertex order seen from outside
(outward normals) for closed bodies and +z normals for the plate.  Output is a
pure function of the arguments, so two processes produce bit-identical meshes.
"""
from __future__ import annotations

import math

import numpy as np


def _icosahedron():
    """The 12 vertices / 20 faces of a regular icosahedron on the unit sphere.

    Faces are found as the vertex triples whose three pairwise distances all
    equal the edge length (2 before normalisation), then oriented outward and
    sorted, so the numbering is reproducible.
    """
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((0.0, s1, s2 * p))
            v.append((s1, s2 * p, 0.0))
            v.append((s2 * p, 0.0, s1))
    v = np.array(v, dtype=np.float64)
    n = len(v)
    faces = []
    for a in range(n):
        for b in range(a + 1, n):
            if abs(np.linalg.norm(v[a] - v[b]) - 2.0) > 1e-9:
                continue
            for c in range(b + 1, n):
                if (abs(np.linalg.norm(v[a] - v[c]) - 2.0) < 1e-9 and
                        abs(np.linalg.norm(v[b] - v[c]) - 2.0) < 1e-9):
                    nrm = np.cross(v[b] - v[a], v[c] - v[a])
                    if np.dot(nrm, v[a] + v[b] + v[c]) < 0:
                        faces.append((a, c, b))
                    else:
                        faces.append((a, b, c))
    assert len(faces) == 20
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, np.array(sorted(faces), dtype=np.int64)


def icosphere(level: int, radius: float = 1.0):
    """Icosahedron subdivided ``level`` times (each triangle into four), every
    new vertex projected onto the sphere of the given radius.

    20*4**level triangles, 30*4**level edges, 10*4**level + 2 vertices.
    """
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    faces = [tuple(x) for x in f]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                m = np.array(verts[a]) + np.array(verts[b])
                m /= np.linalg.norm(m)
                idx = len(verts)
                verts.append(tuple(m))
                cache[key] = idx
            return idx

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    verts = np.array(verts, dtype=np.float64) * float(radius)
    return verts, np.array(faces, dtype=np.int64)


def plate(side: float, ncell: int, z: float = 0.0):
    """Square plate [-side/2, side/2]^2 in the plane z, ncell x ncell square
    cells, each split along the diagonal from its (i, j) to its (i+1, j+1)
    corner.  2*ncell**2 triangles with +z normals.
    """
    h = side / ncell
    xs = -side / 2.0 + h * np.arange(ncell + 1, dtype=np.float64)
    X, Y = np.meshgrid(xs, xs, indexing="ij")          # vertex (i, j) -> i*(n+1)+j
    verts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)
    faces = []
    w = ncell + 1
    for i in range(ncell):
        for j in range(ncell):
            v00 = i * w + j
            v10 = (i + 1) * w + j
            v01 = i * w + j + 1
            v11 = (i + 1) * w + j + 1
            faces.append((v00, v10, v11))
            faces.append((v00, v11, v01))
    return verts, np.array(faces, dtype=np.int64)


def ellipsoid(level: int, semi_axes):
    """Icosphere of unit radius scaled to semi-axes (a, b, c)."""
    v, f = icosphere(level, 1.0)
    return v * np.asarray(semi_axes, dtype=np.float64)[None, :], f


def _zip_rings(ring_a, ring_b, ang_a, ang_b, flip):
    """Triangulate the band between two closed vertex rings by advancing along
    whichever ring has the smaller next angle."""
    na, nb = len(ring_a), len(ring_b)
    ia = ib = 0
    tris = []
    while ia < na or ib < nb:
        next_a = ang_a[ia + 1] if ia < na else np.inf
        next_b = ang_b[ib + 1] if ib < nb else np.inf
        a0, b0 = ring_a[ia % na], ring_b[ib % nb]
        if next_a <= next_b:
            t = (a0, ring_a[(ia + 1) % na], b0)
            ia += 1
        else:
            t = (a0, ring_b[(ib + 1) % nb], b0)
            ib += 1
        tris.append(t[::-1] if flip else t)
    return tris


def closed_cylinder(radius: float, height: float, h: float):
    """Closed circular cylinder (side plus two flat caps) with target edge h.

    The side is an n_phi x n_z grid of quads split into triangles; each cap is
    a set of concentric rings whose vertex counts shrink with the radius,
    zipped together, around a centre vertex.  Closed, outward oriented.
    """
    n_phi = max(6, int(math.ceil(2 * math.pi * radius / h)))
    n_z = max(1, int(math.ceil(height / h)))
    n_r = max(1, int(math.ceil(radius / h)))
    verts = []
    side_rings = []
    for k in range(n_z + 1):
        z = -height / 2 + height * k / n_z
        ring = []
        for i in range(n_phi):
            ph = 2 * math.pi * i / n_phi
            ring.append(len(verts))
            verts.append((radius * math.cos(ph), radius * math.sin(ph), z))
        side_rings.append(ring)
    tris = []
    for k in range(n_z):
        r0, r1 = side_rings[k], side_rings[k + 1]
        for i in range(n_phi):
            a, b = r0[i], r0[(i + 1) % n_phi]
            c, d = r1[i], r1[(i + 1) % n_phi]
            tris.append((a, b, d))
            tris.append((a, d, c))
    for top in (False, True):
        z = height / 2 if top else -height / 2
        outer = side_rings[-1] if top else side_rings[0]
        outer_ang = [2 * math.pi * i / n_phi for i in range(n_phi + 1)]
        rings = [outer]
        angs = [outer_ang]
        for j in range(n_r - 1, 0, -1):
            rr = radius * j / n_r
            nj = max(3, int(round(n_phi * j / n_r)))
            ring = []
            for i in range(nj):
                ph = 2 * math.pi * i / nj
                ring.append(len(verts))
                verts.append((rr * math.cos(ph), rr * math.sin(ph), z))
            rings.append(ring)
            angs.append([2 * math.pi * i / nj for i in range(nj + 1)])
        for q in range(len(rings) - 1):
            # bottom cap seen from below is clockwise in xy: flip for outward -z
            tris += _zip_rings(rings[q], rings[q + 1], angs[q], angs[q + 1],
                               flip=not top)
        centre = len(verts)
        verts.append((0.0, 0.0, z))
        inner = rings[-1]
        m = len(inner)
        for i in range(m):
            t = (inner[i], inner[(i + 1) % m], centre)
            tris.append(t if top else t[::-1])
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int64)


def mesh_stats(verts, tris):
    """Counts used by tests: vertices, triangles, unique edges, boundary edges,
    non-manifold edges, Euler characteristic and enclosed volume (divergence
    theorem; positive when normals point outward)."""
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]],
                                tris[:, [2, 0]]]), axis=1)
    _, counts = np.unique(e, axis=0, return_counts=True)
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    vol = float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)
    return {
        "nv": len(verts), "nt": len(tris), "ne": len(counts),
        "boundary": int((counts == 1).sum()),
        "nonmanifold": int((counts > 2).sum()),
        "euler": len(verts) - len(counts) + len(tris),
        "volume": vol,
    }
