"""Writer (and reader, for round-trip tests) of the neutral block file through
which the GPU library imports an oracle H-matrix, its leaf order and, when
given, its scaling coefficients.  Little-endian; complex numbers as (re, im)
float64 pairs; every matrix row-major.

  magic      8 bytes  b"HMPSBLK1"
  int64      N, n_leaves, n_near, n_far, reading (0 = A, 1 = B, -1 = none), has_scaling
  float64    wavelength, k
  int64      perm[N]                     leaf position -> original RWG index
  int64      leaf_off[n_leaves + 1]
  near x n_near:   int64 i, j (i <= j);  complex128 block[m_i * m_j]
  far  x n_far:    int64 kind (0 low rank, 1 dense), r0, m, c0, n, rank;
                   kind 0: U[m * rank], V[n * rank]  (block = U V^T)
                   kind 1: B[m * n]
  if has_scaling (k, j below are elimination ranks; leaf elim[k] is eliminated k-th):
    int64 n_alpha
    int64 elim[n_leaves]
    per rank k: int64 count, int64 j[count]   (the stored row of alpha)
    alpha blocks in that order: complex128 [m_elim[k] * m_elim[j]]
    Dinv per rank: complex128 [m_elim[k] * m_elim[k]]
  optional sections to the end of the file, each an 8-byte tag and its data:
    b"LEAFCEN1"  float64 cen[n_leaves * 3]     leaf cell centres (the input of
                                               the nested-dissection order)
    b"SUPERND1"  (after scaling only) int64 n_groups, int64 grp[n_groups + 1]
                 (group g = ranks grp[g] .. grp[g+1]-1), then for every group
                 with more than one leaf T_G = (I - A_G^T)^-1, complex128
                 [n_G * n_G] (oracle.scaling.supernode_inverse)
    b"NONSYM01"  a non-symmetric system (the CFIE, oracle.nonsym): the main
                 sections then hold the blocks of their own order only (near
                 i <= j, far blocks whose row cluster starts first), applied
                 without transposes, and this section the rest:
                 int64 n; n x (int64 i, j (i > j); complex128 block[m_i * m_j]);
                 int64 n; n far blocks as above (row cluster after column cluster);
                 int64 has_left; if 1, per (k, j) in alpha's order the left
                 coefficient alphaL_kj transposed, complex128 [m_elim[k] * m_elim[j]]

Parity unpinned beyond the round trip: this is a file format, not arithmetic.
"""
import struct

import numpy as np

MAGIC = b"HMPSBLK1"


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128).tobytes()


def leaf_centres(H):
    """Cell centres of the octree leaves, in the unit cube of the root (the
    coordinates oracle.scaling.nd_order splits on)."""
    return np.array([[(H.tree.nodes[nid].ijk[a] + 0.5) / (1 << H.tree.nodes[nid].level)
                      for a in range(3)] for nid in H.tree.leaves], dtype=np.float64)


def write_blocks(path, H, S=None, centres=True, groups=None):
    """``centres``: append the leaf cell centres (when H carries its tree);
    ``groups``: supernode boundaries in elimination ranks (with S): append
    the groups and their T_G."""
    m = np.diff(H.leaf_off)
    with open(path, "wb") as f:
        f.write(MAGIC)
        reading = -1 if S is None else (0 if S.reading == "A" else 1)
        f.write(struct.pack("<6q", H.N, H.n_leaves, len(H.near), len(H.far),
                            reading, 0 if S is None else 1))
        f.write(struct.pack("<2d", float(H.meta.get("wavelength", 1.0)), float(H.k)))
        f.write(np.ascontiguousarray(H.perm, dtype="<i8").tobytes())
        f.write(np.ascontiguousarray(H.leaf_off, dtype="<i8").tobytes())
        for (i, j) in sorted(H.near):
            f.write(struct.pack("<2q", i, j))
            f.write(_c(H.near[(i, j)]))
        for kind, r0, mm, c0, n, P, Q in H.far:
            if kind == "lr":
                f.write(struct.pack("<6q", 0, r0, mm, c0, n, P.shape[1]))
                f.write(_c(P))
                f.write(_c(Q))
            else:
                f.write(struct.pack("<6q", 1, r0, mm, c0, n, 0))
                f.write(_c(P))
        if S is not None:
            f.write(struct.pack("<q", len(S.alpha)))
            f.write(np.asarray(S.order, dtype="<i8").tobytes())
            for k in range(S.n):
                f.write(struct.pack("<q", len(S.rows[k])))
                f.write(np.asarray(S.rows[k], dtype="<i8").tobytes())
            for k in range(S.n):
                for j in S.rows[k]:
                    f.write(_c(S.alpha[(k, j)]))
            for k in range(S.n):
                f.write(_c(S.Dinv[k]))
        if centres and getattr(H, "tree", None) is not None:
            f.write(b"LEAFCEN1")
            f.write(np.ascontiguousarray(leaf_centres(H), dtype="<f8").tobytes())
        if groups is not None:
            from .scaling import supernode_inverse
            assert S is not None and groups[0] == 0 and groups[-1] == S.n
            f.write(b"SUPERND1")
            f.write(struct.pack("<q", len(groups) - 1))
            f.write(np.asarray(groups, dtype="<i8").tobytes())
            for g in range(len(groups) - 1):
                if groups[g + 1] - groups[g] > 1:
                    f.write(_c(supernode_inverse(S, H.leaf_off, groups[g], groups[g + 1])))


def write_blocks_nonsym(path, H, S=None):
    """Block file of a non-symmetric H-matrix (oracle.nonsym.HMatrixGen) and
    its left and right scaling (ScalingGen): the main sections with the upper
    blocks and alpha, D^-1, then the NONSYM01 section."""
    from types import SimpleNamespace
    up_near = {ij: B for ij, B in H.near.items() if ij[0] <= ij[1]}
    lo_near = {ij: B for ij, B in H.near.items() if ij[0] > ij[1]}
    up_far = [b for b in H.far if b[1] < b[3]]
    lo_far = [b for b in H.far if b[1] > b[3]]
    assert len(up_far) + len(lo_far) == len(H.far)
    Hup = SimpleNamespace(N=H.N, n_leaves=H.n_leaves, near=up_near, far=up_far, perm=H.perm,
                          leaf_off=H.leaf_off, k=H.k, meta=H.meta)
    write_blocks(path, Hup, S, centres=False)
    with open(path, "ab") as f:
        f.write(b"NONSYM01")
        f.write(struct.pack("<q", len(lo_near)))
        for (i, j) in sorted(lo_near):
            f.write(struct.pack("<2q", i, j))
            f.write(_c(lo_near[(i, j)]))
        f.write(struct.pack("<q", len(lo_far)))
        for kind, r0, mm, c0, n, P, Q in lo_far:
            if kind == "lr":
                f.write(struct.pack("<6q", 0, r0, mm, c0, n, P.shape[1]))
                f.write(_c(P))
                f.write(_c(Q))
            else:
                f.write(struct.pack("<6q", 1, r0, mm, c0, n, 0))
                f.write(_c(P))
        f.write(struct.pack("<q", 0 if S is None else 1))
        if S is not None:
            for k in range(S.n):
                for j in S.rows[k]:
                    f.write(_c(S.alphaL[(k, j)].T))


def read_blocks(path):
    """Inverse of write_blocks -> dict of numpy arrays (tests only).  The file
    is memory-mapped: the arrays are read-only views of it."""
    import mmap
    with open(path, "rb") as fh:
        buf = mmap.mmap(fh.fileno(), 0, access=mmap.ACCESS_READ)
    assert buf[:8] == MAGIC
    pos = 8

    def take(fmt):
        nonlocal pos
        out = struct.unpack_from(fmt, buf, pos)
        pos += struct.calcsize(fmt)
        return out

    def arr(dtype, count):
        nonlocal pos
        a = np.frombuffer(buf, dtype=dtype, count=count, offset=pos)
        pos += a.nbytes
        return a

    N, nl, nn, nf, reading, has_s = take("<6q")
    wl, k = take("<2d")
    perm = arr("<i8", N)
    off = arr("<i8", nl + 1)
    m = np.diff(off)
    near = {}
    for _ in range(nn):
        i, j = take("<2q")
        near[(i, j)] = arr("<c16", m[i] * m[j]).reshape(m[i], m[j])

    def far_block():
        kind, r0, mm, c0, n, r = take("<6q")
        if kind == 0:
            return ("lr", r0, mm, c0, n, arr("<c16", mm * r).reshape(mm, r),
                    arr("<c16", n * r).reshape(n, r))
        return ("dense", r0, mm, c0, n, arr("<c16", mm * n).reshape(mm, n), None)

    far = [far_block() for _ in range(nf)]
    out = dict(N=N, perm=perm, leaf_off=off, near=near, far=far, k=k,
               wavelength=wl, reading=reading)
    if has_s:
        (na,) = take("<q")
        elim = arr("<i8", nl).tolist()
        me = m[elim]
        rows = []
        for kk in range(nl):
            (c,) = take("<q")
            rows.append(arr("<i8", c).tolist())
        alpha = {}
        for kk in range(nl):
            for j in rows[kk]:
                alpha[(kk, j)] = arr("<c16", me[kk] * me[j]).reshape(me[kk], me[j])
        dinv = [arr("<c16", me[kk] * me[kk]).reshape(me[kk], me[kk]) for kk in range(nl)]
        assert len(alpha) == na
        out.update(rows=rows, alpha=alpha, Dinv=dinv, elim=elim)
    while pos < len(buf):
        tag = buf[pos:pos + 8]
        pos += 8
        if tag == b"LEAFCEN1":
            out["leaf_cen"] = arr("<f8", 3 * nl).reshape(nl, 3)
        elif tag == b"SUPERND1":
            assert has_s
            (ng,) = take("<q")
            grp = arr("<i8", ng + 1).tolist()
            me = m[out["elim"]]
            T = {}
            for g in range(ng):
                if grp[g + 1] - grp[g] > 1:
                    nG = int(np.sum(me[grp[g]:grp[g + 1]]))
                    T[g] = arr("<c16", nG * nG).reshape(nG, nG)
            out.update(groups=grp, T=T)
        elif tag == b"NONSYM01":
            (nlo,) = take("<q")
            for _ in range(nlo):
                i, j = take("<2q")
                assert i > j
                near[(i, j)] = arr("<c16", m[i] * m[j]).reshape(m[i], m[j])
            (nfl,) = take("<q")
            far.extend(far_block() for _ in range(nfl))
            (has_l,) = take("<q")
            if has_l:
                me = m[out["elim"]]
                out["alphaL"] = {(kk, j): arr("<c16", me[kk] * me[j]).reshape(me[kk], me[j]).T
                                 for kk in range(nl) for j in out["rows"][kk]}
            out["nonsym"] = True
        else:
            raise ValueError(f"unknown section {tag!r}")
    assert pos == len(buf)
    return out


def load_blocks(path):
    """(H, S) of the oracle from a block file written by the GPU library
    (hm_save): its H-matrix and, when present, its scaling coefficients, so
    that the oracle's series can check the library on the library's own
    blocks ("imported blocks").  S.D is not in the file (None)."""
    from .hmatrix import HMatrix
    from .scaling import Scaling
    d = read_blocks(path)
    H = HMatrix(N=int(d["N"]), perm=np.asarray(d["perm"]), leaf_off=np.asarray(d["leaf_off"]),
                near=d["near"], far=d["far"], k=float(d["k"]),
                meta={"wavelength": float(d["wavelength"])})
    S = None
    if "alpha" in d:
        S = Scaling(n=len(d["elim"]), rows=d["rows"], alpha=d["alpha"], D=None,
                    Dinv=d["Dinv"], reading="A" if d["reading"] == 0 else "B",
                    order=d["elim"])
    return H, S
