"""Accuracy of the power-series solution against the leaf size (Sec. V-A,
Fig. 4), computed with the CPU oracle.  Test and study infrastructure only.

For one icosphere and a list of octree leaf caps: build the H-matrix and the
scaling (reading A, depth-first order), solve the x-polarised theta = 0 plane
wave by the series with 2, 3 and 5 terms, and compare each with the direct
(LU) solution of the assembled H-matrix, as the paper does with
||x_dir - x_ps|| / ||x_dir||.  The reference is the LU of each cap's own
assembled matrix (`--ref own`, isolates the series truncation) or of the
first cap's matrix for all caps (`--ref first`, one LU for large N; the
matrices differ only by the ACA tolerance).

    python -m oracle.study_leaf_size --level 4 --radius 1.0 --caps 32 64 128 256 512 1024
    python -m oracle.study_leaf_size --level 4 --radius 1.0 --caps 64 256 --eta 1
    python -m oracle.study_leaf_size --level 4 --radius 1.0 --binary 0.25 0.5 1.0 --eta 1
    python -m oracle.study_leaf_size --level 5 --radius 2.0 --caps 128 256 --cfie 0.5

prints one line per cap: leaves, leaf cell edge in wavelengths (min / median
/ max over the leaves), the Eq. 45 ratio ||it_1|| / ||it_0||, and the errors.
"""
import argparse
import time

import numpy as np


def eta_octree(eta):
    """Octree whose admissibility adds the paper's form with constant eta
    (Eq. 10): cells s, t are far when they do not touch and
    min(diam_s, diam_t) <= eta dist(s, t), diam the cell diagonal and dist
    the distance between the cells, on exact integer cell coordinates (the
    oracle's and the GPU library's `eta`, see oracle.octree)."""
    from .octree import Octree

    class EtaOctree(Octree):
        def __init__(self, points, leaf_max):
            super().__init__(points, leaf_max, eta)

    return EtaOctree


class BinaryTree:
    """The paper's binary tree (Sec. II; Sec. IV: every cell is cut in two,
    level by level), for this study only.  Reading: the root is the bounding
    cube of the points; a cell is cut at the midpoint of its longest edge
    (lowest axis among equal edges; a point goes to the upper half when its
    coordinate is >= the midpoint) while both halves keep a longest edge of
    at least `leaf_size` (so every leaf's longest edge lies in [leaf_size,
    2 leaf_size)), "until the block size is greater than or equal to 0.5
    lambda"; empty halves are dropped; leaves are numbered depth first.  Two
    cells are admissible (far) when they are apart and min(diam_s, diam_t) <=
    eta dist(s, t) (Eq. 10, diam = cell diagonal, dist = distance between the
    cells).  Same interface as oracle.octree.Octree for build_hmatrix."""

    class Node:
        def __init__(self, lo, hi, level, start, count):
            self.lo, self.hi, self.level = lo, hi, level
            self.start, self.count = start, count
            self.children = []
            self.leaf = -1

    def __init__(self, points, leaf_size, eta=1.0):
        pts = np.asarray(points, dtype=np.float64)
        lo, hi = pts.min(axis=0), pts.max(axis=0)
        c, half = (lo + hi) / 2.0, float((hi - lo).max()) / 2.0
        self.pts, self.leaf_size, self.eta = pts, float(leaf_size), float(eta)
        self.nodes, self.leaves, perm = [], [], []
        stack = [(list(range(len(pts))), c - half, c + half, 0, None)]
        # depth-first, lower half first (explicit stack: deep trees)
        while stack:
            idx, blo, bhi, level, parent = stack.pop()
            nid = len(self.nodes)
            node = BinaryTree.Node(blo, bhi, level, len(perm), len(idx))
            self.nodes.append(node)
            if parent is not None:
                self.nodes[parent].children.append(nid)
            ext = bhi - blo
            ax = int(np.argmax(ext))
            halves_ok = max(ext[ax] / 2.0, np.delete(ext, ax).max()) >= self.leaf_size
            if not halves_ok or level >= 60:
                node.leaf = len(self.leaves)
                self.leaves.append(nid)
                perm.extend(idx)
                continue
            mid = blo[ax] + ext[ax] / 2.0
            up = [i for i in idx if pts[i, ax] >= mid]
            dn = [i for i in idx if pts[i, ax] < mid]
            hi_dn, lo_up = bhi.copy(), blo.copy()
            hi_dn[ax] = mid
            lo_up[ax] = mid
            for part, plo, phi in ((up, lo_up, bhi), (dn, blo, hi_dn)):   # dn popped first
                if part:
                    stack.append((part, plo, phi, level + 1, nid))
        self.perm = np.array(perm, dtype=np.int64)
        self.leaf_off = np.array([self.nodes[n].start for n in self.leaves] + [len(pts)],
                                 dtype=np.int64)

    @property
    def n_leaves(self):
        return len(self.leaves)

    def touching(self, s, t):
        """True when the pair is not admissible (near)."""
        a, b = self.nodes[s], self.nodes[t]
        gap = np.maximum(0.0, np.maximum(b.lo - a.hi, a.lo - b.hi))
        dist = float(np.linalg.norm(gap))
        diam = min(float(np.linalg.norm(a.hi - a.lo)), float(np.linalg.norm(b.hi - b.lo)))
        return not (dist > 0.0 and diam <= self.eta * dist)

    def blocks(self):
        near, far = [], []
        stack = [(0, 0)]
        while stack:
            s, t = stack.pop()
            if not self.touching(s, t):
                far.append((s, t))
                continue
            ns, nt = self.nodes[s], self.nodes[t]
            if ns.leaf >= 0 and nt.leaf >= 0:
                near.append((ns.leaf, nt.leaf))
            elif ns.leaf >= 0:
                stack.extend((s, c) for c in reversed(nt.children))
            elif nt.leaf >= 0:
                stack.extend((c, t) for c in reversed(ns.children))
            else:
                stack.extend((cs, ct) for cs in reversed(ns.children)
                             for ct in reversed(nt.children))
        return near, far

    def upper_blocks(self):
        near, far = self.blocks()
        near_u = sorted({(i, j) for (i, j) in near if i <= j})
        far_u = sorted((s, t) for (s, t) in far
                       if self.nodes[s].start < self.nodes[t].start)
        far_u.sort(key=lambda st: (self.nodes[st[0]].start, self.nodes[st[1]].start,
                                   self.nodes[st[0]].count, self.nodes[st[1]].count))
        return near_u, far_u


def binary_tree(leaf_size, eta):
    """A tree class for build_hmatrix(points, leaf_max): the binary tree with
    the given leaf size (the leaf_max argument is ignored)."""
    class _T(BinaryTree):
        def __init__(self, points, leaf_max):
            super().__init__(points, leaf_size, eta)
    return _T


def leaf_edges(tree, wavelength):
    """Longest edge of every leaf cell in wavelengths."""
    if isinstance(tree, BinaryTree):
        return np.array([float((tree.nodes[n].hi - tree.nodes[n].lo).max())
                         for n in tree.leaves]) / wavelength
    return np.array([tree.size / 2 ** tree.nodes[n].level for n in tree.leaves]) / wavelength


def main():
    from hm_workloads import icosphere
    from .efie import EFIE
    from .hmatrix import build_hmatrix, default_processes
    from .scaling import compute_scaling
    from .series import series_solve, rel_err
    ap = argparse.ArgumentParser()
    ap.add_argument("--level", type=int, default=4)
    ap.add_argument("--radius", type=float, default=1.0, help="in wavelengths")
    ap.add_argument("--caps", type=int, nargs="+", default=[32, 64, 128, 256, 512, 1024])
    ap.add_argument("--terms", type=int, nargs="+", default=[2, 3, 5])
    ap.add_argument("--ref", choices=["own", "first"], default="own")
    ap.add_argument("--processes", type=int, default=None)
    ap.add_argument("--eta", type=float, default=None,
                    help="admissibility min(diam) <= eta dist instead of non-touching cells")
    ap.add_argument("--cfie", type=float, default=None, metavar="ALPHA",
                    help="the CFIE of Eq. 8 with this alpha instead of the EFIE (non-symmetric "
                         "scaling, oracle.nonsym); reference: the LU of the full CFIE matrix, "
                         "filled once for all caps")
    ap.add_argument("--binary", type=float, nargs="+", default=None, metavar="LEAF_SIZE",
                    help="the paper's binary tree with these leaf sizes (wavelengths) "
                         "instead of octree caps; admissibility eta (default 1)")
    a = ap.parse_args()
    from . import hmatrix
    if a.binary is not None:
        a.caps = a.binary
        a.eta = 1.0 if a.eta is None else a.eta
    elif a.eta is not None:
        hmatrix.Octree = eta_octree(a.eta)
    v, f = icosphere(a.level, a.radius)
    procs = a.processes or default_processes()
    if a.cfie is not None:
        return cfie_study(a, v, f, procs)
    ref = None
    adm = f"eta {a.eta:g}" if a.eta is not None else "non-touching"
    tree = "binary tree, leaf size" if a.binary is not None else "octree, leaf cap"
    print(f"# icosphere L{a.level}, radius {a.radius} lambda, {tree}, admissibility {adm}, "
          f"reference LU ({a.ref})", flush=True)
    print("# cap leaves edge_min edge_med edge_max ratio_eq45 "
          + " ".join(f"err_{t}" for t in a.terms) + " seconds", flush=True)
    for cap in a.caps:
        t0 = time.perf_counter()
        if a.binary is not None:
            hmatrix.Octree = binary_tree(cap, a.eta)
        H = build_hmatrix(v, f, 1.0, cap, 1e-4, processes=procs, use_c=True)
        S = compute_scaling(H, "A")
        B = EFIE(H.rwg, 1.0).plane_wave([0.0], [0.0], [0])
        if ref is None or a.ref == "own":
            xl = np.linalg.solve(H.to_dense(), B[H.perm])
            ref = np.empty_like(xl)
            ref[H.perm] = xl
        errs, ratio = [], None
        for nt in a.terms:
            X, rat = series_solve(H, S, B, nt)
            errs.append(float(rel_err(X, ref)[0]))
            if ratio is None and rat.size:
                ratio = float(rat[0, 0])
        e = leaf_edges(H.tree, 1.0)
        print(f"{cap} {H.n_leaves} {e.min():.3f} {np.median(e):.3f} {e.max():.3f} "
              f"{ratio:.3f} " + " ".join(f"{x:.3e}" for x in errs)
              + f" {time.perf_counter() - t0:.0f}", flush=True)


def cfie_study(a, v, f, procs):
    """The same sweep for the CFIE (Eq. 8, alpha = a.cfie): the full matrix
    filled once, each cap's H-matrix cut from it (far blocks by truncated SVD
    at the ACA tolerance), the non-symmetric scaling (reading A) and series,
    against the LU of the full matrix."""
    from .mfie import CFIE
    from .nonsym import (compute_scaling_general, dense_cfie, hmatrix_from_dense,
                         series_solve_general)
    from .series import rel_err
    t0 = time.perf_counter()
    rwg, Zd = dense_cfie(v, f, 1.0, a.cfie, procs)
    b = CFIE(rwg, 1.0, a.cfie).plane_wave([0.0], [0.0], [0])
    x_ref = np.linalg.solve(Zd, b)
    adm = f"eta {a.eta:g}" if a.eta is not None else "non-touching"
    tree_name = "binary tree, leaf size" if a.binary is not None else "octree, leaf cap"
    print(f"# icosphere L{a.level}, radius {a.radius} lambda, CFIE alpha {a.cfie}, {tree_name}, "
          f"admissibility {adm}, reference LU of the full matrix "
          f"(fill + LU {time.perf_counter() - t0:.0f} s)", flush=True)
    print("# cap leaves edge_min edge_med edge_max ratio_eq45 "
          + " ".join(f"err_{t}" for t in a.terms) + " seconds", flush=True)
    for cap in a.caps:
        t0 = time.perf_counter()
        if a.binary is not None:
            tree = BinaryTree(rwg.centre, cap, a.eta)
            H = hmatrix_from_dense(Zd, rwg, 0, 1e-4, tree=tree)
        else:
            H = hmatrix_from_dense(Zd, rwg, int(cap), 1e-4, a.eta or 0.0)
        S = compute_scaling_general(H, "A")
        errs, ratio = [], None
        for nt in a.terms:
            X, rat = series_solve_general(H, S, b, nt)
            errs.append(float(rel_err(X, x_ref)[0]))
            if ratio is None and rat.size:
                ratio = float(rat[0, 0])
        e = leaf_edges(H.tree, 1.0)
        print(f"{cap} {H.n_leaves} {e.min():.3f} {np.median(e):.3f} {e.max():.3f} "
              f"{ratio:.3f} " + " ".join(f"{x:.3e}" for x in errs)
              + f" {time.perf_counter() - t0:.0f}", flush=True)


if __name__ == "__main__":
    main()
