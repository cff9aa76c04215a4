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

prints one line per cap: leaves, leaf cell edge in wavelengths (min / median
/ max over the leaves), the Eq. 45 ratio ||it_1|| / ||it_0||, and the errors.
"""
import argparse
import time

import numpy as np


def eta_octree(eta):
    """Octree whose admissibility is the paper's form with constant eta
    (Eq. 10): cells s, t are far when min(diam_s, diam_t) <= eta dist(s, t),
    diam the cell diagonal and dist the distance between the cells, and
    never when they touch.  For the study only; the oracle and the GPU
    library use non-touching admissibility."""
    import math
    from .octree import Octree

    class EtaOctree(Octree):
        def touching(self, s, t):          # True = not admissible (near)
            a, b = self.nodes[s], self.nodes[t]
            ca, cb = self.size / 2 ** a.level, self.size / 2 ** b.level
            lo_a = self.origin + np.array(a.ijk) * ca
            lo_b = self.origin + np.array(b.ijk) * cb
            gap = np.maximum(0.0, np.maximum(lo_b - (lo_a + ca), lo_a - (lo_b + cb)))
            dist = float(np.linalg.norm(gap))
            return not (dist > 0.0 and math.sqrt(3.0) * min(ca, cb) <= eta * dist)

    return EtaOctree


def leaf_edges(tree, wavelength):
    """Cell edge of every leaf in wavelengths."""
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
    a = ap.parse_args()
    if a.eta is not None:
        from . import hmatrix
        hmatrix.Octree = eta_octree(a.eta)
    v, f = icosphere(a.level, a.radius)
    procs = a.processes or default_processes()
    ref = None
    adm = f"eta {a.eta:g}" if a.eta is not None else "non-touching"
    print(f"# icosphere L{a.level}, radius {a.radius} lambda, admissibility {adm}, "
          f"reference LU ({a.ref})", flush=True)
    print("# cap leaves edge_min edge_med edge_max ratio_eq45 "
          + " ".join(f"err_{t}" for t in a.terms) + " seconds", flush=True)
    for cap in a.caps:
        t0 = time.perf_counter()
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


if __name__ == "__main__":
    main()
