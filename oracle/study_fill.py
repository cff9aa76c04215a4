"""Memory of the scaling coefficients against N (Sec. IV; Fig. 3 and 5's
scaling study), computed from the structure alone with the CPU oracle.
Test and study infrastructure only.

For icospheres of increasing level at a fixed mesh density (radius doubling
with every level, so about 10 edges per wavelength) and a leaf cap: the octree
block partition, then the number of complex entries of the upper near field
|Z_N| (blocks i <= j), of D (the diagonal blocks) and of alpha under
  reading A  full block-Cholesky fill (Eq. 23 exact), depth-first order,
  reading A  with the nested-dissection order,
  reading B  fill restricted to the near pattern (the paper's memory claim).
No matrix entry is computed: the counts follow from the leaf sizes and the
symbolic elimination (oracle.scaling), as the paper's estimates of Eq. 46-56
do.

    python -m oracle.study_fill --levels 3 4 5 6 --cap 128
"""
import argparse
import time

import numpy as np


def counts(points, cap):
    """(N, leaves, |Z_N upper|, |D|, |alpha| A-DFS, A-ND, B) for one point set."""
    from .octree import Octree
    from .scaling import symbolic_fill, near_pattern, nd_order
    T = Octree(points, cap)
    near_u, _ = T.upper_blocks()
    m = np.diff(T.leaf_off).astype(np.int64)
    zn = int(sum(m[i] * m[j] for (i, j) in near_u))
    d = int(np.sum(m * m))

    def alpha(order, rows_fn):
        pos = {leaf: q for q, leaf in enumerate(order)}
        rows = rows_fn(T.n_leaves, [(pos[i], pos[j]) for (i, j) in near_u])
        mo = m[order]
        return int(sum(mo[k] * mo[j] for k in range(len(rows)) for j in rows[k]))

    dfs = list(range(T.n_leaves))
    nd = nd_order(T, near_u)
    pattern = lambda n, pairs: [sorted(r) for r in near_pattern(n, pairs)]
    return (len(points), T.n_leaves, zn, d, alpha(dfs, symbolic_fill),
            alpha(nd, symbolic_fill), alpha(dfs, pattern))


def main():
    from hm_workloads import icosphere
    from .rwg import build_rwg
    ap = argparse.ArgumentParser()
    ap.add_argument("--levels", type=int, nargs="+", default=[3, 4, 5, 6])
    ap.add_argument("--cap", type=int, default=128)
    a = ap.parse_args()
    print(f"# icospheres at ~10 edges per wavelength (radius 0.5 * 2^(L-3)), leaf cap {a.cap}")
    print("# level N leaves near_upper D alpha_A_dfs alpha_A_nd alpha_B "
          "(alpha / near_upper: A-dfs A-nd B) seconds", flush=True)
    for L in a.levels:
        t0 = time.perf_counter()
        v, f = icosphere(L, 0.5 * 2 ** (L - 3))
        N, nl, zn, d, ad, an, ab = counts(build_rwg(v, f).centre, a.cap)
        print(f"{L} {N} {nl} {zn} {d} {ad} {an} {ab} "
              f"({ad / zn:.2f} {an / zn:.2f} {ab / zn:.2f}) {time.perf_counter() - t0:.0f}",
              flush=True)


if __name__ == "__main__":
    main()
