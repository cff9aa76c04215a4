"""Why the mixed path's error against FP64 depends on the series ratio: a
precision model on the CPU oracle.  Test and study infrastructure only.

The mixed handle runs the series chain in complex64 (alpha, far factors and
vectors; D^-1 in FP64) and one refinement step with an FP64 residual.  With M
the two-term series operator, a chain error delta in x_0 reaches the refined
solution as (I - M Z) delta, so the difference from the FP64 path grows with
how far the truncated series is from Z^-1, which the Eq. 45 ratio indicates.
This script repeats the oracle's series and refinement with alpha and the
far factors rounded to complex64 and every panel rounded to complex64 after
each operator, first with FP64 arithmetic (storage rounding only), then with
the sweeps and the far product multiplying and adding in complex64, and
reports per sampled RHS the relative difference from the FP64 series +
refinement, beside the Eq. 45 ratio.  It models the rounding level of the GPU
chain, not the tensor cores' own rounding.

    python -m oracle.study_mixed_error --workload sphere_r2_L5 --cols 0 90 181 271 361
"""
import argparse

import numpy as np


def _c64_scaling(S):
    """The scaling with alpha in complex64 (D^-1 stays complex128)."""
    import copy
    S32 = copy.copy(S)
    S32.alpha = {k: a.astype(np.complex64) for k, a in S.alpha.items()}
    return S32


def _c64_far(H):
    """The H-matrix with its far blocks in complex64 (near blocks unchanged,
    they enter only the FP64 residual)."""
    import copy
    H32 = copy.copy(H)
    H32.far = [(kind, r0, m, c0, n, P.astype(np.complex64),
                None if Q is None else Q.astype(np.complex64))
               for kind, r0, m, c0, n, P, Q in H.far]
    return H32


def _rt32(S32, leaf_off, b):
    """R^T b (Eq. 25) by forward block substitution in complex64 arithmetic."""
    out = np.array(b, dtype=np.complex64, copy=True)
    sl = S32.slices(leaf_off)
    for k in range(S32.n):
        for j in S32.rows[k]:
            out[sl[j]] += S32.alpha[(k, j)].T @ out[sl[k]]
    return out


def _r32(S32, leaf_off, x):
    """R x (Eq. 26) by back block substitution in complex64 arithmetic."""
    out = np.array(x, dtype=np.complex64, copy=True)
    sl = S32.slices(leaf_off)
    for k in range(S32.n - 1, -1, -1):
        for j in S32.rows[k]:
            out[sl[k]] += S32.alpha[(k, j)] @ out[sl[j]]
    return out


def _far32(H32, x):
    """Z_F x with complex64 factors, vectors and sums."""
    y = np.zeros_like(x, dtype=np.complex64)
    for kind, r0, m, c0, n, P, Q in H32.far:
        rs, cs = slice(r0, r0 + m), slice(c0, c0 + n)
        if kind == "lr":
            y[rs] += P @ (Q.T @ x[cs])
            y[cs] += Q @ (P.T @ x[rs])
        else:
            y[rs] += P @ x[cs]
            y[cs] += P.T @ x[rs]
    return y


def mixed_model(H, S, B, arithmetic=True):
    """(x_mixed, x_fp64) with one refinement step each; the mixed chain on
    complex64 arrays and vectors, the residual in FP64."""
    from .series import series_solve_perm
    H32, S32 = _c64_far(H), _c64_scaling(S)
    Bp = np.asarray(B, np.complex128)[H.perm]

    from .scaling import apply_Rt, apply_R, apply_Dinv
    off = H.leaf_off
    c64 = lambda v: np.asarray(v).astype(np.complex64).astype(np.complex128)

    Rt, R = (_rt32, _r32) if arithmetic else (apply_Rt, apply_R)
    far = (lambda v: _far32(H32, v.astype(np.complex64))) if arithmetic else H32.far_apply

    def chain32(b):
        # the two-term series of Eq. 25-36 with every panel held in complex64
        # between operators, as the GPU chain keeps them; with `arithmetic`
        # the sweeps and the far product also multiply and add in complex64
        bo = c64(apply_Dinv(S, off, c64(Rt(S32, off, c64(b)))))
        z = c64(far(c64(R(S32, off, bo))))
        wv = c64(apply_Dinv(S, off, c64(Rt(S32, off, z))))
        return c64(R(S32, off, c64(bo - wv)))

    def chain64(b):
        return series_solve_perm(H, S, b, 2)[0]

    out = []
    for chain in (chain32, chain64):
        x = chain(Bp)
        x = x + chain(Bp - H.apply(x))
        X = np.empty_like(x)
        X[H.perm] = x
        out.append(X)
    return out


def main():
    from hm_workloads import get_workload
    from .efie import EFIE
    from .hmatrix import build_hmatrix, default_processes
    from .scaling import compute_scaling, nd_order
    from .series import rel_err, series_solve
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sphere_r2_L5")
    ap.add_argument("--cols", type=int, nargs="+", default=[0])
    a = ap.parse_args()
    w = get_workload(a.workload)
    v, f = w.build_mesh()
    H = build_hmatrix(v, f, w.wavelength, w.leaf_max, w.aca_tol,
                      processes=default_processes(), use_c=True)
    S = compute_scaling(H, "A", nd_order(H.tree, list(H.near.keys())))
    th, ph, po = w.angles()
    B = EFIE(H.rwg, w.wavelength).plane_wave(th, ph, po)[:, a.cols]
    _, ratio = series_solve(H, S, B, 2)
    xs, x64 = mixed_model(H, S, B, arithmetic=False)
    xa, _ = mixed_model(H, S, B, arithmetic=True)
    es, ea = rel_err(xs, x64), rel_err(xa, x64)
    print(f"# {a.workload}: N={H.N}, columns {a.cols}")
    print("# column ratio_eq45 storage_rounding_only complex64_arithmetic "
          "(relative difference from the FP64 series + refinement)")
    for c, r, e1, e2 in zip(a.cols, ratio[0], es, ea):
        print(f"{c} {r:.3f} {e1:.2e} {e2:.2e}")


if __name__ == "__main__":
    main()
