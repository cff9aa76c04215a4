"""EFIE Galerkin matrix entries and plane-wave excitation (Eq. 1-3, 9).

Reading of the garbled signs in Eq. 2-3: time convention e^{+j w t}, Green's
function G = e^{-jkR} / (4 pi R), and

  Z_mn = j w mu <f_m, f_n G> - (j / (w eps)) <div f_m, div' f_n G>
       = j eta0 * sum_{a in T_m+-, b in T_n+-} s_a s_b l_m l_n [ (k/4) A_ij(a,b) - S0(a,b) / k ]

  b_m  = <f_m, E_inc>,  E_inc = p e^{-jk khat.r},
         khat = -(sin t cos p, sin t sin p, cos t)  (incident from (t, p))

where for the triangle pair (a, b) with normalised 7x7-point sums
  S0 = sum w_p w_q G(r_p, r_q),   S1 = sum w_p w_q G r_q,
  S2 = sum w_p w_q G r_p,         S3 = sum w_p w_q G (r_p . r_q),
and A_ij = S3 - (S2 . v_j + v_i . S1) + (v_i . v_j) S0 for the free vertices
v_i of a and v_j of b.  (Areas cancel: each triangle integral is A * sum w.)

Singularity extraction: on pairs that share at least one vertex, G is split
into 1/(4 pi R), integrated in closed form over the inner triangle
(oracle.potentials), plus (e^{-jkR} - 1)/(4 pi R), integrated by the 7x7 rule
(its R -> 0 limit is -jk/(4 pi)).  The closed form is always taken over the
triangle with the higher index, the 7-point rule over the lower one, so the
pair sums of (a, b) and (b, a) are the same numbers and Z = Z^T up to rounding;
stored blocks are mirrored so that the stored matrix is exactly symmetric.

Pinned by: symmetry and reciprocity of Z, agreement of the closed form with
brute-force quadrature (potentials), and (after the solve) the Mie series of a
PEC sphere (rcs).  The smooth 7x7 part is checked against a 16x16-point
collapsed Gauss product rule on separated pairs.
"""
import math

import numpy as np

from .quadrature import dunavant7, triangle_points
from .potentials import static_potentials

C0 = 299792458.0
MU0 = 4e-7 * math.pi
EPS0 = 1.0 / (MU0 * C0 * C0)
ETA0 = MU0 * C0


class EFIE:
    """Entry evaluator for one mesh at one wavelength."""

    def __init__(self, rwg, wavelength=1.0):
        self.rwg = rwg
        self.k = 2.0 * math.pi / wavelength
        self.eta = ETA0
        self.tv = rwg.verts[rwg.tris]                    # (nt, 3, 3)
        self.Q = triangle_points(self.tv)                # (nt, 7, 3)
        _, self.w = dunavant7()
        self.ww = np.outer(self.w, self.w)               # (7, 7)

    # ---------------------------------------------------------------- pairs
    def touching(self, Ta, Tb):
        """(A, B) bool: triangles share at least one vertex."""
        ta = self.rwg.tris[Ta]
        tb = self.rwg.tris[Tb]
        eq = ta[:, None, :, None] == tb[None, :, None, :]
        return eq.any(axis=(2, 3))

    def pair_moments(self, Ta, Tb, chunk=48):
        """S0 (A,B), S1 (A,B,3), S2 (A,B,3), S3 (A,B) for all pairs of the
        triangle index arrays Ta x Tb (see module docstring)."""
        Ta = np.asarray(Ta, dtype=np.int64)
        Tb = np.asarray(Tb, dtype=np.int64)
        A, B = len(Ta), len(Tb)
        S0 = np.empty((A, B), np.complex128)
        S1 = np.empty((A, B, 3), np.complex128)
        S2 = np.empty((A, B, 3), np.complex128)
        S3 = np.empty((A, B), np.complex128)
        for s in range(0, A, chunk):
            e = min(A, s + chunk)
            S0[s:e], S1[s:e], S2[s:e], S3[s:e] = self._smooth_moments(Ta[s:e], Tb)
        touch = self.touching(Ta, Tb)
        ia, ib = np.nonzero(touch)
        if len(ia):
            ga, gb = Ta[ia], Tb[ib]
            lo = np.minimum(ga, gb)
            hi = np.maximum(ga, gb)
            s0, s_in, s_out, s3 = self._static_pair(lo, hi)
            # self pairs: the exact inner and outer moments are equal; take the
            # mean of the two numerical ones so the pair is symmetric
            same = (ga == gb)[:, None]
            mean = 0.5 * (s_in + s_out)
            s_in = np.where(same, mean, s_in)
            s_out = np.where(same, mean, s_out)
            swap = (ga > gb)[:, None]
            S0[ia, ib] += s0
            S3[ia, ib] += s3
            S1[ia, ib] += np.where(swap, s_out, s_in)
            S2[ia, ib] += np.where(swap, s_in, s_out)
        return S0, S1, S2, S3

    def _smooth_moments(self, Ta, Tb):
        """7x7-point sums of G (or of G - 1/(4 pi R) on touching pairs).

        Arrays are laid out (a, p, b, q): test triangle, its point, source
        triangle, its point.  Real and imaginary parts are separate float64
        arrays: G = (cos kR - j sin kR) / (4 pi R)."""
        k = self.k
        A, B = len(Ta), len(Tb)
        rp = self.Q[Ta].reshape(A * 7, 3)
        rq = self.Q[Tb].reshape(B * 7, 3)
        R2 = np.zeros((A * 7, B * 7))
        for c in range(3):
            dc = rp[:, c][:, None] - rq[:, c][None, :]
            dc *= dc
            R2 += dc
        R = np.sqrt(R2, out=R2)
        kR = k * R
        Gr = np.cos(kR)
        Gi = np.sin(kR)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = (1.0 / (4.0 * math.pi)) / R      # inf only on self pairs,
            Gr *= inv                              # which are replaced below
            Gi *= inv
        np.negative(Gi, out=Gi)
        Gr = Gr.reshape(A, 7, B, 7)
        Gi = Gi.reshape(A, 7, B, 7)
        R = R.reshape(A, 7, B, 7)
        ia, ib = np.nonzero(self.touching(Ta, Tb))
        if len(ia):
            # touching pairs: drop the static 1/(4 pi R) part; R = 0 -> -jk/(4 pi)
            Rt = R[ia, :, ib, :]
            zero = Rt == 0.0
            with np.errstate(divide="ignore", invalid="ignore"):
                gr = (np.cos(k * Rt) - 1.0) / (4.0 * math.pi * Rt)
                gi = -np.sin(k * Rt) / (4.0 * math.pi * Rt)
            Gr[ia, :, ib, :] = np.where(zero, 0.0, gr)
            Gi[ia, :, ib, :] = np.where(zero, -k / (4.0 * math.pi), gi)
        dot = (rp @ rq.T).reshape(A, 7, B, 7)
        rp3 = rp.reshape(A, 7, 3)
        rq3 = rq.reshape(B, 7, 3)
        wp = self.w[None, :, None, None]
        wq = self.w[None, None, None, :]
        out = []
        for G in (Gr, Gi):
            G *= wp
            G *= wq
            Gp = G.sum(axis=3)                           # (A, 7, B): summed over q
            Gq = G.sum(axis=1)                           # (A, B, 7): summed over p
            out.append((Gq.sum(axis=2),
                        np.einsum("abq,bqc->abc", Gq, rq3),
                        np.einsum("apb,apc->abc", Gp, rp3),
                        (G * dot).sum(axis=(1, 3))))
        (r0, r1, r2, r3), (i0, i1, i2, i3) = out
        return r0 + 1j * i0, r1 + 1j * i1, r2 + 1j * i2, r3 + 1j * i3

    def _static_pair(self, outer, inner):
        """Closed-form 1/(4 pi R) part for pairs (outer, inner): the outer
        triangle by the 7-point rule, the inner one analytically.  Returns the
        normalised sums (s0, s_inner_moment, s_outer_moment, s3)."""
        P = len(outer)
        obs = self.Q[outer].reshape(P * 7, 3)
        tri = np.repeat(self.tv[inner], 7, axis=0)
        I_s, I_v, rho = static_potentials(obs, tri)
        I_s = I_s.reshape(P, 7)
        Jv = (I_v + rho * I_s.reshape(-1)[:, None]).reshape(P, 7, 3)   # int r'/R
        rp = self.Q[outer]
        scale = self.w[None, :] / (4.0 * math.pi * self.rwg.area[inner])[:, None]
        s0 = (scale * I_s).sum(axis=1)
        s_in = np.einsum("pq,pqc->pc", scale, Jv)
        s_out = np.einsum("pq,pq,pqc->pc", scale, I_s, rp)
        s3 = np.einsum("pq,pqc,pqc->p", scale, rp, Jv)
        return s0, s_in, s_out, s3

    # ---------------------------------------------------------------- blocks
    def block(self, rows, cols):
        """Dense Z[rows][:, cols] (complex128) for RWG index arrays."""
        rwg = self.rwg
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        Ta = np.unique(np.concatenate([rwg.tri_p[rows], rwg.tri_m[rows]]))
        Tb = np.unique(np.concatenate([rwg.tri_p[cols], rwg.tri_m[cols]]))
        S0, S1, S2, S3 = self.pair_moments(Ta, Tb)
        k = self.k
        lm = rwg.length[rows]
        ln = rwg.length[cols]
        terms = {}
        for sa, (tr, fr) in ((1.0, (rwg.tri_p, rwg.free_p)), (-1.0, (rwg.tri_m, rwg.free_m))):
            ia = np.searchsorted(Ta, tr[rows])
            va = rwg.verts[rwg.tris[tr[rows], fr[rows]]]
            for sb, (tc, fc) in ((1.0, (rwg.tri_p, rwg.free_p)), (-1.0, (rwg.tri_m, rwg.free_m))):
                ib = np.searchsorted(Tb, tc[cols])
                vb = rwg.verts[rwg.tris[tc[cols], fc[cols]]]
                s0 = S0[np.ix_(ia, ib)]
                s1 = S1[np.ix_(ia, ib)]
                s2 = S2[np.ix_(ia, ib)]
                s3 = S3[np.ix_(ia, ib)]
                A = (s3 - (np.einsum("mnc,nc->mn", s2, vb) + np.einsum("mc,mnc->mn", va, s1))
                     + (va @ vb.T) * s0)
                terms[(sa, sb)] = (sa * sb) * np.outer(lm, ln) * ((k / 4.0) * A - s0 / k)
        Z = (terms[(1.0, 1.0)] + terms[(-1.0, -1.0)]) + (terms[(1.0, -1.0)] + terms[(-1.0, 1.0)])
        return 1j * self.eta * Z

    def dense(self, chunk=128):
        """Full N x N matrix, symmetrised as (Z + Z^T)/2 (exactly symmetric)."""
        N = self.rwg.n
        Z = np.empty((N, N), dtype=np.complex128)
        cols = np.arange(N)
        for s in range(0, N, chunk):
            rows = np.arange(s, min(N, s + chunk))
            Z[rows] = self.block(rows, cols)
        return 0.5 * (Z + Z.T)

    # ---------------------------------------------------------------- RHS
    def plane_wave(self, theta, phi, pol):
        """B (N, nrhs) for incidence angles (radians) and pol (0 theta, 1 phi)."""
        rwg = self.rwg
        theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
        phi = np.atleast_1d(np.asarray(phi, dtype=np.float64))
        pol = np.atleast_1d(np.asarray(pol))
        st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
        khat = -np.stack([st * cp, st * sp, ct], axis=1)                 # (R, 3)
        th_hat = np.stack([ct * cp, ct * sp, -st], axis=1)
        ph_hat = np.stack([-sp, cp, np.zeros_like(sp)], axis=1)
        phat = np.where((pol == 0)[:, None], th_hat, ph_hat)             # (R, 3)
        B = np.zeros((rwg.n, len(theta)), dtype=np.complex128)
        for s, tr, fr in ((1.0, rwg.tri_p, rwg.free_p), (-1.0, rwg.tri_m, rwg.free_m)):
            rp = self.Q[tr]                                              # (N, 7, 3)
            v = rwg.verts[rwg.tris[tr, fr]]                              # (N, 3)
            phase = np.exp(-1j * self.k * np.einsum("nqc,rc->nqr", rp, khat))
            proj = np.einsum("nqc,rc->nqr", rp - v[:, None, :], phat)
            B += s * (0.5 * rwg.length)[:, None] * np.einsum("q,nqr->nr", self.w, proj * phase)
        return B
