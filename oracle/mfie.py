"""MFIE and CFIE Galerkin matrix entries and plane-wave right-hand sides
(Sec. II, Eq. 4-8), for closed PEC surfaces.  Test and study infrastructure.

MFIE (Eq. 6), tested with the RWG functions f_m (Galerkin):
  <f_m, n x H_inc> = 1/2 <f_m, J> - <f_m, n x int J(r') x grad' G ds'>
so with J = sum_n x_n f_n
  M_mn = 1/2 <f_m, f_n> - K_mn,   K_mn = int f_m . [n x int f_n x grad' G ds'] ds,
  b_m  = <f_m, n x H_inc>,  H_inc = (1/eta0) khat x E_inc,
in the time convention and Green's function of the EFIE (oracle.efie):
G = e^{-jkR} / (4 pi R), grad' G = g(R) (r - r'), g = (1 + jkR) e^{-jkR} / (4 pi R^3)
(Eq. 7).  n is the outward unit normal of the test triangle, taken from the
vertex order (counter-clockwise seen from outside).

Reduction used for every triangle pair (test triangle a, free vertex v_i,
source triangle b, free vertex v_j; f_m = s_a l_m / (2 A_a) (r - v_i) on a,
f_n = s_b l_n / (2 A_b) (r' - v_j) on b): with d = r - r' and the identity
u . [n x (v x w)] = (u . v)(n . w) - (u . w)(n . v),
  f_m . [n x (f_n x g d)] = c (g) [ ((r - v_i).(r - v_j)) (n . d) - (n . (r - v_j)) ((r - v_i) . d) ]
(the terms in (r - v_i).d (n.d) cancel), so the source integral only enters
through the vector V(r) = int_b g(R) (r - r') ds'.  On a flat triangle
n . d = 0 and n . (r - v_j) = 0 when b = a: the self term of K is zero.

V(r) on the 7 test points of a: separated pairs by the 7-point rule over b;
pairs that share a vertex split g into the static 1/(4 pi R^3) part, whose
integral int_b (r - r')/R^3 ds' has the closed form of
oracle.potentials.static_gradient, and g - 1/(4 pi R^3) (bounded times d) by
the 7-point rule.  The outer integral over a is the 7-point rule, as in the
EFIE.  Per pair the moments
  M0 = sum w nu_p,  M1 = sum w nu_p r_p,  M2 = sum w nu_p |r_p|^2,
  M3 = sum w r_p . V_p,  M4 = sum w V_p       (nu_p = n_a . V_p)
give for the free vertices v_i, v_j (e_a = n_a . r on the plane of a)
  T = M2 - M1.v_j - v_i.M1 + (v_i.v_j) M0 - (e_a - n_a.v_j)(M3 - v_i.M4),
  K_mn = sum_{a,b} s_a s_b l_m l_n / (4 A_b) T.

CFIE (Eq. 8): Z = alpha Z_EFIE + eta0 (1 - alpha) M, b = alpha b_EFIE +
eta0 (1 - alpha) b_MFIE (alpha = 0.5 for closed bodies, Sec. II).  Not
symmetric: its near and far blocks are stored for both orders
(oracle.nonsym).

Pinned by: the closed form against brute force (potentials), K = 0 on a
plane (every pair coplanar) so that M is half the Gram matrix computed by an
independent exact rule, outward normals, the Mie series of a PEC sphere
(MFIE and CFIE currents), and the well-conditioned CFIE at an interior
resonance of the sphere where the EFIE and MFIE matrices are nearly singular.
"""
import math

import numpy as np

from .efie import EFIE, ETA0
from .potentials import static_gradient
from .quadrature import dunavant7, triangle_points


class MFIE:
    """Entry evaluator for one closed mesh at one wavelength."""

    def __init__(self, rwg, wavelength=1.0):
        self.rwg = rwg
        self.k = 2.0 * math.pi / wavelength
        self.eta = ETA0
        self.tv = rwg.verts[rwg.tris]                    # (nt, 3, 3)
        self.Q = triangle_points(self.tv)                # (nt, 7, 3)
        _, self.w = dunavant7()
        nv = np.cross(self.tv[:, 1] - self.tv[:, 0], self.tv[:, 2] - self.tv[:, 0])
        self.nrm = nv / np.linalg.norm(nv, axis=1, keepdims=True)

    def touching(self, Ta, Tb):
        ta = self.rwg.tris[Ta]
        tb = self.rwg.tris[Tb]
        eq = ta[:, None, :, None] == tb[None, :, None, :]
        return eq.any(axis=(2, 3))

    def potentials(self, Ta, Tb):
        """V (A, 7, B, 3): int over source triangle b of g(R) (r_p - r') ds'
        at the 7 points r_p of test triangle a."""
        k = self.k
        A, B = len(Ta), len(Tb)
        rp = self.Q[Ta].reshape(A * 7, 3)
        rq = self.Q[Tb].reshape(B * 7, 3)
        d = rp[:, None, :] - rq[None, :, :]                       # (A7, B7, 3)
        R = np.sqrt(np.einsum("pqc,pqc->pq", d, d))
        kR = k * R
        c, s = np.cos(kR), np.sin(kR)
        # (1 + jkR) e^{-jkR} = (c + kR s) + j (kR c - s)
        num_r = c + kR * s
        num_i = kR * c - s
        touch = np.zeros((A * 7, B * 7), bool)
        ia, ib = np.nonzero(self.touching(Ta, Tb))
        if len(ia):
            tmask = np.zeros((A, B), bool)
            tmask[ia, ib] = True
            touch = np.repeat(np.repeat(tmask, 7, axis=0), 7, axis=1)
        num_r = np.where(touch, num_r - 1.0, num_r)               # static part apart
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / (4.0 * math.pi * R ** 3)
        same = np.zeros((A, B), bool)
        same[:, :] = np.asarray(Ta)[:, None] == np.asarray(Tb)[None, :]
        same7 = np.repeat(np.repeat(same, 7, axis=0), 7, axis=1)
        g = np.where(same7, 0.0, (num_r + 1j * num_i) * np.where(same7, 0.0, inv))
        g *= np.tile(self.w, B)[None, :]                          # source weights
        V = np.empty((A * 7, B, 3), np.complex128)
        gq = g.reshape(A * 7, B, 7)
        dq = d.reshape(A * 7, B, 7, 3)
        for cc in range(3):
            V[:, :, cc] = np.einsum("pbq,pbq->pb", gq, dq[..., cc])
        V *= self.rwg.area[Tb][None, :, None]
        V = V.reshape(A, 7, B, 3)
        if len(ia):
            keep = np.asarray(Ta)[ia] != np.asarray(Tb)[ib]
            ia, ib = ia[keep], ib[keep]
        if len(ia):
            obs = self.Q[np.asarray(Ta)[ia]].reshape(-1, 3)
            tri = np.repeat(self.tv[np.asarray(Tb)[ib]], 7, axis=0)
            st = static_gradient(obs, tri).reshape(len(ia), 7, 3) / (4.0 * math.pi)
            V[ia, :, ib, :] += st
        return V

    def pair_moments(self, Ta, Tb, chunk=32):
        """M0 (A,B), M1 (A,B,3), M2 (A,B), M3 (A,B), M4 (A,B,3) (module doc)."""
        Ta = np.asarray(Ta, dtype=np.int64)
        Tb = np.asarray(Tb, dtype=np.int64)
        A, B = len(Ta), len(Tb)
        M0 = np.empty((A, B), np.complex128)
        M1 = np.empty((A, B, 3), np.complex128)
        M2 = np.empty((A, B), np.complex128)
        M3 = np.empty((A, B), np.complex128)
        M4 = np.empty((A, B, 3), np.complex128)
        for s in range(0, A, chunk):
            e = min(A, s + chunk)
            V = self.potentials(Ta[s:e], Tb)                      # (a, 7, B, 3)
            rp = self.Q[Ta[s:e]]                                  # (a, 7, 3)
            na = self.nrm[Ta[s:e]]                                # (a, 3)
            wv = V * self.w[None, :, None, None]
            nu = np.einsum("apbc,ac->apb", wv, na)                # w_p nu_p
            M0[s:e] = nu.sum(axis=1)
            M1[s:e] = np.einsum("apb,apc->abc", nu, rp)
            M2[s:e] = np.einsum("apb,ap->ab", nu, np.einsum("apc,apc->ap", rp, rp))
            M3[s:e] = np.einsum("apbc,apc->ab", wv, rp)
            M4[s:e] = wv.sum(axis=1)
        return M0, M1, M2, M3, M4

    def block(self, rows, cols):
        """Dense M[rows][:, cols] (complex128, amperes per unit current)."""
        rwg = self.rwg
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        Ta = np.unique(np.concatenate([rwg.tri_p[rows], rwg.tri_m[rows]]))
        Tb = np.unique(np.concatenate([rwg.tri_p[cols], rwg.tri_m[cols]]))
        M0, M1, M2, M3, M4 = self.pair_moments(Ta, Tb)
        lm = rwg.length[rows]
        ln = rwg.length[cols]
        out = np.zeros((len(rows), len(cols)), np.complex128)
        for sa, tr, fr in ((1.0, rwg.tri_p, rwg.free_p), (-1.0, rwg.tri_m, rwg.free_m)):
            ta = tr[rows]
            ia = np.searchsorted(Ta, ta)
            va = rwg.verts[rwg.tris[ta, fr[rows]]]                # (m, 3)
            na = self.nrm[ta]
            ea = np.einsum("mc,mc->m", na, self.tv[ta, 0])        # n_a . r on plane a
            rp = self.Q[ta]                                       # (m, 7, 3)
            for sb, tc, fc in ((1.0, rwg.tri_p, rwg.free_p), (-1.0, rwg.tri_m, rwg.free_m)):
                tb = tc[cols]
                ib = np.searchsorted(Tb, tb)
                vb = rwg.verts[rwg.tris[tb, fc[cols]]]            # (n, 3)
                m0 = M0[np.ix_(ia, ib)]
                m1 = M1[np.ix_(ia, ib)]
                m2 = M2[np.ix_(ia, ib)]
                m3 = M3[np.ix_(ia, ib)]
                m4 = M4[np.ix_(ia, ib)]
                T = (m2 - np.einsum("mnc,nc->mn", m1, vb) - np.einsum("mc,mnc->mn", va, m1)
                     + (va @ vb.T) * m0
                     - (ea[:, None] - na @ vb.T) * (m3 - np.einsum("mc,mnc->mn", va, m4)))
                fac = (sa * sb) * np.outer(lm, ln) / (4.0 * rwg.area[tb])[None, :]
                out -= fac * T
                # identity term on shared triangles: 1/2 <f_m, f_n>
                same = ta[:, None] == tb[None, :]
                if same.any():
                    gram = (np.einsum("q,mqc,nc->mn", self.w, rp, -vb)
                            + np.einsum("q,mqc,mqc->m", self.w, rp, rp)[:, None]
                            - (va @ np.einsum("q,nqc->nc", self.w, self.Q[tb]).T)
                            + va @ vb.T)
                    # sum_p w_p (r_p - v_i).(r_p - v_j) with r_p on the common triangle
                    gram = np.where(same, gram, 0.0)
                    out += 0.5 * fac * gram
        return out

    def dense(self, chunk=96):
        N = self.rwg.n
        Z = np.empty((N, N), dtype=np.complex128)
        cols = np.arange(N)
        for s in range(0, N, chunk):
            rows = np.arange(s, min(N, s + chunk))
            Z[rows] = self.block(rows, cols)
        return Z

    def plane_wave(self, theta, phi, pol):
        """B (N, nrhs): <f_m, n x H_inc> for the plane waves of EFIE.plane_wave."""
        rwg = self.rwg
        theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
        phi = np.atleast_1d(np.asarray(phi, dtype=np.float64))
        pol = np.atleast_1d(np.asarray(pol))
        st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
        khat = -np.stack([st * cp, st * sp, ct], axis=1)
        th_hat = np.stack([ct * cp, ct * sp, -st], axis=1)
        ph_hat = np.stack([-sp, cp, np.zeros_like(sp)], axis=1)
        phat = np.where((pol == 0)[:, None], th_hat, ph_hat)
        hdir = np.cross(khat, phat) / self.eta                   # H_inc / e^{-jk khat.r}
        B = np.zeros((rwg.n, len(theta)), dtype=np.complex128)
        for s, tr, fr in ((1.0, rwg.tri_p, rwg.free_p), (-1.0, rwg.tri_m, rwg.free_m)):
            rp = self.Q[tr]                                       # (N, 7, 3)
            v = rwg.verts[rwg.tris[tr, fr]]
            nt = self.nrm[tr]                                     # (N, 3)
            nxh = np.cross(nt[:, None, :], hdir[None, :, :])      # (N, R, 3)
            phase = np.exp(-1j * self.k * np.einsum("nqc,rc->nqr", rp, khat))
            proj = np.einsum("nqc,nrc->nqr", rp - v[:, None, :], nxh)
            B += s * (0.5 * rwg.length)[:, None] * np.einsum("q,nqr->nr", self.w, proj * phase)
        return B


class CFIE:
    """alpha EFIE + eta0 (1 - alpha) MFIE (Eq. 8), entries and right-hand sides."""

    def __init__(self, rwg, wavelength=1.0, alpha=0.5):
        self.rwg = rwg
        self.alpha = float(alpha)
        self.E = EFIE(rwg, wavelength)
        self.M = MFIE(rwg, wavelength)
        self.k = self.E.k
        self.eta = ETA0

    def block(self, rows, cols):
        a = self.alpha
        out = a * self.E.block(rows, cols) if a != 0.0 else 0.0
        if a != 1.0:
            out = out + self.eta * (1.0 - a) * self.M.block(rows, cols)
        return out

    def dense(self, chunk=96):
        N = self.rwg.n
        Z = np.empty((N, N), dtype=np.complex128)
        cols = np.arange(N)
        for s in range(0, N, chunk):
            rows = np.arange(s, min(N, s + chunk))
            Z[rows] = self.block(rows, cols)
        return Z

    def plane_wave(self, theta, phi, pol):
        a = self.alpha
        return (a * self.E.plane_wave(theta, phi, pol)
                + self.eta * (1.0 - a) * self.M.plane_wave(theta, phi, pol))
