"""Closed-form surface integrals of 1/R and (r' - rho)/R over a flat triangle,
R = |r - r'|, rho = projection of the observation point r onto the triangle's
plane.  They carry the static part of the Green's function of Eq. 3 on
self and touching triangle pairs (singularity extraction), in the form derived
by Wilton, Rao, Glisson et al. (1984) and Graglia (1993).

For each edge i of the triangle (running from p_a to p_b in vertex order):
  lhat = unit edge direction, uhat = lhat x nhat (in-plane outward normal),
  l+ = (p_b - rho).lhat, l- = (p_a - rho).lhat,
  t  = (p_a - rho).uhat        (signed distance of rho from the edge line),
  h  = nhat.(r - p_a)          (height of r above the plane),
  R0 = sqrt(t^2 + h^2), R+- = sqrt(R0^2 + l+-^2),
  f  = ln((R+ + l+) / (R- + l-)),
  beta = atan(t l+ / (R0^2 + |h| R+)) - atan(t l- / (R0^2 + |h| R-)).
Then
  int 1/R ds'            = sum_i ( t_i f_i - |h| beta_i )
  int (r' - rho)/R ds'   = 1/2 sum_i uhat_i ( R0_i^2 f_i + l+_i R+_i - l-_i R-_i ).

Pinned by: Duffy-transformed Gauss-Legendre brute force (singular point in the
plane, near point above the plane) to 1e-10, and the far-field limit
int 1/R -> A/|r - c|.
"""
import numpy as np


def static_potentials(obs, tri):
    """obs: (P, 3) observation points; tri: (P, 3, 3) triangle vertices.

    Returns (I_s (P,), I_v (P, 3), rho (P, 3)) with I_s = int_T 1/R ds' and
    I_v = int_T (r' - rho)/R ds'.
    """
    obs = np.asarray(obs, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.float64)
    p0, p1, p2 = tri[:, 0], tri[:, 1], tri[:, 2]
    n = np.cross(p1 - p0, p2 - p0)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    h = np.einsum("pc,pc->p", n, obs - p0)
    rho = obs - h[:, None] * n
    ah = np.abs(h)
    I_s = np.zeros(len(obs))
    I_v = np.zeros((len(obs), 3))
    for pa, pb in ((p0, p1), (p1, p2), (p2, p0)):
        e = pb - pa
        elen = np.linalg.norm(e, axis=1)
        lhat = e / elen[:, None]
        uhat = np.cross(lhat, n)
        lp = np.einsum("pc,pc->p", pb - rho, lhat)
        lm = np.einsum("pc,pc->p", pa - rho, lhat)
        t = np.einsum("pc,pc->p", pa - rho, uhat)
        R0sq = t * t + h * h
        Rp = np.sqrt(R0sq + lp * lp)
        Rm = np.sqrt(R0sq + lm * lm)
        # f = ln((R+ + l+)/(R- + l-)).  When rho projects beyond the p_a end of
        # the edge line (l- < 0) the same value is ln((R- - l-)/(R+ - l+)),
        # which avoids the cancellation in R + l.
        degenerate = R0sq <= (1e-14 * elen) ** 2
        with np.errstate(divide="ignore", invalid="ignore"):
            f_pos = np.log((Rp + lp) / (Rm + lm))
            f_neg = np.log((Rm - lm) / (Rp - lp))
        f = np.where(lm + lp >= 0.0, f_pos, f_neg)
        f = np.where(degenerate, 0.0, f)
        with np.errstate(divide="ignore", invalid="ignore"):
            beta = (np.arctan(t * lp / (R0sq + ah * Rp)) -
                    np.arctan(t * lm / (R0sq + ah * Rm)))
        beta = np.where(ah > 0.0, beta, 0.0)
        beta = np.where(degenerate, 0.0, beta)
        I_s += t * f - ah * beta
        I_v += 0.5 * uhat * (R0sq * f + lp * Rp - lm * Rm)[:, None]
    return I_s, I_v, rho


def static_gradient(obs, tri):
    """obs: (P, 3); tri: (P, 3, 3).  Returns int_T (r - r') / R^3 ds' (P, 3),
    the static kernel of the MFIE's K operator (minus the gradient of the
    1/R potential above), in the same edge quantities:
      int_T (r - r')/R^3 ds' = sum_i uhat_i f_i + sign(h) nhat sum_i beta_i
    (in-plane part from the edge logarithms, normal part the solid angle the
    triangle subtends at r).  At h = 0 the normal part is zero (principal
    value); the in-plane part is singular on the triangle's edges only.

    Pinned by: brute-force Gauss-Legendre quadrature on the collapsed square
    at points above, below and beside the triangle (gradient_brute), and
    the finite-difference gradient of static_potentials' int 1/R."""
    obs = np.asarray(obs, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.float64)
    p0, p1, p2 = tri[:, 0], tri[:, 1], tri[:, 2]
    n = np.cross(p1 - p0, p2 - p0)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    h = np.einsum("pc,pc->p", n, obs - p0)
    rho = obs - h[:, None] * n
    ah = np.abs(h)
    out = np.zeros((len(obs), 3))
    bsum = np.zeros(len(obs))
    for pa, pb in ((p0, p1), (p1, p2), (p2, p0)):
        e = pb - pa
        elen = np.linalg.norm(e, axis=1)
        lhat = e / elen[:, None]
        uhat = np.cross(lhat, n)
        lp = np.einsum("pc,pc->p", pb - rho, lhat)
        lm = np.einsum("pc,pc->p", pa - rho, lhat)
        t = np.einsum("pc,pc->p", pa - rho, uhat)
        R0sq = t * t + h * h
        Rp = np.sqrt(R0sq + lp * lp)
        Rm = np.sqrt(R0sq + lm * lm)
        degenerate = R0sq <= (1e-14 * elen) ** 2
        with np.errstate(divide="ignore", invalid="ignore"):
            f_pos = np.log((Rp + lp) / (Rm + lm))
            f_neg = np.log((Rm - lm) / (Rp - lp))
            beta = (np.arctan(t * lp / (R0sq + ah * Rp)) -
                    np.arctan(t * lm / (R0sq + ah * Rm)))
        f = np.where(lm + lp >= 0.0, f_pos, f_neg)
        f = np.where(degenerate, 0.0, f)
        beta = np.where(degenerate, 0.0, beta)
        out += uhat * f[:, None]
        bsum += beta
    out += (np.sign(h) * bsum)[:, None] * n
    return out


def gradient_brute(obs, tri, order=200):
    """Brute-force reference for int_T (r - r')/R^3 ds' at one point off the
    triangle: the collapsed-square map r' = p0 + u (p1 - p0) + u v (p2 - p1)
    (Jacobian 2 A u) with an order x order Gauss-Legendre rule.  Tests only."""
    obs = np.asarray(obs, dtype=np.float64)
    p0, p1, p2 = np.asarray(tri, dtype=np.float64)
    x, w = np.polynomial.legendre.leggauss(order)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    U, V = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    area2 = np.linalg.norm(np.cross(p1 - p0, p2 - p0))
    r = p0 + U[..., None] * (p1 - p0) + (U * V)[..., None] * (p2 - p1)
    d = obs - r
    R = np.linalg.norm(d, axis=-1)
    return np.einsum("uv,uvc->c", W * U * area2 / R ** 3, d)


def duffy_brute(obs, tri, order=48):
    """Brute-force reference for (I_s, I_v) at one point: split the triangle at
    the projection rho into three sub-triangles with apex rho, map each to the
    unit square with the Duffy transform (Jacobian proportional to the radial
    coordinate, which cancels the 1/R singularity for h = 0) and apply an
    order x order Gauss-Legendre rule.  Used only by tests."""
    obs = np.asarray(obs, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.float64)
    p0, p1, p2 = tri
    n = np.cross(p1 - p0, p2 - p0)
    n /= np.linalg.norm(n)
    h = np.dot(n, obs - p0)
    rho = obs - h * n
    x, w = np.polynomial.legendre.leggauss(order)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    U, V = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    Is = 0.0
    Iv = np.zeros(3)
    for a, b in ((p0, p1), (p1, p2), (p2, p0)):
        # signed area of (rho, a, b) relative to the triangle normal
        area2 = np.dot(np.cross(a - rho, b - rho), n)
        # r'(u, v) = rho + u((1-v)(a - rho) + v(b - rho)), dA = u * area2 du dv
        d = (1 - V)[..., None] * (a - rho) + V[..., None] * (b - rho)
        rp = rho + U[..., None] * d
        R = np.linalg.norm(obs - rp, axis=-1)
        jac = U * area2
        Is += np.sum(W * jac / R)
        Iv += np.einsum("uv,uvc->c", W * jac / R, rp - rho)
    return Is, Iv
