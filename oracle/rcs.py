"""Radar cross section from RWG currents and the Mie series of a PEC sphere
(Sec. V: bistatic RCS of a sphere compared with the Mie series; monostatic
sweeps of the plate).

  N(rhat)  = sum_n x_n int f_n(r') e^{+jk rhat.r'} ds'      (e^{+jwt}, G ~ e^{-jkr}/4 pi r)
  sigma    = k^2 eta0^2 / (4 pi) |rhat x (rhat x N)|^2 / |E0|^2,
  sigma_pp = k^2 eta0^2 / (4 pi) |p . N|^2 for a polarisation p in {theta-hat, phi-hat}.

Mie series (PEC sphere radius a, x = k a, incident along +z, x-polarised):
  a_n = psi_n'(x) / xi_n'(x),  b_n = psi_n(x) / xi_n(x),  psi_n = x j_n, xi_n = x h_n^(1)
  S1(g) = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),  S2(g) = sum (...)(a_n tau_n + b_n pi_n)
  E-plane sigma(g) = 4 pi |S2(g)|^2 / k^2,  H-plane sigma(g) = 4 pi |S1(g)|^2 / k^2
with g the angle from the propagation direction and pi_n, tau_n from the usual
upward recurrence.

Pinned by: Rayleigh limit sigma_back -> 9 pi a^2 (ka)^4 for ka << 1, optical
limit sigma_back -> pi a^2 for ka >> 1, the optical theorem (integral of the
bistatic cross section over all directions equals 4 pi / k^2 Re S(0)), and
the MoM currents of a sphere agreeing with the Mie series.
"""
import math

import numpy as np
from scipy import special

from .efie import ETA0
from .quadrature import dunavant7


def far_field_vector(rwg, k, X, rhat):
    """N (ndir, 3, nrhs) for currents X (N,) or (N, nrhs) in original order."""
    X = np.asarray(X, dtype=np.complex128).reshape(rwg.n, -1)
    bary, w = dunavant7()
    tv = rwg.verts[rwg.tris]
    Q = np.einsum("qk,tkc->tqc", bary, tv)
    out = np.zeros((len(rhat), 3, X.shape[1]), np.complex128)
    for s, tr, fr in ((1.0, rwg.tri_p, rwg.free_p), (-1.0, rwg.tri_m, rwg.free_m)):
        rp = Q[tr]                                          # (N, 7, 3)
        v = rwg.verts[rwg.tris[tr, fr]]
        rho = rp - v[:, None, :]                            # (N, 7, 3)
        phase = np.exp(1j * k * np.einsum("nqc,dc->dnq", rp, rhat))   # (D, N, 7)
        # int f_n e^{jk rhat.r'} = s (l/2) sum_q w_q rho_q e^{...}
        integ = np.einsum("q,dnq,nqc->dnc", w, phase, rho) * (s * 0.5 * rwg.length)[None, :, None]
        out += np.einsum("dnc,nr->dcr", integ, X)
    return out


def sph_dirs(theta, phi):
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    rhat = np.stack([st * cp, st * sp, ct], axis=-1)
    th = np.stack([ct * cp, ct * sp, -st], axis=-1)
    ph = np.stack([-sp, cp, np.zeros_like(sp)], axis=-1)
    return rhat, th, ph


def rcs(rwg, k, X, theta, phi, pol="theta"):
    """sigma (ndir, nrhs) in m^2 for observation angles (radians)."""
    theta = np.atleast_1d(theta)
    phi = np.broadcast_to(np.atleast_1d(phi), theta.shape)
    rhat, th, ph = sph_dirs(theta, phi)
    N = far_field_vector(rwg, k, X, rhat)
    p = th if pol == "theta" else ph
    comp = np.einsum("dc,dcr->dr", p, N)
    return (k * k * ETA0 * ETA0 / (4 * math.pi)) * np.abs(comp) ** 2


def mie_coefficients(x, nmax=None):
    if nmax is None:
        nmax = int(x + 4.05 * x ** (1 / 3) + 10)
    n = np.arange(1, nmax + 1)
    jn = special.spherical_jn(n, x)
    jnp = special.spherical_jn(n, x, derivative=True)
    yn = special.spherical_yn(n, x)
    ynp = special.spherical_yn(n, x, derivative=True)
    psi = x * jn
    dpsi = jn + x * jnp
    xi = x * (jn + 1j * yn)
    dxi = (jn + 1j * yn) + x * (jnp + 1j * ynp)
    return n, dpsi / dxi, psi / xi


def mie_amplitudes(x, gamma, nmax=None):
    """S1, S2 at scattering angles gamma (radians from the forward direction)."""
    n, a, b = mie_coefficients(x, nmax)
    mu = np.cos(np.atleast_1d(gamma))
    pi_prev = np.zeros_like(mu)
    pi_cur = np.ones_like(mu)
    S1 = np.zeros(mu.shape, np.complex128)
    S2 = np.zeros(mu.shape, np.complex128)
    for idx, nn in enumerate(n):
        if nn > 1:
            pi_new = ((2 * nn - 1) / (nn - 1)) * mu * pi_cur - (nn / (nn - 1)) * pi_prev
            pi_prev, pi_cur = pi_cur, pi_new
        tau = nn * mu * pi_cur - (nn + 1) * pi_prev
        c = (2 * nn + 1) / (nn * (nn + 1))
        S1 += c * (a[idx] * pi_cur + b[idx] * tau)
        S2 += c * (a[idx] * tau + b[idx] * pi_cur)
    return S1, S2


def mie_bistatic(radius, k, gamma, plane="E"):
    S1, S2 = mie_amplitudes(k * radius, gamma)
    S = S2 if plane == "E" else S1
    return 4 * math.pi * np.abs(S) ** 2 / (k * k)


def mie_backscatter(radius, k):
    n, a, b = mie_coefficients(k * radius)
    s = np.sum((2 * n + 1) * (-1.0) ** n * (a - b))
    return math.pi / (k * k) * abs(s) ** 2
