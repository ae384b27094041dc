"""Closed-form references that pin the oracle (independent of it).

* Mie series for a sound-soft sphere of radius a (textbook separation of
  variables), in the normalisation u ~ e^{ik|x|}/|x| u_inf of Sec. 6:
      u_inf(xhat) = (i/k) sum_n (2n+1) [j_n(ka)/h_n(ka)] P_n(xhat.d).
* Eigenvalues of the boundary operators on the sphere (addition theorem):
      S Y_n = ik a^2 j_n(ka) h_n(ka) Y_n,
      D Y_n = (ik^2 a^2/2) [j_n(ka) h_n'(ka) + j_n'(ka) h_n(ka)] Y_n.
* The point-source field sum_l e^{ik|x-z_l|}/(4 pi |x - z_l|) (Eq. artificial
  point source solution) and its far field sum_l e^{-ik xhat.z_l}/(4 pi).

Spherical Bessel functions come from scipy (library routines).
"""
from __future__ import annotations

import numpy as np
from scipy import special as sp


def _h(n, z, derivative=False):
    return sp.spherical_jn(n, z, derivative) + 1j * sp.spherical_yn(n, z, derivative)


def mie_farfield(a: float, k: float, d, xhat, nmax: int = None):
    d = np.asarray(d, float)
    xhat = np.asarray(xhat, float)
    ka = k * a
    if nmax is None:
        nmax = int(ka + 4 * ka ** (1 / 3) + 20)
    cosg = xhat @ d
    out = np.zeros(cosg.shape, complex)
    for n in range(nmax + 1):
        out += (2 * n + 1) * sp.spherical_jn(n, ka) / _h(n, ka) * sp.eval_legendre(n, cosg)
    return 1j / k * out


def sphere_eigen(a: float, k: float, n: int, eta: float):
    """Eigenvalue of 1/2 + D - i eta S on spherical harmonics of degree n."""
    ka = k * a
    if k == 0:
        # static limits: S Y_n = a/(2n+1) Y_n, D Y_n = -1/(2(2n+1)) Y_n
        return 0.5 - 1.0 / (2 * (2 * n + 1)) - 1j * eta * a / (2 * n + 1)
    j, jd = sp.spherical_jn(n, ka), sp.spherical_jn(n, ka, True)
    h, hd = _h(n, ka), _h(n, ka, True)
    S = 1j * k * a * a * j * h
    D = 0.5j * k * k * a * a * (j * hd + jd * h)
    return 0.5 + D - 1j * eta * S


def point_source_field(x, z, k: float):
    x = np.asarray(x, float)
    out = np.zeros(x.shape[:-1], complex)
    for zl in np.atleast_2d(z):
        r = np.linalg.norm(x - zl, axis=-1)
        out += np.exp(1j * k * r) / (4 * np.pi * r)
    return out


def point_source_farfield(xhat, z, k: float):
    xhat = np.asarray(xhat, float)
    out = np.zeros(xhat.shape[:-1], complex)
    for zl in np.atleast_2d(z):
        out += np.exp(-1j * k * (xhat @ zl)) / (4 * np.pi)
    return out


def sphere_layer_potentials(a: float, k: float, n: int, r: float):
    """(s_n, d_n): single- and double-layer potentials of a degree-n
    spherical harmonic density Y on the sphere of radius a, at radius r != a,
    are s_n Y(xhat) and d_n Y(xhat) (addition theorem for G):
        r > a:  s_n = ik a^2 j_n(ka) h_n(kr),   d_n = ik^2 a^2 j_n'(ka) h_n(kr),
        r < a:  s_n = ik a^2 h_n(ka) j_n(kr),   d_n = ik^2 a^2 h_n'(ka) j_n(kr)."""
    ka, kr = k * a, k * r
    if r > a:
        return (1j * k * a * a * sp.spherical_jn(n, ka) * _h(n, kr),
                1j * k * k * a * a * sp.spherical_jn(n, ka, True) * _h(n, kr))
    return (1j * k * a * a * _h(n, ka) * sp.spherical_jn(n, kr),
            1j * k * k * a * a * _h(n, ka, True) * sp.spherical_jn(n, kr))
