"""Oracle layer potential at off-surface points (test infrastructure only).

For the near-field evaluation of the scattered field (Sec. 6, the field
compared with Eq. artificial point source solution at test points) the
quantity the discretisation defines at a point x off the surface of one
body is the combined-layer potential of the *interpolated* density
(Sec. 3.1: P_l(s) on each panel, trigonometric L_j(theta) with the
symmetric Nyquist term), with the same readings as the self blocks
(selfblock.py): the double layer integrates the exact area-weighted normal
against the interpolant of mu, the single layer the interpolant of mu |J|,

    u_b(x) = int int { (|J| n)(s,theta) . grad_y G(x, y(s,theta)) mu_I(s,theta)
                       - i eta G(x, y(s,theta)) (mu |J|)_I(s,theta) } ds dtheta,

    G = e^{ik rho}/(4 pi rho),  grad_y G . m = (ik - 1/rho) G m.(y - x)/rho.

This is written out as a plain 2-D integral over the parameter domain of
every panel: theta by the trapezoidal rule (the integrand is periodic and
analytic off the surface) doubled until it settles, s by adaptive
Gauss-Kronrod 7/15 bisection.  No modal Green's functions and no graded
rules: an independent route to what the library's near-field rows compute.

Pins: tests/test_oracle_nearfield.py (Gauss's lemma at k = 0 for the double
layer of a unit density, -1 inside and 0 outside at points close to curved
and paper-shape surfaces, which holds exactly for the interpolated density
because the interpolant of a constant is that constant; the single- and
double-layer potentials of spherical harmonics on a sphere, closed forms
from the addition theorem, to the interpolation error; the plain smooth rule
at points far from the body).
"""
from __future__ import annotations

import numpy as np

from .geometry import BodyNodes, gauss_legendre
from .selfblock import _WG, _WK, _XK, lagrange_basis


def _trig_coeffs(v: np.ndarray) -> np.ndarray:
    """Coefficients c_m (m = -N+1..N-1 at index m mod 2N, and c_N) of the
    trigonometric interpolant of samples v[..., j] at theta_j = j pi/N, with
    the Nyquist term taken as c_N cos(N theta)."""
    return np.fft.fft(v, axis=-1) / v.shape[-1]


def _trig_grid(c: np.ndarray, M: int) -> np.ndarray:
    """The interpolant with coefficients c [..., 2N] on the uniform grid
    theta_q = 2 pi q / M (M a multiple of 2N):
    sum_{|m| < N} c_m e^{i m theta} + c_N cos(N theta), by zero-padding."""
    nth = c.shape[-1]
    N = nth // 2
    pad = np.zeros(c.shape[:-1] + (M,), complex)
    pad[..., :N] = c[..., :N]
    pad[..., M - N + 1:] = c[..., N + 1:]
    pad[..., N] = 0.5 * c[..., N]
    pad[..., M - N] = 0.5 * c[..., N]
    return np.fft.ifft(pad, axis=-1) * M


def _theta_integrand(x_loc, geom, s: float, th: np.ndarray, mu: np.ndarray, mj: np.ndarray, k: float,
                     eta: float) -> np.ndarray:
    """(|J| n).grad_y G mu_I - i eta G (mu|J|)_I at (s, th) for interpolant
    values mu, mj [R, len(th)]."""
    S = np.full(th.shape, s)
    y = geom.local_points(S, th)
    _, _, jac = geom.normal_parts(S, th)
    nloc = geom.local_normals(S, th)
    d = y - x_loc[None, :]                                # y - x
    rho = np.sqrt(np.sum(d * d, axis=1))
    G = np.exp(1j * k * rho) / (4 * np.pi * rho)
    dn = (1j * k - 1.0 / rho) * G * np.sum(nloc * d, axis=1) / rho   # grad_y G . n
    return (jac * dn)[None, :] * mu - 1j * eta * G[None, :] * mj


def _theta_integral(x_loc, geom, s: float, cmu: np.ndarray, cmj: np.ndarray, k: float, eta: float,
                    M0: int, rtol: float):
    """int_0^{2pi} of the integrand at one s by the trapezoidal rule, doubled
    (reusing the previous points) until two successive values agree to rtol,
    for the R columns whose theta-coefficients at s are cmu, cmj [R, 2N]."""
    M = M0
    th = 2 * np.pi * np.arange(M) / M
    f = _theta_integrand(x_loc, geom, s, th, _trig_grid(cmu, M), _trig_grid(cmj, M), k, eta)
    fsum, asum = f.sum(axis=1), np.abs(f).sum(axis=1)
    val = fsum * (2 * np.pi / M)
    while M < 1 << 17:
        M *= 2
        odd = 2 * np.pi * (2 * np.arange(M // 2) + 1) / M
        f = _theta_integrand(x_loc, geom, s, odd, _trig_grid(cmu, M)[:, 1::2], _trig_grid(cmj, M)[:, 1::2], k, eta)
        fsum, asum = fsum + f.sum(axis=1), asum + np.abs(f).sum(axis=1)
        new = fsum * (2 * np.pi / M)
        # relative to the integral of |integrand| (robust when the integral itself cancels)
        done = np.max(np.abs(new - val)) <= rtol * max(float(np.max(asum)) * 2 * np.pi / M, 1e-300)
        val = new
        if done:
            break
    return val


def near_field(bn: BodyNodes, mu: np.ndarray, x, k: float, eta: float, tol: float = 1e-13):
    """Layer potential of body ``bn``'s interpolated density mu [n] or
    [n, R] (node order panel -> l -> j) at the world point x (not on the
    surface): the sum of the 2-D integrals over every panel."""
    mu = np.asarray(mu, complex)
    vec = mu.ndim == 1
    if vec:
        mu = mu[:, None]
    R = mu.shape[1]
    g = bn.geom
    x_loc = g.to_local(np.asarray(x, float))
    nth, order = bn.n_theta, bn.order
    xg, _ = gauss_legendre(order)
    total = np.zeros(R, complex)
    for p in range(bn.n_panels):
        a, b = bn.breaks[p], bn.breaks[p + 1]
        sl = slice(p * order * nth, (p + 1) * order * nth)
        mup = mu[sl].reshape(order, nth, R).transpose(2, 0, 1)           # [R, order, 2N]
        jp = bn.jac[sl].reshape(order, nth)
        cmu = _trig_coeffs(mup)                                           # [R, order, 2N]
        cmj = _trig_coeffs(mup * jp[None])
        nodes_s = 0.5 * (a + b) + 0.5 * (b - a) * xg

        def f_of_s(s):
            P = lagrange_basis(nodes_s, s)                                # [order]
            cu = np.einsum("l,rlm->rm", P, cmu)
            cj = np.einsum("l,rlm->rm", P, cmj)
            return _theta_integral(x_loc, g, s, cu, cj, k, eta, 4 * nth, 1e-14)

        # adaptive Gauss-Kronrod 7/15 on [a, b], bisecting the worst interval
        def gk(lo, hi):
            c, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
            vals = np.array([f_of_s(c + h * t) for t in _XK])             # [15, R]
            kr = h * (_WK @ vals)
            ga = h * (_WG @ vals)
            return kr, float(np.max(np.abs(kr - ga))), h * float(np.max(_WK @ np.abs(vals)))

        pieces = [(lo, hi) + gk(lo, hi) for lo, hi in ((a, 0.5 * (a + b)), (0.5 * (a + b), b))]
        for _ in range(400):
            est = sum(pc[3] for pc in pieces)
            # relative to the integral of |f| (the panel's value may cancel to nearly 0)
            scale = max(sum(pc[4] for pc in pieces), 1e-300)
            if est <= tol * scale:
                break
            i = max(range(len(pieces)), key=lambda q: pieces[q][3])
            lo, hi = pieces.pop(i)[:2]
            mid = 0.5 * (lo + hi)
            pieces += [(lo, mid) + gk(lo, mid), (mid, hi) + gk(mid, hi)]
        total += sum(pc[2] for pc in pieces)
    return total[0] if vec else total
