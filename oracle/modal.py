"""Oracle modal Green's functions (test infrastructure only).

For a target x and the source ring at generating-curve parameter s with local
frame (e1, e2, e3): a, b, c = projections of x - gamma(s); r~ = sqrt(a^2+b^2),
alpha = atan2(b, a), phi = theta - alpha,

    rho^2 = r~^2 + r^2 + c^2 - 2 r r~ cos(phi)                (Eq. rho-standard)
    chi   = (r~^2 + r^2 + c^2) / (2 r r~)                       (Sec. 3.3)

All kernels depend on theta only through cos(phi), so their Fourier
coefficients in phi are even in m; in theta they pick up e^{-i m alpha}.
Coefficients use f^_n = int_0^{2 pi} f(phi) e^{-i n phi} dphi.

Static (k = 0), Eq. modal0 and the derivative formulas of Sec. 3.3:
    g^_m   = Q_{|m|-1/2}(chi) / (2 pi sqrt(r~ r))
    dr g^_m = Q'(chi) d_r chi / (2 pi sqrt(r~ r)) - g^_m / (2 r)
    dz g^_m = Q'(chi) d_z chi / (2 pi sqrt(r~ r))
    d_r chi = (r^2 - r~^2 - c^2) / (2 r~ r^2),  d_z chi = -c / (r r~)

k != 0, Eqs. conv and I1: e^{ik rho}/(4 pi rho) = cos(k rho) g + i sin(k rho)/(4 pi rho)
    G^_m = (1/2pi) sum_n f1^_n g^_{m-n} + i f2^_m
with f1 = cos(k rho) and f2 = sin(k rho)/(4 pi rho) sampled on an
equispaced phi-grid and transformed by the FFT.  For the source-derivative
kernels (Sec. 3.3, details deferred by the paper; reading used here) the
same split of G'(rho) gives

    d_r G = cos(k rho) d_r g + h_r g + i p_r,
    h_r = -k^2 sinc(k rho) (r - r~ cos phi),
    p_r = (k rho cos k rho - sin k rho)/(4 pi rho^3) (r - r~ cos phi),

and d_z G the same with (r - r~ cos phi) replaced by -c.  sinc and the
p-factor are functions of rho^2, so every sampled factor is smooth; their
removable singularities are evaluated by Taylor series.

The FFT grid is doubled until the upper half of every spectrum (|n| >= M/4) is below 1e-15
of its maximum or at the transform's own rounding floor, and the convolution runs over the whole grid (no truncation
tolerance: the paper's 1e-12 is a speed setting, the oracle wants the
converged value).

Lagrange weights (Sec. 3.1, inverse DFT against L_j):
    W_j = (1/2N) [G^_0 + 2 sum_{m=1}^{N-1} G^_m cos m(theta_j - alpha) + G^_N cos N(theta_j - alpha)]

Pins: tests/test_oracle_modal.py (brute-force trapezoid on far rings,
adaptive quadrature on near rings, k -> 0 limit, finite differences in r
and z, exactness of W_j for trigonometric polynomials).
"""
from __future__ import annotations

import math

import numpy as np

from .special import dq_half, q_half


def _sinc(x):
    x = np.asarray(x, float)
    small = np.abs(x) < 0.1
    xs = np.where(small, 1.0, x)
    x2 = x * x
    series = 1 - x2 / 6 + x2 ** 2 / 120 - x2 ** 3 / 5040 + x2 ** 4 / 362880
    return np.where(small, series, np.sin(xs) / xs)


def _q3(x):
    """(x cos x - sin x) / x^3, with its Taylor series for |x| < 0.5."""
    x = np.asarray(x, float)
    small = np.abs(x) < 0.5
    xs = np.where(small, 1.0, x)
    x2 = x * x
    series = np.zeros_like(x)
    fact = 6.0  # (2n+1)! for n = 1
    for n in range(1, 13):
        if n > 1:
            fact *= (2 * n) * (2 * n + 1)
        series = series + ((-1) ** n) * (2 * n) / fact * x2 ** (n - 1)
    return np.where(small, series, (xs * np.cos(xs) - np.sin(xs)) / xs ** 3)


def ring_coords(x_local, ring):
    """a, b, c, r~, alpha of a local-frame target against ring data (one s)."""
    v = x_local - ring["gamma"]
    a = float(v @ ring["e1"])
    b = float(v @ ring["e2"])
    c = float(v @ ring["e3"])
    return a, b, c, math.hypot(a, b), math.atan2(b, a)


def modal_coeffs(r: float, rt: float, c: float, k: float, N: int, dr=None):
    """G^_m, d_r G^_m, d_z G^_m for m = 0..N in the phi variable (call with
    N+1 for the extra mode that cos(theta) products need).

    ``dr`` = r - r~ when known more accurately than the difference of the two.
    Returns three complex arrays of length N+1.
    """
    if dr is None:
        dr = r - rt
    # a ring through the target itself (s = s_t) is excluded by the quadrature;
    # the floor only keeps a vanishing neighbourhood finite
    delta = max((dr * dr + c * c) / (2.0 * r * rt), 1e-300)
    chi = 1.0 + delta
    scale = 1.0 / (2.0 * math.pi * math.sqrt(r * rt))
    dchi_r = (dr * (r + rt) - c * c) / (2.0 * rt * r * r)
    dchi_z = -c / (r * rt)

    if k == 0.0:
        q = q_half(delta, N + 1)
        dq = dq_half(delta, q)
        g0 = q[: N + 1] * scale
        return (g0.astype(complex), (dq * dchi_r * scale - g0 / (2 * r)).astype(complex),
                (dq * dchi_z * scale).astype(complex))

    # spectra of the smooth factors on an equispaced phi grid
    M = 64
    while M < 4 * N:
        M *= 2
    while True:
        phi = 2 * np.pi * np.arange(M) / M
        s2 = np.sin(0.5 * phi) ** 2
        rho = np.sqrt(dr * dr + c * c + 4.0 * r * rt * s2)
        kr = k * rho
        sk = _sinc(kr)
        q3 = k ** 3 / (4 * np.pi) * _q3(kr)
        radial = dr + 2.0 * rt * s2  # r - r~ cos(phi)
        samples = np.stack([np.cos(kr), k * sk / (4 * np.pi), -k * k * sk * radial,
                            k * k * sk * c, q3 * radial, -q3 * c])
        spec = np.fft.fft(samples, axis=1) * (2 * np.pi / M)
        H = M // 2
        mag = np.abs(spec)
        top = np.max(mag[:, H // 2: H + H // 2], axis=1)
        # converged when the upper half is at the tail tolerance or at the
        # rounding floor of the transform itself (a few ulps of sum |f|)
        floor = np.maximum(1e-15 * np.max(mag, axis=1),
                           32 * np.finfo(float).eps * np.sum(np.abs(samples), axis=1) * (2 * np.pi / M))
        if np.all(top <= floor) or M >= 1 << 14:
            break
        M *= 2
    H = M // 2 - 1  # use modes -H..H
    idx = np.arange(-H, H + 1)
    sp = spec[:, idx % M]
    f1, f2, hr, h3, pr, p3 = sp

    # static coefficients on -(N+H)..(N+H), and their derivatives
    P = N + H
    q = q_half(delta, P + 1)
    dq = dq_half(delta, q)
    g0h = q[: P + 1] * scale
    dr0h = dq * dchi_r * scale - g0h / (2 * r)
    dz0h = dq * dchi_z * scale
    full = lambda v: np.concatenate([v[:0:-1], v])  # index p = -P..P
    g0, dr0, dz0 = full(g0h), full(dr0h), full(dz0h)

    def conv(fhat, ghat):
        out = np.convolve(fhat, ghat)  # index k <-> m = k - N - 2H
        return out[N + 2 * H: N + 2 * H + N + 1] / (2 * np.pi)

    m = np.arange(N + 1)
    G = conv(f1, g0) + 1j * f2[m + H]
    Gr = conv(f1, dr0) + conv(hr, g0) + 1j * pr[m + H]
    Gz = conv(f1, dz0) + conv(h3, g0) + 1j * p3[m + H]
    return G, Gr, Gz


def _shifted_weights(coef: np.ndarray, alpha: float, n_theta: int):
    """Weights of K cos(phi) (even, coefficients (k^_{m-1} + k^_{m+1})/2) and of
    K sin(phi) (odd, coefficients (k^_{m-1} - k^_{m+1})/(2i)), phi = theta - alpha."""
    N = n_theta // 2
    kk = lambda m: coef[abs(m)]
    even = np.array([0.5 * (kk(m - 1) + kk(m + 1)) for m in range(N + 1)])
    Wc = lagrange_weights(even, alpha, n_theta)
    theta = 2 * np.pi * np.arange(n_theta) / n_theta
    ph = theta - alpha
    Ws = np.zeros(n_theta, complex)
    for m in range(1, N + 1):
        f = 1.0 if m < N else 0.5
        Ws = Ws + f * (kk(m - 1) - kk(m + 1)) * np.sin(m * ph)
    return Wc, Ws / (2 * N)


def lagrange_weights_cos_theta(coef: np.ndarray, alpha: float, n_theta: int):
    """int K(theta - alpha) cos(theta) L_j(theta) dtheta for j = 0..2N-1 from the
    phi-coefficients k^_0..k^_{N+1} of an even kernel K;
    cos(theta) = cos(phi) cos(alpha) - sin(phi) sin(alpha)."""
    Wc, Ws = _shifted_weights(coef, alpha, n_theta)
    return np.cos(alpha) * Wc - np.sin(alpha) * Ws


def lagrange_weights_sin_theta(coef: np.ndarray, alpha: float, n_theta: int):
    """The same with sin(theta) = sin(phi) cos(alpha) + cos(phi) sin(alpha)."""
    Wc, Ws = _shifted_weights(coef, alpha, n_theta)
    return np.sin(alpha) * Wc + np.cos(alpha) * Ws


def lagrange_weights(coef: np.ndarray, alpha: float, n_theta: int):
    """W_j = int G(theta) L_j(theta) dtheta for j = 0..2N-1 from the phi-coefficients."""
    N = n_theta // 2
    theta = 2 * np.pi * np.arange(n_theta) / n_theta
    m = np.arange(1, N)
    ph = theta[:, None] - alpha
    s = coef[0] + 2.0 * np.cos(ph * m[None, :]) @ coef[1:N] + coef[N] * np.cos(N * ph[:, 0])
    return s / (2 * N)
