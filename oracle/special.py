"""Oracle special functions (test infrastructure only).

* complete elliptic integrals K, E by the arithmetic-geometric mean of Gauss;
* half-integer Legendre functions of the second kind Q_{m-1/2}(chi), chi > 1,
  from the starting values of Sec. 3.3
      Q_{-1/2} = mu K(mu),  Q_{1/2} = chi mu K(mu) - sqrt(2(chi+1)) E(mu),
      mu = sqrt(2/(chi+1)),
  and the three-term recursion (Eq. leg_recur);
* their chi-derivatives by Eq. dleg_recur.

The paper defers the stability treatment of the recursion to a cited work
that is not at hand.  Reading used here: the recursion is run forward from
the two starting values when acosh(chi) * m_max <= 0.5 (the dominant
solution can grow by at most e^0.5 over the range), and otherwise backward
(Miller's algorithm, on ratios, from m_start = m_max + 20 + 40/acosh(chi))
normalised by Q_{-1/2}.

The elliptic modulus is called ``mu`` as in the paper; chi is passed as its
excess delta = chi - 1 >= 0 so that rings close to the target keep full
relative precision.

Pins: tests/test_oracle_special.py (K(0) = E(0) = pi/2, Legendre's relation,
library K/E, direct quadrature of the defining integral, mpmath's Legendre Q,
recursion residuals, forward/backward agreement, derivative by finite
differences).
"""
from __future__ import annotations

import math

import numpy as np


def ellip_KE(mu: float, mu_c: float):
    """K(mu), E(mu) by the AGM; ``mu_c`` = sqrt(1 - mu^2) passed separately
    (accurate when mu -> 1)."""
    a, b, c = 1.0, mu_c, mu
    s = 0.5 * c * c  # sum 2^(n-1) c_n^2, n = 0
    p = 0.5
    for _ in range(60):
        an = 0.5 * (a + b)
        bn = math.sqrt(a * b)
        cn = 0.25 * c * c / an  # c_{n+1} = (a_n - b_n)/2 written without cancellation
        a, b, c = an, bn, cn
        p *= 2.0
        s += p * c * c
        if c < 1e-18 * a:
            break
    K = math.pi / (2.0 * a)
    return K, K * (1.0 - s)


def q_half(delta: float, m_max: int):
    """Q_{m-1/2}(1 + delta) for m = 0..m_max (numpy array)."""
    chi = 1.0 + delta
    mu = math.sqrt(2.0 / (chi + 1.0))
    mu_c = math.sqrt(delta / (2.0 + delta))
    K, E = ellip_KE(mu, mu_c)
    q = np.zeros(m_max + 1)
    q[0] = mu * K
    if m_max == 0:
        return q
    eta = math.acosh(chi) if delta > 1e-3 else math.log1p(delta + math.sqrt(delta * (2.0 + delta)))
    if eta * m_max <= 0.5:
        # forward recursion from both starting values
        q[1] = chi * mu * K - math.sqrt(2.0 * (chi + 1.0)) * E
        for n in range(2, m_max + 1):
            q[n] = (4.0 * (n - 1) * chi * q[n - 1] - (2 * n - 3) * q[n - 2]) / (2 * n - 1)
        return q
    # backward recursion on ratios rho_n = q_n / q_{n-1}
    n_start = m_max + 20 + int(40.0 / eta)
    ratio = np.zeros(m_max + 1)
    rho = 0.0
    for n in range(n_start, 1, -1):
        # rho_{n-1} = (2n-3) / (4(n-1) chi - (2n-1) rho_n)
        rho = (2 * n - 3) / (4.0 * (n - 1) * chi - (2 * n - 1) * rho)
        if n - 1 <= m_max:
            ratio[n - 1] = rho
    for n in range(1, m_max + 1):
        q[n] = q[n - 1] * ratio[n]
    return q


def dq_half(delta: float, q: np.ndarray):
    """dQ_{m-1/2}/dchi for m = 0..len(q)-2, Eq. dleg_recur:
    (2m-1)/(2(chi^2-1)) (chi Q_{m-1/2} - Q_{m-3/2}),  with Q_{-3/2} = Q_{1/2}."""
    chi = 1.0 + delta
    chi2m1 = delta * (2.0 + delta)
    m = np.arange(len(q) - 1)
    prev = np.concatenate([[q[1]], q[:-2]])
    return (2 * m - 1) / (2.0 * chi2m1) * (chi * q[:-1] - prev)
