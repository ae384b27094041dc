"""Pins for the oracle's special functions (Sec. 3.3: Eqs. modal0, leg_recur,
dleg_recur and the elliptic starting values)."""
import math

import mpmath
import numpy as np
import pytest
from scipy import special as sp

from oracle.special import dq_half, ellip_KE, q_half


def test_elliptic_special_values():
    K, E = ellip_KE(0.0, 1.0)
    assert abs(K - math.pi / 2) < 1e-15 and abs(E - math.pi / 2) < 1e-15
    K, E = ellip_KE(1.0 - 1e-300, 1e-300)
    assert abs(E - 1.0) < 1e-12 and K > 300


@pytest.mark.parametrize("mu", [0.05, 0.3, 0.7, 0.95, 0.9999])
def test_elliptic_legendre_relation_and_library(mu):
    mc = math.sqrt(1 - mu * mu)
    K, E = ellip_KE(mu, mc)
    Kp, Ep = ellip_KE(mc, mu)
    assert abs(E * Kp + Ep * K - K * Kp - math.pi / 2) < 1e-14
    assert abs(K - sp.ellipk(mu * mu)) < 1e-14 * K
    assert abs(E - sp.ellipe(mu * mu)) < 1e-14


@pytest.mark.parametrize("delta", [1e-9, 1e-5, 2e-3, 0.05, 0.7, 5.0, 300.0])
def test_q_against_mpmath_legendre_q(delta):
    mpmath.mp.dps = 40
    q = q_half(delta, 60)
    for m in (0, 1, 2, 7, 30, 60):
        ref = float(mpmath.re(mpmath.legenq(m - 0.5, 0, 1 + mpmath.mpf(delta), type=3)))
        assert abs(q[m] - ref) <= 2e-13 * abs(q[0])


@pytest.mark.parametrize("delta", [0.02, 1.5])
def test_q_against_defining_integral(delta):
    chi = 1 + delta
    q = q_half(delta, 6)
    for m in (0, 3, 6):
        ref = mpmath.quad(lambda p: mpmath.cos(m * p) / mpmath.sqrt(2 * (chi - mpmath.cos(p))), [0, mpmath.pi])
        assert abs(q[m] - float(ref)) < 1e-13 * q[0]


def test_forward_and_backward_recursions_agree():
    # eta*m_max straddles the 0.5 switch: compare the two regimes on one chi
    delta = 2e-4
    fw = q_half(delta, 20)           # eta*20 ~ 0.4 -> forward
    bw = q_half(delta, 200)[:21]     # eta*200 > 0.5 -> Miller
    assert np.max(np.abs(fw - bw)) < 1e-13 * fw[0]


@pytest.mark.parametrize("delta", [1e-3, 0.1, 3.0])
def test_recursion_residual_and_derivative(delta):
    chi = 1 + delta
    q = q_half(delta, 40)
    n = np.arange(2, 41)
    res = (2 * n - 1) * q[n] - 4 * (n - 1) * chi * q[n - 1] + (2 * n - 3) * q[n - 2]
    assert np.max(np.abs(res)) < 1e-13 * q[0] * 40
    dq = dq_half(delta, q)
    h = 1e-6 * delta
    fd = (q_half(delta + h, 40) - q_half(delta - h, 40)) / (2 * h)
    assert np.max(np.abs(dq[:20] - fd[:20])) < 1e-6 * np.max(np.abs(dq[:20]))
