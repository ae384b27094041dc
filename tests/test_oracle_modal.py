"""Pins for the oracle's modal Green's functions (Sec. 3.2-3.3: Eqs.
modalgreen, conv, I1, modal-normal; the inverse DFT against L_j, Sec. 3.1)."""
import math

import mpmath
import numpy as np
import pytest

from oracle.modal import lagrange_weights, modal_coeffs


def brute(r, rt, c, k, N, M=1 << 14):
    phi = 2 * np.pi * np.arange(M) / M
    rho = np.sqrt((r - rt) ** 2 + c * c + 4 * r * rt * np.sin(phi / 2) ** 2)
    G = np.exp(1j * k * rho) / (4 * np.pi * rho)
    dG = np.exp(1j * k * rho) * (1j * k * rho - 1) / (4 * np.pi * rho ** 2)
    f = lambda v: (np.fft.fft(v) * (2 * np.pi / M))[: N + 1]
    return f(G), f(dG * (r - rt * np.cos(phi)) / rho), f(-dG * c / rho)


@pytest.mark.parametrize("r,rt,c,k", [(0.5, 0.7, 0.3, 0.0), (0.5, 0.7, 0.3, 5.0),
                                      (0.3, 0.35, 0.05, 10.0), (0.05, 0.6, 0.4, 3.0),
                                      (0.45, 0.3, -0.2, 15.0)])
def test_far_ring_against_brute_force_trapezoid(r, rt, c, k):
    # the trapezoid in phi is spectrally exact for a ring away from the target
    a = modal_coeffs(r, rt, c, k, 24)
    b = brute(r, rt, c, k, 24)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) < 2e-14 * np.max(np.abs(y))


@pytest.mark.parametrize("k", [0.0, 7.0])
def test_near_ring_against_adaptive_quadrature(k):
    mpmath.mp.dps = 30
    r, rt, c = 0.4, 0.41, 0.01
    G, Gr, Gz = modal_coeffs(r, rt, c, k, 8)
    R, RT, C = mpmath.mpf(r), mpmath.mpf("0.41"), mpmath.mpf("0.01")
    rho = lambda p: mpmath.sqrt((R - RT) ** 2 + C ** 2 + 4 * R * RT * mpmath.sin(p / 2) ** 2)
    brk = [0, 0.001, 0.01, 0.05, 0.2, 1, mpmath.pi]
    for m in (0, 5):
        g = lambda p: mpmath.exp(1j * k * rho(p)) / (4 * mpmath.pi * rho(p)) * mpmath.cos(m * p)
        gr = lambda p: (mpmath.exp(1j * k * rho(p)) * (1j * k * rho(p) - 1) / (4 * mpmath.pi * rho(p) ** 3)
                        * (R - RT * mpmath.cos(p)) * mpmath.cos(m * p))
        # the source derivative along the ring axis, d/dz_y G with c = z_t - z
        gz = lambda p: (-mpmath.exp(1j * k * rho(p)) * (1j * k * rho(p) - 1) / (4 * mpmath.pi * rho(p) ** 3)
                        * C * mpmath.cos(m * p))
        ref_g = complex(2 * mpmath.quad(g, brk))
        ref_r = complex(2 * mpmath.quad(gr, brk))
        ref_z = complex(2 * mpmath.quad(gz, brk))
        assert abs(G[m] - ref_g) < 1e-13 * abs(ref_g)
        assert abs(Gr[m] - ref_r) < 1e-13 * abs(ref_r)
        assert abs(Gz[m] - ref_z) < 1e-13 * abs(ref_z)


def test_k_to_zero_limit():
    a = modal_coeffs(0.4, 0.5, 0.1, 0.0, 16)
    b = modal_coeffs(0.4, 0.5, 0.1, 1e-7, 16)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) < 1e-6 * np.max(np.abs(x))


def test_derivatives_by_finite_differences():
    r, rt, c, k, h = 0.4, 0.5, 0.1, 4.0, 1e-5
    G, Gr, Gz = modal_coeffs(r, rt, c, k, 12)
    fd_r = (modal_coeffs(r + h, rt, c, k, 12)[0] - modal_coeffs(r - h, rt, c, k, 12)[0]) / (2 * h)
    # c = z_t - z: a source shift +h in z lowers c by h
    fd_z = -(modal_coeffs(r, rt, c + h, k, 12)[0] - modal_coeffs(r, rt, c - h, k, 12)[0]) / (2 * h)
    assert np.max(np.abs(Gr - fd_r)) < 1e-8 * np.max(np.abs(Gr))
    assert np.max(np.abs(Gz - fd_z)) < 1e-8 * np.max(np.abs(Gz))


def test_lagrange_weights_exact_for_trig_polynomials():
    """W_j against a fine trapezoid of G(theta) L_j(theta), L_j as printed in Sec. 3.1."""
    N, alpha = 8, 0.37
    # G(theta) = 1 + 0.3 cos 2(theta - alpha) + 0.1 cos N(theta - alpha); phi-coefficients:
    coef = np.zeros(N + 1, complex)
    coef[0] = 2 * np.pi
    coef[2] = 0.3 * np.pi
    coef[N] = 0.1 * np.pi
    W = lagrange_weights(coef, alpha, 2 * N)
    M = 4096
    th = 2 * np.pi * np.arange(M) / M
    G = 1 + 0.3 * np.cos(2 * (th - alpha)) + 0.1 * np.cos(N * (th - alpha))
    ref = []
    for j in range(2 * N):
        tj = j * np.pi / N
        L = (1 + 2 * sum(np.cos(m * (th - tj)) for m in range(1, N)) + np.cos(N * (th - tj))) / (2 * N)
        ref.append(np.sum(G * L) * 2 * np.pi / M)
    assert np.max(np.abs(W - np.array(ref))) < 1e-14


def test_cos_theta_weights_against_trapezoid():
    """int K^r(theta - alpha) cos(theta) L_j dtheta from shifted modal coefficients
    (the area-weighted normal's cos(theta) factor) against a fine trapezoid."""
    from oracle.modal import lagrange_weights_cos_theta
    r, rt, c, k, N, al = 0.4, 0.5, 0.3, 3.0, 8, 0.7
    G, Gr, Gz = modal_coeffs(r, rt, c, k, N + 1)
    W = lagrange_weights_cos_theta(Gr, al, 2 * N)
    M = 1 << 13
    th = 2 * np.pi * np.arange(M) / M
    phi = th - al
    rho = np.sqrt(rt ** 2 + r ** 2 + c ** 2 - 2 * r * rt * np.cos(phi))
    dG = np.exp(1j * k * rho) * (1j * k * rho - 1) / (4 * np.pi * rho ** 2)
    Kr = dG * (r - rt * np.cos(phi)) / rho
    ref = []
    for j in range(2 * N):
        tj = j * np.pi / N
        L = (1 + 2 * sum(np.cos(m * (th - tj)) for m in range(1, N)) + np.cos(N * (th - tj))) / (2 * N)
        ref.append(np.sum(Kr * np.cos(th) * L) * 2 * np.pi / M)
    assert np.max(np.abs(W - np.array(ref))) < 1e-14 * np.max(np.abs(ref))


def test_sin_theta_weights_against_trapezoid():
    """int K^z(theta - alpha) sin(theta) L_j dtheta (the sin(theta) part of the
    area-weighted normal on the paper's shapes) against a fine trapezoid."""
    from oracle.modal import lagrange_weights_sin_theta
    r, rt, c, k, N, al = 0.45, 0.35, -0.25, 2.0, 8, 2.3
    G, Gr, Gz = modal_coeffs(r, rt, c, k, N + 1)
    W = lagrange_weights_sin_theta(Gz, al, 2 * N)
    M = 1 << 13
    th = 2 * np.pi * np.arange(M) / M
    phi = th - al
    rho = np.sqrt(rt ** 2 + r ** 2 + c ** 2 - 2 * r * rt * np.cos(phi))
    dG = np.exp(1j * k * rho) * (1j * k * rho - 1) / (4 * np.pi * rho ** 2)
    Kz = dG * (-c) / rho
    ref = []
    for j in range(2 * N):
        tj = j * np.pi / N
        L = (1 + 2 * sum(np.cos(m * (th - tj)) for m in range(1, N)) + np.cos(N * (th - tj))) / (2 * N)
        ref.append(np.sum(Kz * np.sin(th) * L) * 2 * np.pi / M)
    assert np.max(np.abs(W - np.array(ref))) < 1e-14 * np.max(np.abs(ref))
