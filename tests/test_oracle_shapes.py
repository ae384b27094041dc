"""Pins for the paper's own shapes (Eqs. quasiwave and geometries: horizontal
rings with a moving centre), for non-uniform panels (dyadic refinement toward
the poles, Sec. 6.1) and for the shared geometry formulas of both families."""
import math

import mpmath
import numpy as np
import pytest

import scenes
from oracle.geometry import body_nodes, geometry
from oracle.selfblock import self_block_rows

# volumes by Cavalieri's principle: horizontal slices are discs of radius r(t)
# at height z(t), whatever their centres, so V = int pi r^2 z' dt
PAPER_SHAPES = [
    (scenes.quasi_wave, math.pi * 2.0 * 4.0 / 3.0),            # r = cos t, z = 2 sin t
    (scenes.quasi_ellipsoid, math.pi * 4.0 * 3.0 * 4.0 / 3.0),  # r = 2 cos t, z = 3 sin t
    (scenes.spiral, math.pi * 2.25 * 2.0 * 4.0 / 3.0),          # r = 1.5 cos t, z = 2 sin t
    (scenes.conch, math.pi * 1.5 * 4.0 / 3.0),                  # r = cos t, z = 1.5 sin t
]


@pytest.mark.parametrize("make,vol", PAPER_SHAPES)
def test_divergence_theorem_volume(make, vol):
    """(1/3) int y.n dS = V on the Nystrom nodes, uniform and dyadically refined panels."""
    for breaks_args in [None, (6, 3)]:
        if breaks_args is None:
            b = make(n_panels=8, order=16, n_theta=48)
        else:
            br = scenes.dyadic_breaks(*breaks_args)
            b = make(n_panels=len(br) - 1, order=16, n_theta=48, breaks=br)
        b.rotation = scenes.rot_zy(0.4, 1.3)
        b.center = (1.0, -2.0, 0.5)
        bn = body_nodes(b)
        v = np.sum(bn.w * np.einsum("ij,ij->i", bn.x - np.asarray(b.center), bn.n)) / 3.0
        assert abs(v - vol) < 1e-11 * vol


@pytest.mark.parametrize("body", [
    scenes.conch(), scenes.spiral(),
    scenes.Body(2, 8, 16, 0.5, (0.1, -0.05), (0.07,), 1.0, 0.4)])
def test_area_normal_is_cross_product_of_tangents(body):
    """|J| n = d_theta y x d_s y, the tangents by central differences of the
    surface points, at several (s, theta); the five coefficients of
    ``area_normal`` reproduce n_r and n_3 at every theta."""
    g = geometry(body)
    eps = 1e-5
    for s in [-1.3, -0.2, 0.7, 1.45]:
        a0, a1, b0, b1, b2 = g.area_normal(s)
        for th in [0.0, 1.1, 2.9, 4.4]:
            P = lambda ss, tt: g.local_points(np.array([ss]), np.array([tt]))[0]
            ds = (P(s + eps, th) - P(s - eps, th)) / (2 * eps)
            dt = (P(s, th + eps) - P(s, th - eps)) / (2 * eps)
            cr = np.cross(dt, ds)
            ring = g.ring(np.array([s]))
            er = math.cos(th) * ring["e1"][0] + math.sin(th) * ring["e2"][0]
            nr = a0 + a1 * math.cos(th)
            n3 = b0 + b1 * math.cos(th) + b2 * math.sin(th)
            assert np.linalg.norm(nr * er + n3 * ring["e3"][0] - cr) < 1e-8 * np.linalg.norm(cr)
            un_r, un_3, jac = g.normal_parts(np.array([s]), np.array([th]))
            assert abs(jac[0] * un_r[0] - nr) < 1e-13 and abs(jac[0] * un_3[0] - n3) < 1e-13


def _ring_exact(body, s_t, th_t, h):
    """r, r - r~, r~, c of the ring at s_t + h seen from (s_t, th_t), in 50-digit
    arithmetic straight from the parametrisation (no difference formulas)."""
    mpmath.mp.dps = 50
    f = lambda part, s: sum(mpmath.mpf(A) * mpmath.cos(om * s) + mpmath.mpf(B) * mpmath.sin(om * s)
                            for (om, A, B) in part)
    st, s = mpmath.mpf(s_t), mpmath.mpf(s_t) + mpmath.mpf(h)
    xc, yc, z, r = body.series
    rt0 = f(r, st)
    xt = f(xc, st) + rt0 * mpmath.cos(th_t)
    yt = f(yc, st) + rt0 * mpmath.sin(th_t)
    a, b, c = xt - f(xc, s), yt - f(yc, s), f(z, st) - f(z, s)
    rr = f(r, s)
    rtil = mpmath.sqrt(a * a + b * b)
    return float(rr), float(rr - rtil), float(rtil), float(c)


@pytest.mark.parametrize("make", [scenes.conch, scenes.spiral, scenes.quasi_wave])
def test_self_ring_difference_formulas_keep_relative_precision(make):
    body = make()
    g = geometry(body)
    for s_t, th in [(-0.9, 0.3), (0.35, 2.2), (1.2, 5.0)]:
        for h in [0.4, -1e-3, 1e-6, -1e-9]:
            r, dr, rt, c, _ = g.self_ring(s_t, th, h)
            er, edr, ert, ec = _ring_exact(body, s_t, th, h)
            assert abs(r - er) < 1e-14 * abs(er) and abs(rt - ert) < 1e-14 * abs(ert)
            assert abs(dr - edr) < 1e-12 * abs(edr) + 1e-300
            assert abs(c - ec) < 1e-12 * abs(ec)


@pytest.mark.parametrize("make,disc", [(scenes.conch, (2, 8, 16)), (scenes.spiral, (2, 8, 16))])
def test_gauss_identity_on_paper_shapes(make, disc):
    """k = 0, eta = 0: (1/2 I + D) 1 = 0 row by row (Gauss's lemma); every
    term of the area-weighted normal, including the sin(theta) one, enters."""
    bn = body_nodes(make(*disc, scale=0.5))
    rows = [0, bn.count // 2 + 5, bn.count - 3, 77]
    A = self_block_rows(bn, rows, 0.0, 0.0, tol=1e-13)
    assert np.max(np.abs(A.sum(axis=1))) < 1e-12


def test_gauss_identity_with_dyadic_panels():
    """The same on a curved arc-axis body with panels refined toward the poles:
    the near-panel rules follow non-uniform panel widths.  Panels two or more
    steps away take the plain rule (Eq. sx), whose error is part of the
    discretisation, so the resolution is chosen where it is below 1e-12
    (at 8 x 16 nodes per panel it is ~5e-10 here)."""
    br = scenes.dyadic_breaks(2, 2)
    b = scenes.Body(len(br) - 1, 12, 24, 0.5, (0.1,), (0.05,), 1.0, 0.3, panel_breaks=br)
    bn = body_nodes(b)
    per = 12 * 24
    rows = [per + 20, 2 * per + per * 3 // 4 + 4]
    A = self_block_rows(bn, rows, 0.0, 0.0, tol=1e-13)
    assert np.max(np.abs(A.sum(axis=1))) < 2e-12


def test_dyadic_breaks():
    br = np.array(scenes.dyadic_breaks(12, 5))
    assert len(br) == 12 + 2 * 5 + 1 and np.all(np.diff(br) > 0)
    w = np.diff(br)
    assert np.allclose(w[:6], np.pi / 12 * np.array([1 / 32, 1 / 32, 1 / 16, 1 / 8, 1 / 4, 1 / 2]))
    assert np.allclose(w[::-1][:6], w[:6])
