"""Pins for the oracle's layer potential at off-surface points
(oracle/nearfield.py; Sec. 3.1 interpolants, Sec. 6 field evaluation)."""
import numpy as np
import pytest

import closed_forms as cf
import scenes
from oracle import operator as op
from oracle.geometry import body_nodes
from oracle.nearfield import near_field

ARC = scenes.Body(2, 12, 16, 0.5, (0.1, 0.05), (0.04,), 1.0, 0.35, tuple(scenes.rot_zy(0.7, 1.2)),
                  (0.3, -0.2, 0.1))
CONCH = scenes.conch(2, 12, 16, scale=0.5, rotation=tuple(scenes.rot_zy(0.2, 0.5)), center=(0.1, 0.2, -0.3))


@pytest.mark.parametrize("body", [ARC, CONCH], ids=["arc", "conch"])
def test_gauss_lemma_near_the_surface(body):
    """k = 0, eta = 0, mu = 1: the double layer is -1 inside and 0 outside,
    exactly, for the interpolated density (the interpolant of 1 is 1), however
    close the point is to the surface."""
    bn = body_nodes(body)
    mu = np.ones(bn.count)
    for t in (100,):
        for d in (0.02, 0.002):
            for side, want in ((1.0, 0.0), (-1.0, -1.0)):
                x = bn.x[t] + side * d * bn.n[t]
                u = near_field(bn, mu, x, 0.0, 0.0)
                assert abs(u - want) < 1e-10, (t, d, side, u)


def test_sphere_harmonic_potentials_off_the_surface():
    """Degree-1 and degree-2 harmonics on a sphere: D - i eta S at radii 0.97a
    and 1.03a against the addition-theorem closed forms (to the interpolation
    error of the density in s)."""
    a, k, eta = 0.8, 3.0, 1.0
    bn = body_nodes(scenes.sphere(a, 2, 16, 32))
    X = bn.x
    dens = {1: X[:, 2] / a, 2: X[:, 0] * X[:, 2] / a ** 2}
    rng = np.random.default_rng(4)
    for n, mu in dens.items():
        for rad in (0.97 * a, 1.03 * a):
            v = rng.normal(size=3)
            xh = v / np.linalg.norm(v)
            x = rad * xh
            Y = xh[2] if n == 1 else xh[0] * xh[2]
            s_n, d_n = cf.sphere_layer_potentials(a, k, n, rad)
            want = (d_n - 1j * eta * s_n) * Y
            u = near_field(bn, mu, x, k, eta)
            assert abs(u - want) < 1e-9 * max(1.0, abs(want)), (n, rad, u, want)


def test_far_points_agree_with_the_smooth_rule():
    """Far from the body the plain Gauss-Legendre x trapezoidal sum of a smooth
    density converges to the same integral (2 x 16 x 32 nodes, k = 2)."""
    body = scenes.Body(2, 16, 32, 0.5, (0.1, 0.05), (0.04,), 1.0, 0.35, tuple(scenes.rot_zy(0.7, 1.2)),
                       (0.3, -0.2, 0.1))
    bn = body_nodes(body)
    X = bn.x
    mu = np.stack([np.cos(X[:, 0]) + 1j * np.sin(0.5 * X[:, 2]), np.exp(0.3j * X[:, 1])], axis=1)
    for x in (np.array([3.0, 0.5, -0.4]), np.array([-1.0, 2.8, 1.5])):
        ref = np.array([op.field([bn], mu[:, r], x[None, :], 2.0, 1.0)[0] for r in range(2)])
        u = near_field(bn, mu, x, 2.0, 1.0)
        assert np.max(np.abs(u - ref)) < 1e-10 * np.max(np.abs(ref))


def test_planted_slip_is_caught():
    """A sign slip in the area-weighted normal (inward normals) breaks Gauss's lemma."""
    bn = body_nodes(ARC)
    g = bn.geom
    orig = g.local_normals
    try:
        g.local_normals = lambda s, th: -orig(s, th)
        x = bn.x[100] - 0.01 * bn.n[100]       # inside: -1 with outward normals, +1 with inward
        assert abs(near_field(bn, np.ones(bn.count), x, 0.0, 0.0) + 1.0) > 0.5
    finally:
        del g.local_normals
