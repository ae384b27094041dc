"""Host logic of the near-field correction (Sec. 6 field evaluation): the
nearest surface point found by Gauss-Newton from the nearest node, checked
with the oracle's independent surface map (oracle/geometry.py)."""
import numpy as np
import pytest

import scenes
from oracle.geometry import body_nodes

ARC = scenes.Body(2, 12, 16, 0.5, (0.1, 0.05), (0.04,), 1.0, 0.35, tuple(scenes.rot_zy(0.7, 1.2)),
                  (0.3, -0.2, 0.1))
CONCH = scenes.conch(2, 12, 16, scale=0.5, rotation=tuple(scenes.rot_zy(0.2, 0.5)), center=(0.1, 0.2, -0.3))


def surface_world(bn, s, th):
    g = bn.geom
    return g.to_world(g.local_points(np.array([s]), np.array([th]))[0])


@pytest.mark.parametrize("body", [ARC, CONCH], ids=["arc", "conch"])
def test_points_off_nodes_project_back_to_the_node(body):
    """x = y_node + d n_node with d well below the radii of curvature: the nearest
    point is the node itself, at distance d."""
    import paper_2606_31380_b300 as q
    bn = body_nodes(body)
    nth = bn.n_theta
    for t in (5, 77, 200, 300):
        for d in (1e-3, -2e-3, 0.02):
            x = bn.x[t] + d * bn.n[t]
            s, th, dist = q.nearest_surface_point(body, x)
            assert abs(dist - abs(d)) < 1e-12
            # the point itself (theta is ill-conditioned near a pole, the position is not;
            # |x - y|^2 is flat to second order there, so ~sqrt(eps) d is the resolution)
            assert np.linalg.norm(surface_world(bn, s, th) - bn.x[t]) < 1e-9
            assert abs(s - bn.s[t // nth]) < 1e-8


@pytest.mark.parametrize("body", [ARC, CONCH], ids=["arc", "conch"])
def test_random_points_are_orthogonal_projections(body):
    """Random points within a node spacing or two of the surface: the returned
    point lies on the surface at the returned distance, the offset is normal to
    the surface (orthogonal to both tangents), and no node is closer."""
    import paper_2606_31380_b300 as q
    bn = body_nodes(body)
    rng = np.random.default_rng(9)
    for _ in range(12):
        t = int(rng.integers(0, bn.count - 1))
        base = 0.5 * (bn.x[t] + bn.x[t + 1]) if (t + 1) % bn.n_theta else bn.x[t]
        x = base + rng.normal(size=3) * 0.05
        s, th, dist = q.nearest_surface_point(body, x)
        y = surface_world(bn, s, th)
        assert abs(np.linalg.norm(x - y) - dist) < 1e-12
        h = 1e-6
        ts = (surface_world(bn, s + h, th) - surface_world(bn, s - h, th)) / (2 * h)
        tt = (surface_world(bn, s, th + h) - surface_world(bn, s, th - h)) / (2 * h)
        for tv in (ts, tt):
            assert abs(np.dot(x - y, tv)) < 1e-7 * max(dist, 1e-3) * np.linalg.norm(tv)
        assert dist <= np.min(np.linalg.norm(bn.x - x, axis=1)) + 1e-12
