"""The library's host-side Nystrom nodes (Eq. para_quasi, Sec. 3.1, Eq. sx) equal
the oracle's for both shape families and for dyadically refined panels (no
device: qams_body_nodes)."""
import numpy as np
import pytest

import scenes
from oracle.geometry import body_nodes


def _bodies():
    return [
        scenes.Body(2, 16, 32, 0.5, (0.06, 0.03), (0.04,), 1.0, 0.35, scenes.rot_zy(0.7, 2.1), (1.0, -2.0, 0.5)),
        scenes.Body(6, 8, 16, 0.5, (0.1,), (0.05,), 1.0, 0.3, panel_breaks=scenes.dyadic_breaks(2, 2)),
        scenes.conch(2, 8, 16, scale=0.4, rotation=scenes.rot_zy(0.3, 1.2), center=(4.0, 0.0, 1.0)),
        scenes.spiral(3, 6, 12, scale=0.3),
        scenes.quasi_ellipsoid(10, 16, 40, scale=0.25, breaks=scenes.dyadic_breaks(6, 2)),
        scenes.quasi_wave(8, 16, 40),
        scenes.sphere(0.5, 2, 12, 24),
    ]


@pytest.mark.parametrize("body", _bodies())
def test_host_nodes_match_oracle(body):
    import paper_2606_31380_b300 as q
    x, n, w = q.body_nodes(body)
    ref = body_nodes(body)
    scale = np.max(np.abs(ref.x))
    assert np.max(np.abs(x - ref.x)) < 1e-14 * scale
    assert np.max(np.abs(n - ref.n)) < 1e-14
    assert np.max(np.abs(w - ref.w)) < 1e-13 * np.max(ref.w)


def test_invalid_descriptor_refused():
    import paper_2606_31380_b300 as q
    bad = scenes.Body(2, 8, 16, panel_breaks=(-1.5, 0.0, np.pi / 2))
    with pytest.raises(q.QamsError):
        q.body_nodes(bad)
