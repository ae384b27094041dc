"""Near-field correction of the scattered field (Sec. 6 field evaluation;
the self blocks' product integration of Sec. 3 taken at off-surface
targets) against the oracle's layer potential of the interpolated density
(oracle/nearfield.py, an adaptive 2-D integral) and against closed forms,
through the C ABI."""
import numpy as np
import pytest

import closed_forms as cf
import scenes
from oracle.geometry import body_nodes
from oracle.nearfield import near_field

pytestmark = pytest.mark.gpu

ARC = scenes.Body(2, 12, 16, 0.5, (0.1, 0.05), (0.04,), 1.0, 0.35, tuple(scenes.rot_zy(0.7, 1.2)),
                  (0.3, -0.2, 0.1))
CONCH = scenes.conch(2, 12, 16, scale=0.5, rotation=tuple(scenes.rot_zy(0.2, 0.5)), center=(0.1, 0.2, -0.3))
TOL = 1e-10  # relative to the largest |u| of the case: both sides converged quadratures


def make(bodies, k, eta):
    import paper_2606_31380_b300 as q
    ctx = q.Context(0)
    ctx.set_bodies(bodies)
    ctx.set_wavenumber(k, eta)
    return ctx


def gpu_field(ctx, mu, pts, near=None):
    import torch
    import paper_2606_31380_b300 as q
    if near is not None:
        ctx.set_option(q.OPT_NEAR_FIELD, near)
    m = torch.from_numpy(np.ascontiguousarray(mu.reshape(mu.shape[0], -1))).cuda()
    u = torch.zeros((len(pts), m.shape[1]), dtype=torch.complex128, device="cuda")
    ctx.field(m, np.asarray(pts, float), u)
    return u.cpu().numpy()


def near_points(bn, t, spacing):
    """Points off node t and off the midpoint of nodes t, t+1, at 0.4 and 0.02
    node spacings outside and 0.1 inside."""
    pts = []
    for base, nrm in ((bn.x[t], bn.n[t]), (0.5 * (bn.x[t] + bn.x[t + 1]), bn.n[t] + bn.n[t + 1])):
        nrm = nrm / np.linalg.norm(nrm)
        for d in (0.4, 0.02, -0.1):
            pts.append(base + d * spacing * nrm)
    return np.array(pts)


def spacing_of(bn):
    x = bn.x.reshape(-1, bn.n_theta, 3)
    return max(np.max(np.linalg.norm(x - np.roll(x, 1, axis=1), axis=2)),
               np.max(np.linalg.norm(np.diff(x.reshape(bn.n_panels, bn.order, bn.n_theta, 3), axis=1), axis=3)))


@pytest.mark.parametrize("body,k", [(ARC, 3.0), (CONCH, 10.0)], ids=["arc-k3", "conch-k10"])
def test_near_points_against_oracle(body, k):
    bn = body_nodes(body)
    ctx = make([body], k, 1.0)
    rng = np.random.default_rng(8)
    mu = rng.normal(size=(bn.count, 2)) + 1j * rng.normal(size=(bn.count, 2))
    pts = near_points(bn, 133, spacing_of(bn))
    got = gpu_field(ctx, mu, pts)
    assert ctx.field_near_pairs() == len(pts)
    ref = np.array([near_field(bn, mu, x, k, 1.0) for x in pts])
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) < TOL * scale, np.max(np.abs(got - ref), axis=1) / scale
    # the smooth rule alone is far off so close to the surface
    plain = gpu_field(ctx, mu, pts, near=0)
    assert ctx.field_near_pairs() == 0
    assert np.max(np.abs(plain - ref)) > 1e-3 * scale


def test_gauss_lemma_near_the_surface():
    """k -> 0 (1e-6), eta = 0, mu = 1: the double layer is -1 inside, 0 outside."""
    bn = body_nodes(CONCH)
    ctx = make([CONCH], 1e-6, 0.0)
    h = spacing_of(bn)
    pts, want = [], []
    for t in (40, 200, 350):
        for d, w in ((0.3, 0.0), (0.01, 0.0), (-0.01, -1.0), (-0.3, -1.0)):
            pts.append(bn.x[t] + d * h * bn.n[t])
            want.append(w)
    got = gpu_field(ctx, np.ones(bn.count, complex), np.array(pts))[:, 0]
    assert np.max(np.abs(got - np.array(want))) < 1e-9


def test_sphere_harmonics_near_the_surface():
    """Degree-2 harmonic density on a sphere: D - i eta S at radii 1 +- 0.01
    node spacings against the addition-theorem closed form."""
    a, k, eta = 0.8, 3.0, 1.0
    body = scenes.sphere(a, 2, 16, 32)
    bn = body_nodes(body)
    ctx = make([body], k, eta)
    X = bn.x
    mu = X[:, 0] * X[:, 2] / a ** 2 + 0j
    h = spacing_of(bn)
    rng = np.random.default_rng(6)
    pts, want = [], []
    for rad in (a + 0.01 * h, a - 0.01 * h, a + 0.5 * h):
        for _ in range(2):
            v = rng.normal(size=3)
            xh = v / np.linalg.norm(v)
            s_n, d_n = cf.sphere_layer_potentials(a, k, 2, rad)
            pts.append(rad * xh)
            want.append((d_n - 1j * eta * s_n) * xh[0] * xh[2])
    got = gpu_field(ctx, mu, np.array(pts))[:, 0]
    assert np.max(np.abs(got - np.array(want))) < 1e-8 * np.max(np.abs(want))


def test_point_source_field_near_two_bodies():
    """The paper's check (Eq. artificial point source solution): sources inside
    two bodies, the solved density's field at points a fraction of a node
    spacing off either surface against the exact field; and a point near both
    bodies at once (two corrected pairs)."""
    import torch
    import paper_2606_31380_b300 as q
    k = 2.0
    b1 = scenes.Body(2, 16, 32, 0.5, (0.06, 0.03), (0.04,), 1.0, 0.35, tuple(scenes.rot_zy(0.3, 1.1)), (0, 0, 0))
    b2 = scenes.Body(2, 16, 32, 0.5, (0.06, 0.03), (0.04,), 1.0, 0.35, tuple(scenes.rot_zy(2.0, 0.4)),
                     (2.2, 0.5, -0.3))
    ctx = make([b1, b2], k, 1.0)
    nodes = [body_nodes(b1), body_nodes(b2)]
    X = np.concatenate([n.x for n in nodes])
    z = np.array([b1.center, b2.center], float)
    b = torch.from_numpy(cf.point_source_field(X, z, k)[:, None].copy()).cuda()
    ctx.assemble()
    mu = torch.zeros_like(b)
    ctx.solve(b, mu, q.PREC_FP64, tol=1e-13)
    h = spacing_of(nodes[0])
    pts = [nodes[0].x[300] + 0.05 * h * nodes[0].n[300], nodes[1].x[700] + 0.3 * h * nodes[1].n[700],
           nodes[0].x[1000] + 2.0 * h * nodes[0].n[1000]]
    # the point of each body nearest to the other, and a point between them
    d = np.linalg.norm(nodes[0].x[:, None, :] - nodes[1].x[None, :, :], axis=2)
    i, j = np.unravel_index(np.argmin(d), d.shape)
    pts.append(0.5 * (nodes[0].x[i] + nodes[1].x[j]))
    pts = np.array(pts)
    ex = cf.point_source_field(pts, z, k)
    m = mu.cpu().numpy()
    got = gpu_field(ctx, m, pts, near=8)[:, 0]       # 8 spacings: the midpoint is near both bodies
    pairs = ctx.field_near_pairs()
    plain = gpu_field(ctx, m, pts, near=0)[:, 0]
    err = np.abs(got - ex) / np.max(np.abs(ex))
    err_plain = np.abs(plain - ex) / np.max(np.abs(ex))
    assert pairs >= 4
    assert np.max(err) < 1e-6, err
    assert np.max(err_plain) > 100 * np.max(err), (err, err_plain)
