"""GPU parity on the paper's own shapes (Eqs. quasiwave and geometries:
horizontal rings with a moving centre) and on panels refined dyadically
toward the poles (Sec. 6.1), against the FP64 oracle and closed forms."""
import numpy as np
import pytest

import closed_forms as cf
import scenes
from gpu_util import make_ctx, rel_err
from oracle.geometry import body_nodes
from oracle.selfblock import self_block_rows_parallel

pytestmark = pytest.mark.gpu

BLOCK_TOL = 1e-12


def gpu_block(scene, body=0):
    import torch
    ctx = make_ctx(scene)
    ctx.assemble()
    off = ctx.body_offsets()
    n = int(off[body + 1] - off[body])
    A = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    ctx.copy_selfblock(body, A)
    torch.cuda.synchronize()
    return ctx, A.cpu().numpy()


def row_err(A, ref):
    return max(np.max(np.abs(a - r)) / np.max(np.abs(r)) for a, r in zip(A, ref))


def _placed(b, rot, center):
    b.rotation = scenes.rot_zy(*rot)
    b.center = center
    return b


def test_nodes_match_oracle_paper_shapes_and_dyadic_panels():
    bodies = [_placed(scenes.conch(2, 8, 16, scale=0.4), (0.3, 1.2), (0.0, 0.0, 0.0)),
              _placed(scenes.spiral(3, 6, 12, scale=0.3), (2.0, 0.4), (3.0, 0.5, -0.4)),
              _placed(scenes.quasi_ellipsoid(6, 8, 20, scale=0.2, breaks=scenes.dyadic_breaks(4, 1)),
                      (1.0, 2.5), (-2.5, 1.0, 1.0)),
              scenes.Body(6, 8, 16, 0.5, (0.1,), (0.05,), 1.0, 0.3, panel_breaks=scenes.dyadic_breaks(2, 2),
                          center=(0.5, 3.0, 0.0))]
    sc = scenes.Scene("shapes", bodies, 2.0, 1.0, scenes.paper_direction())
    ctx = make_ctx(sc)
    x, n, w = ctx.get_nodes()
    nodes = [body_nodes(b) for b in bodies]
    assert rel_err(x, np.concatenate([b.x for b in nodes])) < 1e-14
    assert rel_err(n, np.concatenate([b.n for b in nodes])) < 1e-14
    assert rel_err(w, np.concatenate([b.w for b in nodes])) < 1e-13


@pytest.mark.parametrize("make,k,eta", [(scenes.conch, 3.0, 1.0), (scenes.spiral, 5.0, 1.0),
                                        (scenes.quasi_wave, 2.0, 0.0)])
def test_paper_shape_rows_match_oracle(make, k, eta):
    body = _placed(make(2, 12, 24, scale=0.5), (0.7, 2.1), (1.0, -2.0, 0.5))
    _, A = gpu_block(scenes.Scene("shape", [body], k, eta, scenes.paper_direction()))
    bn = body_nodes(body)
    n, nth, per = bn.count, 24, 12 * 24
    rows = sorted({0, 5, per - 1, per + 7, n // 2 + 9, n - 1, 3 * nth + 13})
    ref = self_block_rows_parallel(bn, rows, k, eta, tol=1e-13)
    assert row_err(A[rows], ref) < BLOCK_TOL


def test_dyadic_panel_rows_match_oracle():
    """Six panels (two uniform, each end panel bisected twice): the self and
    neighbour rules on unequal panels and the plain rule beyond them."""
    br = scenes.dyadic_breaks(2, 2)
    body = scenes.Body(len(br) - 1, 12, 24, 0.5, (0.1,), (0.05,), 1.0, 0.3, panel_breaks=br)
    _, A = gpu_block(scenes.Scene("dyadic", [body], 4.0, 1.0, scenes.paper_direction()))
    bn = body_nodes(body)
    per = 12 * 24
    rows = [3, per + 20, 2 * per + per * 3 // 4 + 4, 3 * per + 1, 5 * per + 100, 6 * per - 1]
    ref = self_block_rows_parallel(bn, rows, 4.0, 1.0, tol=1e-13)
    assert row_err(A[rows], ref) < BLOCK_TOL


@pytest.mark.parametrize("make", [scenes.conch, scenes.spiral, scenes.quasi_ellipsoid])
def test_gauss_identity_paper_shapes(make):
    """k -> 0, eta = 0: (1/2 I + D) 1 = 0 on every row (Gauss's lemma) where all
    panels are near (two panels); the sin(theta) part of the normal enters."""
    body = make(2, 12, 24, scale=0.5)
    _, A = gpu_block(scenes.Scene("g", [body], 1e-9, 0.0, scenes.paper_direction()))
    assert np.max(np.abs(A.sum(axis=1))) < 1e-11


def test_point_sources_paper_shapes_converge():
    """Two quasi-ellipsoids and a conch with interior point sources: the field of
    the GPU density converges to the exact one as the panels are refined
    (uniform, then dyadically toward the poles)."""
    import torch
    import paper_2606_31380_b300 as q
    k = 3.0
    errs = []
    pts = np.array([[5.0, 1.0, 2.0], [-3.0, 2.5, 1.0], [1.0, -4.0, 0.5], [0.8, 3.0, -3.0]])
    for npan, order, nth, br in [(4, 8, 16, ()), (6, 12, 24, ()), (10, 16, 32, scenes.dyadic_breaks(6, 2))]:
        kw = dict(breaks=br) if br else {}
        bodies = [_placed(scenes.quasi_ellipsoid(npan, order, nth, scale=0.25, **kw), (0.3, 1.1), (0.0, 0.0, 0.0)),
                  _placed(scenes.quasi_ellipsoid(npan, order, nth, scale=0.25, **kw), (2.0, 0.4), (3.0, 0.4, -0.3)),
                  _placed(scenes.conch(npan, order, nth, scale=0.4, **kw), (1.0, 2.0), (0.5, 3.0, 0.6))]
        sc = scenes.Scene("pts", bodies, k, 1.0, scenes.paper_direction())
        ctx = make_ctx(sc)
        ctx.assemble()
        x, _, _ = ctx.get_nodes()
        z = np.array([b.center for b in bodies], float)
        rhs = torch.from_numpy(cf.point_source_field(x, z, k)[:, None].copy()).cuda()
        mu = torch.zeros_like(rhs)
        ctx.solve(rhs, mu, q.PREC_FP64, tol=1e-13)
        u = torch.zeros((len(pts), 1), dtype=torch.complex128, device="cuda")
        ctx.field(mu, pts, u)
        ex = cf.point_source_field(pts, z, k)
        errs.append(np.max(np.abs(u.cpu().numpy()[:, 0] - ex)) / np.max(np.abs(ex)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6
