"""GPU self-block assembly (Sec. 3.1-3.4) and full operator apply (Eq.
linearsys) against the FP64 oracle and closed forms."""
import numpy as np
import pytest
from scipy import special as sp

import closed_forms as cf
import scenes
from gpu_util import make_ctx, rel_err
from oracle import operator as op
from oracle.geometry import body_nodes
from oracle.selfblock import self_block, self_block_rows_parallel

pytestmark = pytest.mark.gpu

BLOCK_TOL = 1e-12   # self-block rows, relative to the row's largest entry
CURVED = dict(base_radius=0.5, mode_cos=(0.06, 0.03), mode_sin=(0.04,), axis_length=1.0, curvature=0.35)


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


def test_sphere_block_matches_oracle_and_eigenvalues():
    a, k = 0.5, 2.0
    body = scenes.sphere(a, 2, 12, 24)
    sc = scenes.Scene("sphere", [body], k, 1.0, scenes.paper_direction())
    _, A = gpu_block(sc)
    bn = body_nodes(body)
    ref = self_block(bn, k, 1.0, tol=1e-13)
    assert row_err(A, ref) < BLOCK_TOL
    S, T = np.meshgrid(bn.s, bn.theta, indexing="ij")
    S, T = S.reshape(-1), T.reshape(-1)
    for n, m, tol in [(0, 0, 1e-13), (1, 0, 1e-10), (2, 1, 1e-9)]:
        Y = sp.lpmv(m, n, np.sin(S)) * np.exp(1j * m * T)
        assert np.linalg.norm(A @ Y - cf.sphere_eigen(a, k, n, 1.0) * Y) / np.linalg.norm(Y) < tol


@pytest.mark.parametrize("k,eta,disc", [(5.0, 1.0, (2, 16, 32)), (15.0, 1.0, (2, 12, 24)), (3.0, 0.0, (1, 16, 32)),
                                        (1e-9, 0.0, (2, 8, 16)), (3.0, 1.0, (1, 8, 16))])
def test_curved_body_rows_match_oracle(k, eta, disc):
    body = scenes.Body(*disc, **CURVED, rotation=scenes.rot_zy(0.7, 2.1), center=(1.0, -2.0, 0.5))
    sc = scenes.Scene("curved", [body], k, eta, scenes.paper_direction())
    _, A = gpu_block(sc)
    bn = body_nodes(body)
    nth, per = disc[2], disc[1] * disc[2]
    n = bn.count
    rows = sorted({0, 3, per - 1, min(n - 1, per + 5), n // 2 + nth // 3, n - 1, 7 * nth + 11})
    ref = self_block_rows_parallel(bn, rows, k, eta, tol=1e-13)
    assert row_err(A[rows], ref) < BLOCK_TOL


def test_gauss_identity_on_gpu_block():
    """k -> 0, eta = 0: (1/2 I + D) 1 = 0 (Gauss's lemma) holds to quadrature
    accuracy on every row, for several discretisations."""
    for disc in [(1, 8, 16), (2, 12, 24), (2, 16, 32)]:
        body = scenes.Body(*disc, **CURVED)
        _, A = gpu_block(scenes.Scene("g", [body], 1e-9, 0.0, scenes.paper_direction()))
        assert np.max(np.abs(A.sum(axis=1))) < 1e-11


def test_apply_matches_oracle_congruent_bodies():
    """Three congruent bodies of revolution (the oracle's circulant shortcut
    gives their common self block), R = 3, FP64 and FP32 paths."""
    import torch
    import paper_2606_31380_b300 as q
    shape = dict(base_radius=0.5, mode_cos=(0.1, 0.02), mode_sin=(0.05,), axis_length=1.0, curvature=0.0)
    bodies = [scenes.Body(2, 8, 16, **shape, rotation=scenes.rot_zy(0.3 * i, 1.0 + i), center=(2.6 * i, 0.4 * i, -0.5 * i))
              for i in range(3)]
    sc = scenes.Scene("congruent", bodies, 4.0, 1.0, scenes.paper_direction())
    ctx = make_ctx(sc)
    ctx.assemble()
    nodes = [body_nodes(b) for b in bodies]
    A1 = self_block(nodes[0], sc.k, sc.eta, tol=1e-13)
    x = scenes.rhs_seeded(ctx.N, 3, 4)
    ref = op.apply(nodes, [A1] * 3, x, sc.k, sc.eta)
    for prec, dt, tol in [(q.PREC_FP64, torch.complex128, 1e-12), (q.PREC_FP32, torch.complex64, 5e-6)]:
        xd = torch.from_numpy(x).to(dt).cuda()
        y = torch.empty_like(xd)
        ctx.apply(xd, y, prec)
        torch.cuda.synchronize()
        assert rel_err(y.cpu().numpy(), ref) < tol


def test_apply_full_size_sampled_rows():
    """16 quasi-axisymmetric bodies, 32 x 64 nodes each, k = 5: all rows on the
    GPU, sampled rows against oracle self-block rows plus oracle pair sums."""
    import torch
    import paper_2606_31380_b300 as q
    sc = scenes.config(1)
    ctx = make_ctx(sc)
    ctx.assemble()
    nodes = [body_nodes(b) for b in sc.bodies]
    off = ctx.body_offsets()
    x = scenes.rhs_seeded(ctx.N, 1, 9)
    rows = [5, 2048 * 3 + 1000, 2048 * 9 + 2047, 2048 * 15 + 64]
    ref = np.zeros((len(rows), 1), complex)
    w = np.concatenate([b.w for b in nodes])
    ref += op.pair_sum(nodes, w[:, None] * x, sc.k, sc.eta, targets=rows)
    for i, g in enumerate(rows):
        b = int(np.searchsorted(off, g, side="right") - 1)
        t = g - off[b]
        Arow = self_block_rows_parallel(nodes[b], [t], sc.k, sc.eta, tol=1e-13, workers=1)[0]
        ref[i] += Arow @ x[off[b]:off[b + 1]]
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    ctx.apply(xd, y, q.PREC_FP64)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy()[rows], ref) < 1e-12
    # the refinement residual's operator: float-float pair sum, FP64 blocks
    ctx.apply(xd, y, q.PREC_FF)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy()[rows], ref) < 1e-12


def test_limits_and_single_body():
    """A body beyond the kernel's limits (n_theta/2 > 32) is refused at assembly
    with QAMS_EINVAL; a single body has no inter-body part: its pair sum is zero
    and the operator apply equals its self-block product exactly."""
    import torch
    import paper_2606_31380_b300 as q
    big = scenes.Body(1, 8, 80, 0.5, (0.1,), (), 1.0, 0.2)
    ctx = make_ctx(scenes.Scene("big", [big], 2.0, 1.0, scenes.paper_direction()))
    with pytest.raises(q.QamsError) as err:
        ctx.assemble()
    assert err.value.code == -1
    one = scenes.Body(1, 8, 16, 0.5, (0.1,), (), 1.0, 0.2)
    ctx = make_ctx(scenes.Scene("one", [one], 2.0, 1.0, scenes.paper_direction()))
    ctx.assemble()
    x = torch.from_numpy(scenes.rhs_seeded(ctx.N, 2, 3)).cuda()
    y = torch.full_like(x, float("nan"))
    ctx.pairsum(x, y, q.PREC_FP64)
    assert float(torch.abs(y).max()) == 0.0
    ya, yb = torch.empty_like(x), torch.empty_like(x)
    ctx.apply(x, ya, q.PREC_FP64)
    ctx.selfblock_apply(x, yb, q.PREC_FP64)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
