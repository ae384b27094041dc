"""GPU solves (Sec. 4, Eq. linearsys; Sec. 6) against the oracle's dense
direct solve and against closed forms."""
import numpy as np
import pytest

import closed_forms as cf
import scenes
from gpu_util import make_ctx
from oracle import operator as op
from oracle import solve as osolve
from oracle.geometry import body_nodes
from oracle.selfblock import self_block

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10   # densities / far field, FP64 path (relative L2)
MIXED_TOL = 1e-8   # densities / far field, FP32 operator + FP64 refinement


def l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def gpu_solve(scene, rhs, precision, **kw):
    import torch
    ctx = make_ctx(scene)
    ctx.assemble()
    b = torch.from_numpy(np.ascontiguousarray(rhs)).cuda()
    mu = torch.zeros_like(b)
    stats = ctx.solve(b, mu, precision, **kw)
    return ctx, mu, stats


def test_two_axisymmetric_bodies_against_dense_lu():
    """Two straight bodies rho = 0.5(1 + 0.2 cos 2 pi u), 16 x 32 nodes, centres
    3 apart, k = 1, plane wave along x: oracle dense LU to machine precision."""
    import torch
    import paper_2606_31380_b300 as q
    sc = scenes.config(0)
    nodes = [body_nodes(b) for b in sc.bodies]
    A1 = self_block(nodes[0], sc.k, sc.eta)
    A = op.dense_matrix(nodes, [A1, A1], sc.k, sc.eta)
    b = op.incident(nodes, sc.directions, sc.k)
    mu_ref = osolve.dense_solve(A, b)
    xh = scenes.fibonacci_directions(400)
    u_ref = op.farfield(nodes, mu_ref, xh, sc.k, sc.eta)
    for prec, tol in [(q.PREC_FP64, FP64_TOL), (q.PREC_FP32, MIXED_TOL)]:
        ctx, mu, st = gpu_solve(sc, b, prec, tol=1e-13 if prec == q.PREC_FP64 else 1e-11)
        assert l2(mu.cpu().numpy(), mu_ref) < tol, st
        u = torch.zeros((400, 1), dtype=torch.complex128, device="cuda")
        ctx.farfield(mu, xh, u)
        assert l2(u.cpu().numpy(), u_ref) < tol


def test_mie_sphere_through_gpu_solve():
    import torch
    import paper_2606_31380_b300 as q
    a, k = 0.5, 2.0
    d = np.array([[0.3, 0.5, np.sqrt(1 - 0.34)]])
    sc = scenes.Scene("sphere", [scenes.sphere(a, 2, 12, 24)], k, 1.0, d)
    ctx = make_ctx(sc)
    ctx.assemble()
    b = torch.zeros((ctx.N, 1), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(d, b)
    mu = torch.zeros_like(b)
    ctx.solve(b, mu, q.PREC_FP64, tol=1e-13)
    xh = scenes.fibonacci_directions(50)
    u = torch.zeros((50, 1), dtype=torch.complex128, device="cuda")
    ctx.farfield(mu, xh, u)
    ref = cf.mie_farfield(a, k, d[0], xh)
    assert l2(u.cpu().numpy()[:, 0], ref) < 1e-11


def test_point_sources_curved_bodies_and_multi_rhs():
    """Interior point sources on two congruent curved bodies: GPU densities match
    the oracle's dense solve, the exterior field matches the exact one to the
    discretisation error, and a 3-column solve equals three 1-column solves."""
    import torch
    import paper_2606_31380_b300 as q
    k = 2.0
    shape = dict(base_radius=0.5, mode_cos=(0.06, 0.03), mode_sin=(0.04,), axis_length=1.0, curvature=0.35)
    b1 = scenes.Body(2, 8, 16, **shape, rotation=scenes.rot_zy(0.3, 1.1), center=(0, 0, 0))
    b2 = scenes.Body(2, 8, 16, **shape, rotation=scenes.rot_zy(2.0, 0.4), center=(2.2, 0.5, -0.3))
    sc = scenes.Scene("pts", [b1, b2], k, 1.0, scenes.paper_direction())
    nodes = [body_nodes(b1), body_nodes(b2)]
    X = np.concatenate([n.x for n in nodes])
    z = np.array([b1.center, b2.center], float)
    g = cf.point_source_field(X, z, k)
    rhs = np.stack([g, op.incident(nodes, scenes.paper_direction(), k)[:, 0], np.cos(X[:, 0]) + 0j], axis=1)
    A1 = self_block(nodes[0], k, 1.0)
    A = op.dense_matrix(nodes, [A1, A1], k, 1.0)
    mu_ref = osolve.dense_solve(A, rhs)
    ctx, mu, st = gpu_solve(sc, rhs, q.PREC_FP64, tol=1e-13)
    mu3 = mu.cpu().numpy()
    assert l2(mu3, mu_ref) < FP64_TOL
    for r in range(3):
        _, m1, _ = gpu_solve(sc, rhs[:, r:r + 1], q.PREC_FP64, tol=1e-13)
        assert l2(m1.cpu().numpy()[:, 0], mu3[:, r]) < 1e-11
    pts = np.array([[4.0, 1, 2], [-3, 2, 1], [1, -4, 0.5]])
    u = op.field(nodes, mu3[:, 0], pts, k, 1.0)
    ex = cf.point_source_field(pts, z, k)
    assert np.max(np.abs(u - ex)) / np.max(np.abs(ex)) < 5e-4
    ug = torch.zeros((3, 1), dtype=torch.complex128, device="cuda")
    ctx.field(mu[:, :1].contiguous(), pts, ug)
    assert l2(ug.cpu().numpy()[:, 0], u) < 1e-12
    _, mm, st = gpu_solve(sc, rhs, q.PREC_FP32, tol=1e-11)
    assert l2(mm.cpu().numpy(), mu_ref) < MIXED_TOL


def test_sixteen_bodies_full_size_residual_rows():
    """16 bodies x 2048 nodes, k = 5: the mixed solve's densities satisfy the
    oracle's equations -- sampled rows of b - A mu (oracle self-block rows and
    explicit pair sums) are small against |b|."""
    import torch
    import paper_2606_31380_b300 as q
    from oracle.selfblock import self_block_rows_parallel
    sc = scenes.config(1)
    ctx = make_ctx(sc)
    ctx.assemble()
    b = torch.zeros((ctx.N, 1), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    mu = torch.zeros_like(b)
    st = ctx.solve(b, mu, q.PREC_FP32, tol=1e-11)
    assert st["rel_residual"] <= 1e-11
    nodes = [body_nodes(x) for x in sc.bodies]
    off = ctx.body_offsets()
    m = mu.cpu().numpy()
    bb = op.incident(nodes, sc.directions, sc.k)
    w = np.concatenate([n.w for n in nodes])
    rows = [17, 2048 * 5 + 999, 2048 * 12 + 2040]
    Am = op.pair_sum(nodes, w[:, None] * m, sc.k, sc.eta, targets=rows)
    for i, gidx in enumerate(rows):
        bi = int(np.searchsorted(off, gidx, side="right") - 1)
        row = self_block_rows_parallel(nodes[bi], [gidx - off[bi]], sc.k, sc.eta, workers=1)[0]
        Am[i] += row @ m[off[bi]:off[bi + 1]]
    assert np.max(np.abs(Am - bb[rows])) < 1e-9 * np.max(np.abs(bb))
    # one row per body, every column: the GPU self-block part (its rows are checked against
    # the oracle's elsewhere to 1e-12) plus the oracle's explicit pair sum
    ys = torch.zeros_like(mu)
    ctx.selfblock_apply(mu, ys, q.PREC_FP64)
    rows_all = off[:-1] + (np.arange(len(sc.bodies)) * 37) % 512
    Ap = op.pair_sum(nodes, w[:, None] * m, sc.k, sc.eta, targets=rows_all)
    res_all = bb[rows_all] - ys.cpu().numpy()[rows_all] - Ap
    assert np.max(np.abs(res_all)) < 1e-9 * np.max(np.abs(bb))


def test_block_jacobi_preconditioner():
    """P_b A_b = I up to complex64 rounding for bodies of ragged sizes (one, several
    and a partial pivot block), and the preconditioned FP64 solve returns the same
    densities as the plain one in fewer iterations (Sec. 6 block-diagonal
    preconditioner)."""
    import torch
    import paper_2606_31380_b300 as q
    rng = np.random.default_rng(8)
    discs = [(1, 6, 10), (2, 12, 24), (1, 16, 32)]  # 60, 576, 512 nodes
    bodies = []
    for i, disc in enumerate(discs):
        b = scenes.random_bodies(rng, 1, 1.0, 0.5, *disc)[0]
        b.center = (3.2 * i, 0.5 * i, 0.0)
        bodies.append(b)
    sc = scenes.Scene("ragged", bodies, 6.0, 1.0, scenes.paper_direction())
    ctx = make_ctx(sc)
    ctx.assemble()
    ctx.build_preconditioner()
    off = ctx.body_offsets()
    for bi in range(len(bodies)):
        n = int(off[bi + 1] - off[bi])
        A = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
        P = torch.zeros_like(A)
        ctx.copy_selfblock(bi, A)
        ctx.copy_preconditioner(bi, P)
        E = (P @ A).cpu().numpy() - np.eye(n)
        assert np.max(np.abs(E)) < 1e-3
    # the block-diagonal products through the C ABI, R = 3 (FP64 and FP32)
    x = torch.from_numpy(scenes.rhs_seeded(ctx.N, 3, 21)).cuda()
    for prec, dt, tol in [(q.PREC_FP64, torch.complex128, 1e-14), (q.PREC_FP32, torch.complex64, 1e-5)]:
        ya = torch.full_like(x.to(dt), float("nan"))
        yp = torch.full_like(x.to(dt), float("nan"))
        ctx.selfblock_apply(x.to(dt).contiguous(), ya, prec)
        ctx.precond_apply(x.to(dt).contiguous(), yp, prec)
        for bi in range(len(bodies)):
            n = int(off[bi + 1] - off[bi])
            rows = slice(int(off[bi]), int(off[bi + 1]))
            A = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
            P = torch.zeros_like(A)
            ctx.copy_selfblock(bi, A)
            ctx.copy_preconditioner(bi, P)
            refa = (A @ x[rows]).cpu().numpy()
            refp = (P @ x[rows]).cpu().numpy()
            assert np.max(np.abs(ya[rows].cpu().numpy() - refa)) < tol * np.max(np.abs(refa))
            assert np.max(np.abs(yp[rows].cpu().numpy() - refp)) < tol * np.max(np.abs(refp))
    b = torch.zeros((ctx.N, 1), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    m0 = torch.zeros_like(b)
    m1 = torch.zeros_like(b)
    s0 = ctx.solve(b, m0, q.PREC_FP64, tol=1e-13, precondition=False)
    s1 = ctx.solve(b, m1, q.PREC_FP64, tol=1e-13, precondition=True)
    assert l2(m1.cpu().numpy(), m0.cpu().numpy()) < 1e-11
    assert s1["iterations"] < s0["iterations"]
    m2 = torch.zeros_like(b)
    ctx.solve(b, m2, q.PREC_FP32, tol=1e-11, precondition=True)
    assert l2(m2.cpu().numpy(), m0.cpu().numpy()) < MIXED_TOL


def test_farfield_reciprocity_curved_bodies():
    """u_inf(xhat; d) = u_inf(-d; -xhat) for the GPU solutions of four curved
    random bodies (directions closed under negation, one multi-RHS solve)."""
    import torch
    import paper_2606_31380_b300 as q
    rng = np.random.default_rng(17)
    bodies = scenes.random_bodies(rng, 4, 4.0, 0.5, 2, 16, 32)
    d = scenes.fibonacci_directions(4, rng)
    D = np.concatenate([d, -d])
    sc = scenes.Scene("reciprocity", bodies, 3.0, 1.0, D)
    ctx = make_ctx(sc)
    ctx.assemble()
    b = torch.zeros((ctx.N, 8), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(D, b)
    mu = torch.zeros_like(b)
    ctx.solve(b, mu, q.PREC_FP64, tol=1e-13)
    U = torch.zeros((8, 8), dtype=torch.complex128, device="cuda")
    ctx.farfield(mu, D, U)
    U = U.cpu().numpy()                      # U[i, j] = u_inf(D_i; D_j)
    neg = (np.arange(8) + 4) % 8
    off = ~np.eye(8, dtype=bool)
    err = np.max(np.abs(U - U[neg][:, neg].T)[off]) / np.max(np.abs(U))
    assert err < 1e-6


def test_hundred_bodies_sixteen_rhs_residual_rows():
    """100 bodies x 1152 nodes, k = 10, 16 incident directions (N = 115,200):
    the mixed solve of all 16 columns, then sampled rows of b - A mu from
    oracle self-block rows and explicit pair sums, every column."""
    import torch
    import paper_2606_31380_b300 as q
    from oracle.selfblock import self_block_rows_parallel
    sc = scenes.config(2)
    ctx = make_ctx(sc)
    ctx.assemble()
    R = sc.n_rhs
    b = torch.zeros((ctx.N, R), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    mu = torch.zeros_like(b)
    st = ctx.solve(b, mu, q.PREC_FP32, tol=1e-11)
    assert st["rel_residual"] <= 1e-11
    nodes = [body_nodes(x) for x in sc.bodies]
    off = ctx.body_offsets()
    m = mu.cpu().numpy()
    bb = op.incident(nodes, sc.directions, sc.k)
    w = np.concatenate([n.w for n in nodes])
    rows = [3, 1152 * 41 + 577, 1152 * 99 + 1151]
    Am = op.pair_sum(nodes, w[:, None] * m, sc.k, sc.eta, targets=rows)
    for i, gidx in enumerate(rows):
        bi = int(np.searchsorted(off, gidx, side="right") - 1)
        row = self_block_rows_parallel(nodes[bi], [gidx - off[bi]], sc.k, sc.eta, workers=1)[0]
        Am[i] += row @ m[off[bi]:off[bi + 1]]
    assert np.max(np.abs(Am - bb[rows])) < 1e-9 * np.max(np.abs(bb))


def test_thousand_bodies_four_rhs_residual_rows():
    """1000 bodies x 512 nodes, k = 3, 4 incident directions (N = 512,000): the
    mixed solve of all 4 columns, then sampled rows of b - A mu from oracle
    self-block rows and explicit pair sums over all 511,488 other-body nodes."""
    import torch
    import paper_2606_31380_b300 as q
    from oracle.selfblock import self_block_rows_parallel
    sc = scenes.config(3)
    ctx = make_ctx(sc)
    ctx.assemble()
    R = sc.n_rhs
    b = torch.zeros((ctx.N, R), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    mu = torch.zeros_like(b)
    st = ctx.solve(b, mu, q.PREC_FP32, tol=1e-11)
    assert st["rel_residual"] <= 1e-11
    nodes = [body_nodes(x) for x in sc.bodies]
    off = ctx.body_offsets()
    m = mu.cpu().numpy()
    bb = op.incident(nodes, sc.directions, sc.k)
    w = np.concatenate([n.w for n in nodes])
    rows = [0, 512 * 433 + 100, 512 * 999 + 511]
    Am = op.pair_sum(nodes, w[:, None] * m, sc.k, sc.eta, targets=rows)
    for i, gidx in enumerate(rows):
        bi = int(np.searchsorted(off, gidx, side="right") - 1)
        row = self_block_rows_parallel(nodes[bi], [gidx - off[bi]], sc.k, sc.eta, workers=1)[0]
        Am[i] += row @ m[off[bi]:off[bi + 1]]
    assert np.max(np.abs(Am - bb[rows])) < 1e-9 * np.max(np.abs(bb))
