"""GPU parity of the inter-body pair sum, incident field and far field against
the FP64 oracle (Eq. multi2part; Sec. 6)."""
import numpy as np
import pytest

import scenes
from gpu_util import make_ctx, rel_err
from oracle import operator as op
from oracle.geometry import body_nodes

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # pair-sum parity, FP64 path (apply-level target <= 1e-13 per entry norm)
FP32_TOL = 3e-5    # FP32 path: FP32 pair arithmetic with per-body-pair phase split
FF_TOL = 1e-12     # float-float path: ~48-bit pair arithmetic, FP64-accurate by design


def _ragged_scene(k=2.5, eta=1.0, n_rhs=1):
    rng = np.random.default_rng(21)
    discs = [(1, 6, 10), (2, 5, 12), (1, 7, 18), (1, 16, 16)]  # 60, 120, 126, 256 nodes
    bodies = []
    for i, disc in enumerate(discs):
        b = scenes.random_bodies(rng, 1, 1.0, 0.5, *disc)[0]
        b.center = (3.0 * i, 0.7 * (i % 2), -0.4 * i)
        bodies.append(b)
    d = scenes.paper_direction() if n_rhs == 1 else scenes.fibonacci_directions(n_rhs, rng)
    return scenes.Scene("ragged", bodies, k, eta, d)


def _gpu_pairsum(ctx, sigma, prec):
    import torch
    import paper_2606_31380_b300 as q
    dt = torch.complex64 if prec == q.PREC_FP32 else torch.complex128
    s = torch.from_numpy(sigma).to(dt).cuda()
    y = torch.full_like(s, float("nan"))
    ctx.pairsum(s, y, prec)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


def test_nodes_match_oracle_geometry():
    sc = _ragged_scene()
    ctx = make_ctx(sc)
    x, n, w = ctx.get_nodes()
    nodes = [body_nodes(b) for b in sc.bodies]
    assert rel_err(x, np.concatenate([b.x for b in nodes])) < 1e-14
    assert rel_err(n, np.concatenate([b.n for b in nodes])) < 1e-14
    assert rel_err(w, np.concatenate([b.w for b in nodes])) < 1e-13


@pytest.mark.parametrize("n_rhs", [1, 3, 16, 21])
def test_pairsum_ragged_fp64_and_fp32(n_rhs):
    import paper_2606_31380_b300 as q
    sc = _ragged_scene(n_rhs=n_rhs)
    ctx = make_ctx(sc)
    nodes = [body_nodes(b) for b in sc.bodies]
    sigma = scenes.rhs_seeded(ctx.N, n_rhs, 5)
    ref = op.pair_sum(nodes, sigma, sc.k, sc.eta)
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FP64), ref) < FP64_TOL
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FP32), ref) < FP32_TOL
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FF), ref) < FF_TOL


@pytest.mark.parametrize("eta,k", [(0.0, 1.0), (1.0, 15.0)])
def test_pairsum_small_random_scene(eta, k):
    import paper_2606_31380_b300 as q
    sc = scenes.small_scene(5, 1, 8, 16, k=k, eta=eta, seed=9, box=8.0)
    ctx = make_ctx(sc)
    nodes = [body_nodes(b) for b in sc.bodies]
    sigma = scenes.rhs_seeded(ctx.N, 2, 6)
    ref = op.pair_sum(nodes, sigma, sc.k, sc.eta)
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FP64), ref) < FP64_TOL
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FP32), ref) < FP32_TOL
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FF), ref) < FF_TOL


@pytest.mark.parametrize("cfg", [1, 2])
def test_pairsum_full_size_sampled_rows(cfg):
    """Full-size workloads (16 bodies x 2048 nodes, k = 5; 100 bodies x 1152
    nodes, k = 10, 16 RHS): every row computed on the GPU, sampled rows
    checked against the oracle's explicit sums."""
    import paper_2606_31380_b300 as q
    sc = scenes.config(cfg)
    ctx = make_ctx(sc)
    nodes = [body_nodes(b) for b in sc.bodies]
    R = sc.n_rhs
    sigma = scenes.rhs_seeded(ctx.N, R, 7)
    rng = np.random.default_rng(3)
    rows = np.concatenate([[0, ctx.N - 1], rng.integers(0, ctx.N, 30)])
    ref = op.pair_sum(nodes, sigma, sc.k, sc.eta, targets=rows)
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FP64)[rows], ref) < FP64_TOL
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FP32)[rows], ref) < FP32_TOL
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FF)[rows], ref) < FF_TOL


def test_incident_and_farfield():
    import torch
    sc = _ragged_scene(n_rhs=3)
    ctx = make_ctx(sc)
    nodes = [body_nodes(b) for b in sc.bodies]
    rhs = torch.zeros((ctx.N, 3), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, rhs)
    assert rel_err(rhs.cpu().numpy(), op.incident(nodes, sc.directions, sc.k)) < 1e-13
    mu = scenes.rhs_seeded(ctx.N, 3, 8)
    xh = scenes.fibonacci_directions(37)
    u = torch.zeros((37, 3), dtype=torch.complex128, device="cuda")
    ctx.farfield(torch.from_numpy(mu).cuda(), xh, u)
    assert rel_err(u.cpu().numpy(), op.farfield(nodes, mu, xh, sc.k, sc.eta)) < 1e-12


def test_pairsum_thousand_bodies_fp32_sampled_rows():
    """1000 bodies x 512 nodes (N = 512,000), k = 3, 4 RHS: the FP32 pair sum on
    every row, sampled rows against the oracle's explicit FP64 sums."""
    import paper_2606_31380_b300 as q
    sc = scenes.config(3)
    ctx = make_ctx(sc)
    nodes = [body_nodes(b) for b in sc.bodies]
    sigma = scenes.rhs_seeded(ctx.N, sc.n_rhs, 12)
    rng = np.random.default_rng(4)
    rows = np.concatenate([[0, ctx.N - 1], rng.integers(0, ctx.N, 14)])
    ref = op.pair_sum(nodes, sigma, sc.k, sc.eta, targets=rows)
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FP32)[rows], ref) < FP32_TOL
    assert rel_err(_gpu_pairsum(ctx, sigma, q.PREC_FF)[rows], ref) < FF_TOL


def test_scattered_field_against_oracle():
    """qams_field: the combined-layer field at off-surface points equals the
    oracle's explicit sum; 17 right-hand sides cover the 16-column chunking."""
    import torch
    sc = _ragged_scene()
    ctx = make_ctx(sc)
    nodes = [body_nodes(b) for b in sc.bodies]
    R = 17
    mu = scenes.rhs_seeded(ctx.N, R, 9)
    rng = np.random.default_rng(5)
    cand = rng.uniform(-4.0, 13.0, size=(400, 3))
    keep = [p for p in cand
            if all(np.linalg.norm(p - np.asarray(b.center)) > b.bound_radius() + 0.5 for b in sc.bodies)]
    pts = np.concatenate([np.asarray(keep[:29]), [[60.0, -40.0, 25.0]]])
    u = torch.full((len(pts), R), float("nan"), dtype=torch.complex128, device="cuda")
    ctx.field(torch.from_numpy(mu).cuda(), pts, u)
    ref = np.stack([op.field(nodes, mu[:, r], pts, sc.k, sc.eta) for r in range(R)], axis=1)
    assert rel_err(u.cpu().numpy(), ref) < 1e-12


def test_pairsum_fp64_large_phases():
    """FP64 pair sum with k rho up to ~3300: the table-driven e^{ik rho} (k rho
    below 3000) and the library fallback beyond it, entry by entry against
    the oracle's explicit sums."""
    import paper_2606_31380_b300 as q
    rng = np.random.default_rng(8)
    bodies = []
    for c in [(0.0, 0.0, 0.0), (120.0, 10.0, 5.0), (210.0, -30.0, 40.0), (3.0, 1.0, -2.0)]:
        b = scenes.random_bodies(rng, 1, 1.0, 0.5, 1, 6, 8)[0]
        b.center = c
        bodies.append(b)
    sc = scenes.Scene("far apart", bodies, 15.0, 1.0, scenes.paper_direction())
    ctx = make_ctx(sc)
    nodes = [body_nodes(b) for b in sc.bodies]
    sigma = scenes.rhs_seeded(ctx.N, 2, 13)
    ref = op.pair_sum(nodes, sigma, sc.k, sc.eta)
    got = _gpu_pairsum(ctx, sigma, q.PREC_FP64)
    gff = _gpu_pairsum(ctx, sigma, q.PREC_FF)
    # each body's rows separately: their scales differ by the distances.  Both
    # sides round rho differently by ~1 ulp, i.e. k rho by ~2e-13 at these
    # distances, which sets the tolerance; a wrong table entry, index or
    # reduction constant gives O(1) errors.
    off = np.cumsum([0] + [b.n_nodes for b in bodies])
    for a in range(len(bodies)):
        rows = slice(off[a], off[a + 1])
        assert rel_err(got[rows], ref[rows]) < FP64_TOL
        assert rel_err(gff[rows], ref[rows]) < FF_TOL
