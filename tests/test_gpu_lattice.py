"""Regular arrays of one body (Sec. 4, the block-Toeplitz structure of
P x Q x R lattices; Table tab:multibody_cubic) through the C ABI: the pair
sum applied through the circulant embedding against the oracle's pair sum
(Eq. multi2part, an explicit double loop) and against the direct GPU pair
sum, and lattice solves against the oracle's dense solve (Eq. linearsys)."""
import numpy as np
import pytest

import scenes
from gpu_util import rel_err
from oracle import operator as op
from oracle import solve as osolve
from oracle.geometry import body_nodes
from oracle.selfblock import self_block

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # FP64 blocks, FP64 transforms (the direct FP64 pair sum's bar)
FP32_TOL = 3e-5    # complex64 blocks and transforms (the direct FP32 pair sum's bar)


def skew_lattice(dims=(3, 2, 2), k=5.0):
    """A curved, rotated body on a non-orthogonal lattice."""
    body = scenes.Body(1, 8, 8, 0.5, (0.1, 0.05), (0.03,), 1.0, 0.3, tuple(scenes.rot_zy(0.4, 1.1)),
                       (0.2, -0.1, 0.3))
    basis = np.array([[2.6, 0.2, 0.0], [0.3, 2.5, 0.1], [0.0, -0.4, 2.7]])
    return scenes.lattice_scene("skew lattice", body, dims, basis, k, 1.0, scenes.fibonacci_directions(3))


def lattice_ctx(sc, min_gap=0.0):
    import paper_2606_31380_b300 as q
    ctx = q.Context(0)
    ctx.set_lattice(sc.body, sc.dims, sc.basis, min_gap)
    ctx.set_wavenumber(sc.k, sc.eta)
    return ctx


def gpu_pairsum(ctx, sigma, prec):
    import torch
    import paper_2606_31380_b300 as q
    dt = torch.complex64 if prec == q.PREC_FP32 else torch.complex128
    s = torch.from_numpy(sigma).to(dt).cuda()
    y = torch.full_like(s, float("nan"))
    ctx.pairsum(s, y, prec)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


def test_lattice_nodes_are_the_expanded_bodies():
    sc = skew_lattice()
    ctx = lattice_ctx(sc)
    x, n, w = ctx.get_nodes()
    nodes = [body_nodes(b) for b in sc.bodies]
    assert rel_err(x, np.concatenate([b.x for b in nodes])) < 1e-14
    assert rel_err(w, np.concatenate([b.w for b in nodes])) < 1e-13


@pytest.mark.parametrize("dims,n_rhs", [((3, 2, 2), 3), ((1, 1, 4), 1), ((2, 3, 1), 16), ((1, 1, 1), 2)])
def test_lattice_pairsum_against_oracle(dims, n_rhs):
    import paper_2606_31380_b300 as q
    sc = skew_lattice(dims)
    ctx = lattice_ctx(sc)
    ctx.lattice_prepare()
    nodes = [body_nodes(b) for b in sc.bodies]
    sigma = scenes.rhs_seeded(ctx.N, n_rhs, 11)
    ref = op.pair_sum(nodes, sigma, sc.k, sc.eta)
    ctx.profile(True)
    got64 = gpu_pairsum(ctx, sigma, q.PREC_FP64)
    got_ff = gpu_pairsum(ctx, sigma, q.PREC_FF)
    got32 = gpu_pairsum(ctx, sigma, q.PREC_FP32)
    assert ctx.profile_read(q.PROF_PAIRSUM_LATTICE)[0] == 3
    assert ctx.profile_read(q.PROF_PAIRSUM_FP64)[0] == 0
    if len(sc.bodies) == 1:
        assert np.all(got64 == 0) and np.all(got32 == 0)
        return
    assert rel_err(got64, ref) < FP64_TOL
    assert rel_err(got_ff, ref) < FP64_TOL
    assert rel_err(got32, ref) < FP32_TOL


def test_lattice_option_off_uses_the_direct_sum():
    import paper_2606_31380_b300 as q
    sc = skew_lattice()
    ctx = lattice_ctx(sc)
    ctx.lattice_prepare()
    sigma = scenes.rhs_seeded(ctx.N, 2, 12)
    on = gpu_pairsum(ctx, sigma, q.PREC_FP64)
    ctx.set_option(q.OPT_LATTICE, 0)
    assert ctx.get_option(q.OPT_LATTICE) == 0
    ctx.profile(True)
    off = gpu_pairsum(ctx, sigma, q.PREC_FP64)
    assert ctx.profile_read(q.PROF_PAIRSUM_LATTICE)[0] == 0
    assert ctx.profile_read(q.PROF_PAIRSUM_FP64)[0] >= 1
    assert rel_err(on, off) < FP64_TOL
    # a new wavenumber drops the transformed blocks: the direct sum until prepared again
    ctx.set_option(q.OPT_LATTICE, 1)
    ctx.set_wavenumber(7.0, 1.0)
    ctx.profile(True)
    direct7 = gpu_pairsum(ctx, sigma, q.PREC_FP64)
    assert ctx.profile_read(q.PROF_PAIRSUM_LATTICE)[0] == 0
    ctx.lattice_prepare()
    assert rel_err(gpu_pairsum(ctx, sigma, q.PREC_FP64), direct7) < FP64_TOL


def test_lattice_arguments():
    import paper_2606_31380_b300 as q
    sc = skew_lattice()
    ctx = q.Context(0)
    for dims in [(0, 1, 1), (33, 1, 1)]:
        with pytest.raises(q.QamsError):
            ctx.set_lattice(sc.body, dims, sc.basis)
    with pytest.raises(q.QamsError):
        ctx.set_lattice(sc.body, (2, 2, 2), np.full((3, 3), np.nan))
    with pytest.raises(q.QamsError) as e:           # spacing below the bounding balls
        ctx.set_lattice(sc.body, (2, 1, 1), 0.5 * sc.basis)
    assert e.value.code == -3
    ctx.set_lattice(sc.body, sc.dims, sc.basis)
    with pytest.raises(q.QamsError):                # no wavenumber yet
        ctx.lattice_prepare()
    ctx.set_bodies(sc.bodies)                        # plain bodies end the lattice mode
    ctx.set_wavenumber(sc.k, sc.eta)
    with pytest.raises(q.QamsError):
        ctx.lattice_prepare()


def test_paper_cubic_array_full_size():
    """10^3 quasi-ellipsoids, 16 x 6 nodes (Table tab:multibody_cubic), k = 5:
    the lattice apply against the direct GPU pair sum on every row and the
    oracle on sampled rows, all three precisions."""
    import paper_2606_31380_b300 as q
    sc = scenes.paper_cubic(10, 5.0)
    ctx = lattice_ctx(sc, min_gap=0.05)
    assert ctx.N == 96000
    sigma = scenes.rhs_seeded(ctx.N, 1, 13)
    ctx.set_option(q.OPT_LATTICE, 0)
    direct = gpu_pairsum(ctx, sigma, q.PREC_FP64)
    ctx.set_option(q.OPT_LATTICE, 1)
    ctx.lattice_prepare()
    got64 = gpu_pairsum(ctx, sigma, q.PREC_FP64)
    got32 = gpu_pairsum(ctx, sigma, q.PREC_FP32)
    assert rel_err(got64, direct) < FP64_TOL
    assert rel_err(got32, direct) < FP32_TOL
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(ctx.N, 40, replace=False))
    nodes = [body_nodes(b) for b in sc.bodies]
    ref = op.pair_sum(nodes, sigma, sc.k, sc.eta, targets=rows)
    assert rel_err(got64[rows], ref) < FP64_TOL


def test_workload_size_lattice_against_direct_sum():
    """10^3 copies of the 1000-body workload's first body (N = 512,000, k = 3,
    4 RHS): FP32 and float-float lattice applies against the direct ones."""
    import paper_2606_31380_b300 as q
    sc = scenes.lattice_of_workload(3)
    ctx = lattice_ctx(sc, min_gap=0.4)   # bounding balls 0.5 apart
    sigma = scenes.rhs_seeded(ctx.N, 4, 14)
    ctx.set_option(q.OPT_LATTICE, 0)
    d32 = gpu_pairsum(ctx, sigma, q.PREC_FP32)
    dff = gpu_pairsum(ctx, sigma, q.PREC_FF)
    ctx.set_option(q.OPT_LATTICE, 1)
    ctx.lattice_prepare()
    l32 = gpu_pairsum(ctx, sigma, q.PREC_FP32)
    lff = gpu_pairsum(ctx, sigma, q.PREC_FF)
    assert rel_err(lff, dff) < FP64_TOL
    assert rel_err(l32, dff) < FP32_TOL
    assert rel_err(d32, dff) < FP32_TOL
    rows = np.arange(0, ctx.N, 512 * 97 + 5)
    ref = op.pair_sum([body_nodes(b) for b in sc.bodies], sigma, sc.k, sc.eta, targets=rows)
    assert rel_err(lff[rows], ref) < FP64_TOL


@pytest.mark.parametrize("k", [2.0, 10.0])
def test_lattice_solve_against_oracle_dense_solve(k):
    """2^3 quasi-ellipsoids at the paper's discretisation: FP64 and mixed
    lattice solves and far fields against the oracle's dense LU."""
    import torch
    import paper_2606_31380_b300 as q
    sc = scenes.paper_cubic(2, k)
    nodes = [body_nodes(b) for b in sc.bodies]
    A1 = self_block(nodes[0], sc.k, sc.eta)
    A = op.dense_matrix(nodes, [A1] * len(nodes), sc.k, sc.eta)
    b_ref = op.incident(nodes, sc.directions, sc.k)
    mu_ref = osolve.dense_solve(A, b_ref)
    xh = scenes.fibonacci_directions(24)
    u_ref = op.farfield(nodes, mu_ref, xh, sc.k, sc.eta)
    ctx = lattice_ctx(sc, min_gap=0.05)
    ctx.assemble()
    b = torch.zeros((ctx.N, 1), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    for prec, tol, stol in [(q.PREC_FP64, 1e-10, 1e-13), (q.PREC_FP32, 1e-8, 1e-11)]:
        mu = torch.zeros_like(b)
        ctx.profile(True)
        st = ctx.solve(b, mu, prec, tol=stol)
        assert ctx.profile_read(q.PROF_PAIRSUM_LATTICE)[0] >= 1
        assert ctx.profile_read(q.PROF_PAIRSUM_FP32)[0] == 0 and ctx.profile_read(q.PROF_PAIRSUM_FF)[0] == 0
        u = torch.zeros((xh.shape[0], 1), dtype=torch.complex128, device="cuda")
        ctx.farfield(mu, xh, u)
        m = mu.cpu().numpy()
        assert np.linalg.norm(m - mu_ref) / np.linalg.norm(mu_ref) < tol, (prec, st)
        uu = u.cpu().numpy()
        assert np.linalg.norm(uu - u_ref) / np.linalg.norm(u_ref) < tol, (prec, st)
