"""Pins for the oracle self block (Sec. 3.1-3.4 product integration; jump
relation Eq. jump3) and, through full solves, the whole oracle path."""
import numpy as np
import pytest
from scipy import special as sp

import closed_forms as cf
import scenes
from oracle import operator as op
from oracle import solve
from oracle.geometry import body_nodes
from oracle.selfblock import self_block, self_block_rows

CURVED = dict(base_radius=0.5, mode_cos=(0.06, 0.03), mode_sin=(0.04,), axis_length=1.0, curvature=0.35)


def test_gauss_identity_on_curved_body():
    """k = 0, eta = 0: (1/2 I + D) 1 = 0 on a closed surface (Gauss's lemma).
    The double layer integrates the exact area-weighted normal against an
    interpolant of mu, which is exact for mu = 1, so the identity holds to
    the accuracy of the quadrature itself at any discretisation."""
    for disc in [(1, 8, 16), (2, 12, 24)]:
        bn = body_nodes(scenes.Body(*disc, **CURVED))
        rows = [bn.count // 2 + 3, 5, bn.count - 1]
        A = self_block_rows(bn, rows, 0.0, 0.0, tol=1e-13)
        assert np.max(np.abs(A.sum(axis=1))) < 1e-12


def test_sphere_eigenvalues():
    a, k = 0.5, 2.0
    bn = body_nodes(scenes.sphere(a, 2, 12, 24))
    A = self_block(bn, k, 1.0, tol=1e-13)
    S, T = np.meshgrid(bn.s, bn.theta, indexing="ij")
    S, T = S.reshape(-1), T.reshape(-1)
    for n, m, tol in [(0, 0, 1e-13), (1, 0, 1e-10), (2, 1, 1e-9), (3, 3, 1e-8)]:
        Y = sp.lpmv(m, n, np.sin(S)) * np.exp(1j * m * T)
        lam = cf.sphere_eigen(a, k, n, 1.0)
        assert np.linalg.norm(A @ Y - lam * Y) / np.linalg.norm(Y) < tol


def test_mie_series_sphere():
    a, k = 0.5, 2.0
    d = np.array([0.3, 0.5, np.sqrt(1 - 0.34)])
    bn = body_nodes(scenes.sphere(a, 2, 12, 24))
    A = self_block(bn, k, 1.0, tol=1e-13)
    mu = solve.dense_solve(A, op.incident([bn], d[None, :], k)[:, 0])
    xh = np.random.default_rng(1).normal(size=(20, 3))
    xh /= np.linalg.norm(xh, axis=1, keepdims=True)
    uinf = op.farfield([bn], mu, xh, k, 1.0)
    ref = cf.mie_farfield(a, k, d, xh)
    assert np.linalg.norm(uinf - ref) / np.linalg.norm(ref) < 1e-11


def test_circulant_shortcut_matches_direct_rows():
    body = scenes.Body(1, 8, 16, 0.5, (0.1,), (0.05,), 1.0, 0.0)
    bn = body_nodes(body)
    full = self_block(bn, 3.0, 1.0, tol=1e-13)
    rows = [3, 42, 77]
    direct = self_block_rows(bn, rows, 3.0, 1.0, tol=1e-13)
    assert np.max(np.abs(full[rows] - direct)) < 1e-12 * np.max(np.abs(direct))


@pytest.mark.slow
def test_point_sources_two_curved_bodies_converge():
    """Interior point sources (Eq. artificial point source solution): the exterior
    field of the computed density converges to the exact one."""
    k = 2.0
    errs = []
    for disc in [(1, 8, 16), (2, 8, 16)]:
        b1 = scenes.Body(*disc, **CURVED, rotation=scenes.rot_zy(0.3, 1.1), center=(0, 0, 0))
        b2 = scenes.Body(*disc, **CURVED, rotation=scenes.rot_zy(2.0, 0.4), center=(2.2, 0.5, -0.3))
        nodes = [body_nodes(b1), body_nodes(b2)]
        A1 = self_block(nodes[0], k, 1.0, tol=1e-13)  # congruent bodies share one block
        A = op.dense_matrix(nodes, [A1, A1], k, 1.0)
        z = np.array([b1.center, b2.center], float)
        X = np.concatenate([n.x for n in nodes])
        mu = solve.dense_solve(A, cf.point_source_field(X, z, k))
        pts = np.array([[4.0, 1, 2], [-3, 2, 1], [1, -4, 0.5], [1.1, 3, -2]])
        u = op.field(nodes, mu, pts, k, 1.0)
        ex = cf.point_source_field(pts, z, k)
        errs.append(np.max(np.abs(u - ex)) / np.max(np.abs(ex)))
    assert errs[0] < 2e-2 and errs[1] < 5e-4 and errs[0] / errs[1] > 20


def test_farfield_reciprocity_two_bodies():
    """Reciprocity of the far-field pattern (the textbook relation for the
    sound-soft problem, u_inf(xhat; d) = u_inf(-d; -xhat)) holds for the
    discrete solutions to the discretisation error.  A sign or conjugation
    slip in the incident field, the far field or the kernel breaks it at O(1)."""
    k = 2.0
    shape = dict(base_radius=0.5, mode_cos=(0.15, 0.05), mode_sin=(0.08,), axis_length=1.0, curvature=0.0)
    b1 = scenes.Body(2, 8, 16, **shape, rotation=scenes.rot_zy(0.3, 1.1), center=(0, 0, 0))
    b2 = scenes.Body(2, 8, 16, **shape, rotation=scenes.rot_zy(2.0, 0.4), center=(2.0, 0.6, -0.4))
    nodes = [body_nodes(b1), body_nodes(b2)]
    A1 = self_block(nodes[0], k, 1.0, tol=1e-13)
    A = op.dense_matrix(nodes, [A1, A1], k, 1.0)
    d = scenes.fibonacci_directions(3, np.random.default_rng(2))
    D = np.concatenate([d, -d])          # closed under negation: neg(j) = (j + 3) % 6
    mu = solve.dense_solve(A, op.incident(nodes, D, k))
    U = op.farfield(nodes, mu, D, k, 1.0)  # U[i, j] = u_inf(D_i; D_j)
    neg = (np.arange(6) + 3) % 6
    Ur = U[neg][:, neg].T                   # u_inf(-D_j; -D_i)
    off = ~np.eye(6, dtype=bool)
    err = np.max(np.abs(U - Ur)[off]) / np.max(np.abs(U))
    assert err < 1e-4
    # the same relation fails by O(1) with the incident phase conjugated
    mu_bad = solve.dense_solve(A, np.conj(op.incident(nodes, D, k)))
    Ub = op.farfield(nodes, mu_bad, D, k, 1.0)
    assert np.max(np.abs(Ub - Ub[neg][:, neg].T)[off]) / np.max(np.abs(Ub)) > 1e-2
