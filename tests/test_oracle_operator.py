"""Pins for the oracle's inter-body sum (Eq. multi2part), incident and far field."""
import math

import numpy as np

import scenes
from oracle import operator as op
from oracle.geometry import body_nodes, gauss_legendre
from oracle.selfblock import pair_kernel


def test_kernel_hand_value():
    # x = 0, y = (2,0,0), n(y) = (1,0,0): rho = 2, n.(y-x) = 2.
    # K = e^{2ik}/(8 pi) [(ik/2 - 1/4) 2 - i eta]; k = 1, eta = 0.5:
    #   = e^{2i}/(8 pi) (-1/2 + 0.5 i)
    K = pair_kernel(np.zeros(3), np.array([2.0, 0, 0]), np.array([1.0, 0, 0]), 1.0, 0.5)
    ref = complex(math.cos(2), math.sin(2)) / (8 * math.pi) * complex(-0.5, 0.5)
    assert abs(K - ref) < 1e-16


def test_gauss_legendre_exactness():
    x, w = gauss_legendre(12)
    for p in range(24):
        assert abs(np.sum(w * x ** p) - (2.0 / (p + 1) if p % 2 == 0 else 0.0)) < 1e-14


def test_sphere_area_and_divergence_theorem():
    bn = body_nodes(scenes.sphere(0.7, 2, 16, 32, center=(1, 2, 3)))
    assert abs(bn.w.sum() - 4 * math.pi * 0.49) < 1e-12
    body = scenes.Body(2, 16, 32, 0.5, (0.06, 0.03), (0.04,), 1.0, 0.35, scenes.rot_zy(0.4, 1.0), (1, -1, 2))
    bn = body_nodes(body)
    # int x.n dS = 3 Vol and int n dS = 0 on a closed surface (outward normals)
    vol = np.sum(bn.w * np.sum(bn.x * bn.n, axis=1)) / 3
    assert vol > 0
    assert np.max(np.abs(bn.w @ bn.n)) < 1e-10
    assert abs(np.sum(bn.w * bn.x[:, 0] * bn.n[:, 0]) - vol) < 1e-10


def test_static_double_layer_vanishes_across_bodies():
    # k = 0, eta = 0, sigma = w: D_ab 1 = 0 for targets outside body b (Gauss's lemma)
    sc = scenes.small_scene(2, 2, 12, 24, k=0.0, eta=0.0, seed=3, box=4.0)
    nodes = [body_nodes(b) for b in sc.bodies]
    w = np.concatenate([n.w for n in nodes])
    y = op.pair_sum(nodes, w, 0.0, 0.0)
    assert np.max(np.abs(y)) < 1e-7


def test_pair_sum_matches_dense_blocks_and_multi_rhs():
    sc = scenes.small_scene(3, 1, 6, 8, k=2.5, seed=5)
    nodes = [body_nodes(b) for b in sc.bodies]
    N = sum(n.count for n in nodes)
    zero_blocks = [np.zeros((n.count, n.count)) for n in nodes]
    A = op.dense_matrix(nodes, zero_blocks, 2.5, 1.0)
    mu = scenes.rhs_seeded(N, 3, 11)
    y = op.apply(nodes, zero_blocks, mu, 2.5, 1.0)
    assert np.max(np.abs(y - A @ mu)) < 1e-13 * np.max(np.abs(y))
    y0 = op.apply(nodes, zero_blocks, mu[:, 0], 2.5, 1.0)
    assert np.max(np.abs(y0 - y[:, 0])) < 1e-15 * np.max(np.abs(y))


def test_farfield_of_point_density_is_plane_wave_factor():
    # one node with w mu = 1 at y: u_inf = (1/4pi)(-ik xhat.n - i eta) e^{-ik xhat.y}
    class One:
        x = np.array([[0.3, -0.2, 0.5]])
        n = np.array([[0.0, 0.6, 0.8]])
        w = np.array([1.0])
        count = 1
    xh = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])
    u = op.farfield([One], np.array([1.0]), xh, 2.0, 1.0)
    ref = (1 / (4 * math.pi)) * (-2j * (xh @ One.n[0]) - 1j) * np.exp(-2j * (xh @ One.x[0]))
    assert np.max(np.abs(u - ref)) < 1e-16
