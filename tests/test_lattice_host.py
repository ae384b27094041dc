"""Host-side checks of the regular-array workloads (Sec. 4, regular P x Q x R
arrays; Table tab:multibody_cubic): body order and spacing of the lattice
scenes, and the circulant-embedding identity the lattice pair sum relies
on (periods 2P - 1 hold every displacement on its own residue)."""
import itertools

import numpy as np

import scenes


def test_lattice_scene_order_and_centres():
    sc = scenes.paper_cubic(3, 2.0)
    assert sc.dims == (3, 3, 3) and len(sc.bodies) == 27
    c0 = np.asarray(sc.body.center)
    for idx, (p, q, r) in enumerate(itertools.product(range(3), range(3), range(3))):
        want = c0 + p * sc.basis[0] + q * sc.basis[1] + r * sc.basis[2]
        assert np.allclose(sc.bodies[idx].center, want, atol=0, rtol=0)
        assert sc.bodies[idx].rotation == sc.body.rotation


def test_paper_cubic_array_fits_the_paper_box_and_gap():
    sc = scenes.paper_cubic(10, 2.0)
    rb = sc.body.bound_radius()
    assert sc.n_nodes == 96000
    assert 0.5 - 2 * rb > 0.05          # bounding balls (so surfaces) more than 0.05 apart
    c = np.array([b.center for b in sc.bodies])
    assert c.min() - rb > -1.0 and c.max() + rb < 4.0


def test_workload_lattice_matches_the_workload():
    sc = scenes.lattice_of_workload(3)
    base = scenes.config(3)
    assert sc.n_nodes == base.n_nodes and sc.k == base.k
    assert np.array_equal(sc.directions, base.directions)
    h = sc.basis[0, 0]
    assert h == 2 * sc.body.bound_radius() + 0.5


def test_circulant_embedding_reproduces_the_block_toeplitz_sum():
    """y_t = sum_{s != t} T(t - s) sigma_s over a 3 x 2 x 4 lattice equals the
    inverse DFT of T^(f) sigma^(f) with periods 2P - 1 (random blocks)."""
    rng = np.random.default_rng(5)
    P = (3, 2, 4)
    L = tuple(2 * p - 1 for p in P)
    n, R = 3, 2
    T = rng.normal(size=L + (n, n)) + 1j * rng.normal(size=L + (n, n))
    T[0, 0, 0] = 0.0
    sig = rng.normal(size=P + (n, R)) + 1j * rng.normal(size=P + (n, R))
    direct = np.zeros(P + (n, R), complex)
    for t in itertools.product(*map(range, P)):
        for s in itertools.product(*map(range, P)):
            d = tuple((a - b) % l for a, b, l in zip(t, s, L))
            direct[t] += T[d] @ sig[s]
    pad = np.zeros(L + (n, R), complex)
    pad[: P[0], : P[1], : P[2]] = sig
    Th = np.fft.fftn(T, axes=(0, 1, 2))
    Sh = np.fft.fftn(pad, axes=(0, 1, 2))
    y = np.fft.ifftn(np.einsum("abcij,abcjr->abcir", Th, Sh), axes=(0, 1, 2))[: P[0], : P[1], : P[2]]
    assert np.max(np.abs(y - direct)) < 1e-12 * np.max(np.abs(direct))
