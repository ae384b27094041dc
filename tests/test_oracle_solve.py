"""Pins for the oracle solvers (Sec. 6 solver description; GMRES reading)."""
import numpy as np

from oracle.solve import dense_solve, gmres


def _mat(n, seed):
    rng = np.random.default_rng(seed)
    return np.eye(n) * 0.5 + (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / (3 * np.sqrt(n))


def test_gmres_matches_direct_solve():
    A = _mat(80, 1)
    b = np.random.default_rng(2).normal(size=80) + 0j
    x, it, rel = gmres(lambda v: A @ v, b, tol=1e-13, restart=30)
    assert rel < 1e-13
    assert np.linalg.norm(x - dense_solve(A, b)) < 1e-11 * np.linalg.norm(x)


def test_gmres_terminates_in_n_steps_without_restart():
    A = _mat(12, 3) + 2 * np.diag(np.arange(12))
    b = np.ones(12, complex)
    x, it, rel = gmres(lambda v: A @ v, b, tol=1e-14, restart=12)
    assert it <= 12 and rel < 1e-12


def test_block_jacobi_right_preconditioning():
    A = _mat(60, 4)
    blocks = [slice(0, 20), slice(20, 45), slice(45, 60)]
    inv = [np.linalg.inv(A[s, s]) for s in blocks]

    def prec(v):
        out = np.empty_like(v)
        for s, M in zip(blocks, inv):
            out[s] = M @ v[s]
        return out

    b = np.arange(60) + 1j
    x0, it0, _ = gmres(lambda v: A @ v, b, tol=1e-13, restart=60)
    x1, it1, _ = gmres(lambda v: A @ v, b, tol=1e-13, restart=60, precond=prec)
    assert np.linalg.norm(x0 - x1) < 1e-11 * np.linalg.norm(x0)
    assert it1 <= it0
