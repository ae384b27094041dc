"""Oracle linear solvers (test infrastructure only).

The paper solves the dense system with a direct solver or with GMRES and a
block-diagonal preconditioner built from the LU factors of the self matrix
(Sec. 6, solver description).  Restart length, tolerance, initial guess and
orthogonalisation are not stated; the reading used here is restarted
GMRES(m) from x0 = 0 with right preconditioning, classical Gram-Schmidt
applied twice, Givens rotations, stopping at ||b - A x|| <= tol ||b||.

Pins: tests/test_oracle_solve.py (GMRES against the dense direct solve,
exact convergence in n steps on an n x n system, preconditioned and plain
runs agree).
"""
from __future__ import annotations

import numpy as np


def dense_solve(A, b):
    """Direct solve by LU with partial pivoting (library routine)."""
    return np.linalg.solve(A, b)


def gmres(apply_fn, b, tol=1e-12, restart=50, maxiter=2000, precond=None):
    """Right-preconditioned restarted GMRES for one right-hand side.

    ``apply_fn(x)`` returns A x; ``precond(x)`` returns M^{-1} x (identity if
    None).  Returns (x, iterations, relative residual)."""
    b = np.asarray(b, complex)
    n = b.shape[0]
    P = precond if precond is not None else (lambda v: v)
    x = np.zeros(n, complex)
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, 0, 0.0
    it = 0
    r = b - apply_fn(x)
    beta = np.linalg.norm(r)
    while it < maxiter:
        V = np.zeros((restart + 1, n), complex)
        H = np.zeros((restart + 1, restart), complex)
        cs = np.zeros(restart, complex)
        sn = np.zeros(restart, complex)
        g = np.zeros(restart + 1, complex)
        V[0] = r / beta
        g[0] = beta
        j_done = 0
        for j in range(restart):
            w = apply_fn(P(V[j]))
            for _ in range(2):  # classical Gram-Schmidt, twice
                h = V[: j + 1].conj() @ w
                w = w - h @ V[: j + 1]
                H[: j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # apply previous rotations G_i = [[c*, s*], [-s, c]]
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = a / den if den else 1.0
            sn[j] = bb / den if den else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol * bnorm or it >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + P(y @ V[:j_done])
        r = b - apply_fn(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
    return x, it, beta / bnorm
