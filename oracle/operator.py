"""Oracle multi-body operator, incident field and far field (test infrastructure only).

* ``pair_sum`` -- the inter-body smooth rule (Eq. multi2part) written as the
  explicit double sum over every target node and every node of every *other*
  body, with the combined-layer kernel (Sec. 2 Remark)
      K(x, y) = e^{ik rho}/(4 pi rho) [(ik/rho - 1/rho^2) n(y).(y - x) - i eta],
  and the quadrature weights folded into the density, sigma = w mu.
  This is the plain definition of the matrix-free off-diagonal blocks
  D_{t',t} of Eq. linearsys; nothing is blocked or reordered.
* ``apply`` -- (1/2 I + D - i eta S) mu: self blocks (diagonal of Eq.
  linearsys) plus the pair sum.
* ``incident`` -- right-hand side -u^inc with u^inc = e^{ik d.x} (Sec. 6).
* ``farfield`` -- u_inf(xhat) = (1/4pi) sum_y (-ik xhat.n(y) - i eta) e^{-ik xhat.y} w mu
  (Sec. 6 far-field formula, restated for the combined layer).
* ``field`` -- the scattered field (D - i eta S)[mu] at off-surface points.

Pins: tests/test_oracle_operator.py (hand-computed two-node values, k = 0
Gauss identity across bodies, Mie series, interior point sources, reciprocity).
"""
from __future__ import annotations

import numpy as np

from .selfblock import pair_kernel


def _cat(nodes, attr):
    return np.concatenate([getattr(b, attr) for b in nodes])


def body_offsets(nodes):
    off = [0]
    for b in nodes:
        off.append(off[-1] + b.count)
    return off


def pair_sum(nodes, sigma, k: float, eta: float, targets=None):
    """y_t = sum over nodes s of other bodies of K(x_t, y_s) sigma_s.

    ``sigma`` is (N,) or (N, R); ``targets`` optionally restricts to a list of
    global target indices (the rows are returned in that order)."""
    sigma = np.asarray(sigma)
    vec = sigma.ndim == 1
    if vec:
        sigma = sigma[:, None]
    off = body_offsets(nodes)
    X = _cat(nodes, "x")
    Nn = _cat(nodes, "n")
    owner = np.concatenate([np.full(b.count, i) for i, b in enumerate(nodes)])
    tlist = np.arange(len(X)) if targets is None else np.asarray(targets)
    out = np.zeros((len(tlist), sigma.shape[1]), complex)
    for row, t in enumerate(tlist):
        bt = owner[t]
        src = np.r_[0:off[bt], off[bt + 1]:len(X)]
        K = pair_kernel(X[t][None, :], X[src], Nn[src], k, eta)
        out[row] = K @ sigma[src]
    return out[:, 0] if vec else out


def apply(nodes, self_blocks, mu, k: float, eta: float):
    """(1/2 I + D - i eta S) mu for the whole scene (Eq. linearsys)."""
    mu = np.asarray(mu)
    off = body_offsets(nodes)
    w = _cat(nodes, "w")
    sig = (w[:, None] * mu) if mu.ndim == 2 else w * mu
    y = pair_sum(nodes, sig, k, eta)
    for i, A in enumerate(self_blocks):
        y[off[i]:off[i + 1]] += A @ mu[off[i]:off[i + 1]]
    return y


def dense_matrix(nodes, self_blocks, k: float, eta: float):
    """The full N x N system matrix (small scenes only)."""
    off = body_offsets(nodes)
    X, Nn, w = _cat(nodes, "x"), _cat(nodes, "n"), _cat(nodes, "w")
    N = len(X)
    A = np.zeros((N, N), complex)
    for a in range(len(nodes)):
        for b in range(len(nodes)):
            ra, rb = slice(off[a], off[a + 1]), slice(off[b], off[b + 1])
            if a == b:
                A[ra, rb] = self_blocks[a]
            else:
                A[ra, rb] = pair_kernel(X[ra][:, None, :], X[rb][None, :, :], Nn[rb][None, :, :],
                                        k, eta) * w[rb][None, :]
    return A


def incident(nodes, dirs, k: float):
    """-u^inc = -e^{ik d.x} at every node, (N, R)."""
    X = _cat(nodes, "x")
    return -np.exp(1j * k * (X @ np.asarray(dirs).T))


def farfield(nodes, mu, xhat, k: float, eta: float):
    """u_inf at unit directions ``xhat`` (M, 3) for densities mu (N,) or (N, R)."""
    X, Nn, w = _cat(nodes, "x"), _cat(nodes, "n"), _cat(nodes, "w")
    mu = np.asarray(mu)
    vec = mu.ndim == 1
    if vec:
        mu = mu[:, None]
    xhat = np.asarray(xhat)
    E = np.exp(-1j * k * (xhat @ X.T)) * (-1j * k * (xhat @ Nn.T) - 1j * eta)
    out = E @ (w[:, None] * mu) / (4 * np.pi)
    return out[:, 0] if vec else out


def field(nodes, mu, points, k: float, eta: float):
    """Scattered field (D - i eta S)[mu] at off-surface points (P, 3)."""
    X, Nn, w = _cat(nodes, "x"), _cat(nodes, "n"), _cat(nodes, "w")
    K = pair_kernel(np.asarray(points)[:, None, :], X[None, :, :], Nn[None, :, :], k, eta)
    return K @ (w * np.asarray(mu))
