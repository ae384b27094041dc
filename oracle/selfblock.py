"""Oracle self-interaction block (test infrastructure only).

Row t of the self block of one body, for the combined-layer operator
1/2 + D - i eta S (Sec. 2 Remark, Sec. 3.1-3.4), target x_t on panel p:

* source panels i with |i - p| <= 1 (singular / near-singular, Eq. sx):
  product integration against a tensor Lagrange interpolant, P_l(s) in s
  and L_j(theta) in theta (Sec. 3.1):
      A[t, (i,l,j)] = int_{panel i} P_l(s) [F^D_j(s) + |J_ilj| F^S_j(s)] ds,
      F^D_j(s) = int [(|J| n_r)(s,theta) K^r + (|J| n_z)(s,theta) K^z] L_j dtheta,
      F^S_j(s) = -i eta int G L_j dtheta,
  where K^r, K^z are the source-derivative kernels of Sec. 3.2 and all
  theta-integrals come from modal Green's functions (modal.py).
  Reading used for quasi-axisymmetric bodies: the paper interpolates mu |J|
  and treats n_r, n_z as constants, which holds only on bodies of
  revolution.  Here the single layer keeps the mu |J| interpolant, and the
  double layer interpolates mu and integrates the exact area-weighted
  normal, which on both surface families is a trigonometric polynomial of
  degree one in theta (geometry.py):
      |J| n_r = a0 + a1 cos theta,   |J| n_z = b0 + b1 cos theta + b2 sin theta,
  e.g. a0 = r l', a1 = -kappa r^2 l', b0 = -r r' on an arc axis.
  (The unit normal itself has complex singularities close to the real
  s-axis on wavy profiles; the area-weighted one is entire.)
* other panels: the plain Gauss-Legendre x trapezoidal rule (Eq. sx);
* plus 1/2 on the diagonal (jump relation, Eq. jump3).

Outer integral: the paper uses generalised Gaussian rules whose tables are
not available.  The oracle instead integrates adaptively: each near panel is
split at s_t (self panel) and mapped by s = s* + (e - s*) v^4 toward the
(near-)singular point s*; v in [0, 1] is bisected adaptively with a
vector-valued Gauss-Kronrod 7/15 pair until the estimated error is below
``tol`` times the largest entry.

Pins: tests/test_oracle_selfblock.py (Gauss identity at k = 0, sphere
eigenvalues of S and D, Mie series, interior point sources, circulant
structure on bodies of revolution) and
tests/test_oracle_selfblock_bruteforce.py (single entries on the self and
adjacent panels of a curved arc-axis body and of the paper's conch at
k = 3 and 10 against an independent adaptive 2-D cubature of the defining
integral, in extended precision, to 1e-12 of the row maximum).
"""
from __future__ import annotations

import heapq
import math

import numpy as np

from .geometry import BodyNodes
from .modal import (lagrange_weights, lagrange_weights_cos_theta, lagrange_weights_sin_theta,
                    modal_coeffs, ring_coords)

# Gauss-Kronrod 7/15 on [-1, 1]
_XK = np.array([-0.991455371120812639206854697526329, -0.949107912342758524526189684047851,
                -0.864864423359769072789712788640926, -0.741531185599394439863864773280788,
                -0.586087235467691130294144845693013, -0.405845151377397166906606412076961,
                -0.207784955007898467600689403773245, 0.0,
                0.207784955007898467600689403773245, 0.405845151377397166906606412076961,
                0.586087235467691130294144845693013, 0.741531185599394439863864773280788,
                0.864864423359769072789712788640926, 0.949107912342758524526189684047851,
                0.991455371120812639206854697526329])
_WK = np.array([0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                0.204432940075298892414161999234649, 0.209482141084727828012999174891714,
                0.204432940075298892414161999234649, 0.190350578064785409913256402421014,
                0.169004726639267902826583426598550, 0.140653259715525918745189590510238,
                0.104790010322250183839876322541518, 0.063092092629978553290700663189204,
                0.022935322010529224963732008058970])
_WG = np.zeros(15)
_WG[1::2] = [0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
             0.381830050505118944950369775488975, 0.417959183673469387755102040816327,
             0.381830050505118944950369775488975, 0.279705391489276667901467771423780,
             0.129484966168869693270611432679082]


def lagrange_basis(nodes: np.ndarray, s: float) -> np.ndarray:
    """P_l(s) for the Lagrange basis on ``nodes`` (Sec. 3.1)."""
    n = len(nodes)
    out = np.ones(n)
    for l in range(n):
        for m in range(n):
            if m != l:
                out[l] *= (s - nodes[m]) / (nodes[l] - nodes[m])
    return out


def _integrand(bn: BodyNodes, s_t: float, theta_t: float, h: float, pan_nodes, pan_jac,
               k: float, eta: float):
    """P_l(s) [F^D_j(s) + |J_lj| F^S_j(s)] at s = s_t + h for the body's own
    target (s_t, theta_t); ``pan_jac`` is |J| at the panel's nodes (order, n_theta)."""
    geom = bn.geom
    s = s_t + h
    r, dr, rt, c, alpha = geom.self_ring(s_t, theta_t, h)
    N = bn.n_theta // 2
    G, Gr, Gz = modal_coeffs(r, rt, c, k, N + 1, dr=dr)
    W0 = lagrange_weights(G[: N + 1], alpha, bn.n_theta)
    a0, a1, b0, b1, b2 = geom.area_normal(s)
    FD = a0 * lagrange_weights(Gr[: N + 1], alpha, bn.n_theta) + b0 * lagrange_weights(Gz[: N + 1], alpha, bn.n_theta)
    if a1 != 0.0:
        FD = FD + a1 * lagrange_weights_cos_theta(Gr, alpha, bn.n_theta)
    if b1 != 0.0:
        FD = FD + b1 * lagrange_weights_cos_theta(Gz, alpha, bn.n_theta)
    if b2 != 0.0:
        FD = FD + b2 * lagrange_weights_sin_theta(Gz, alpha, bn.n_theta)
    FS = -1j * eta * W0
    P = lagrange_basis(pan_nodes, s)
    return P[:, None] * (FD[None, :] + pan_jac * FS[None, :])


def _adaptive(fun, tol_rel: float, max_intervals: int = 500):
    """Integrate a vector function of v over [0, 1] by adaptive GK 7/15."""
    def rule(a, b):
        h = 0.5 * (b - a)
        vals = [fun(0.5 * (a + b) + h * x) for x in _XK]
        vals = np.stack(vals)
        k15 = h * np.tensordot(_WK, vals, axes=1)
        g7 = h * np.tensordot(_WG, vals, axes=1)
        # round-off floor of the pair: differences at the level of a few
        # hundred ulps of h * max|f| are rounding, not truncation
        floor = 200 * np.finfo(float).eps * abs(h) * float(np.max(np.abs(vals)))
        return k15, max(0.0, float(np.max(np.abs(k15 - g7))) - floor)

    heap = []
    total = 0
    for i in range(4):
        a, b = i / 4, (i + 1) / 4
        val, err = rule(a, b)
        heapq.heappush(heap, (-err, a, b, val))
    count = 4
    while True:
        total = sum(item[3] for item in heap)
        err = sum(-item[0] for item in heap)
        scale = float(np.max(np.abs(total))) + 1e-300
        if err <= tol_rel * scale or count >= max_intervals:
            return total
        e, a, b, val = heapq.heappop(heap)
        if b - a < 1e-6:
            # The double-layer pieces W^r, W^z each grow like 1/|s - s_t| and
            # cancel; their rounding leaves a noise floor of a few ulps per
            # dyadic interval in v.  Intervals this narrow carry a vanishing
            # part of the integral (~v^4 log v) and are not split further.
            heapq.heappush(heap, (0.0, a, b, val))
            count += 1
            continue
        m = 0.5 * (a + b)
        for (aa, bb) in ((a, m), (m, b)):
            val, er = rule(aa, bb)
            heapq.heappush(heap, (-er, aa, bb, val))
        count += 1


def pair_kernel(x, y, ny, k: float, eta: float):
    """Combined-layer smooth kernel d G/d n_y - i eta G (Eq. multi2part),
    x (..., 3) targets, y (..., 3) sources, ny their unit normals."""
    d = y - x
    rho = np.sqrt(np.sum(d * d, axis=-1))
    nd = np.sum(ny * d, axis=-1)
    g = np.exp(1j * k * rho) / (4 * np.pi * rho)
    return g * ((1j * k / rho - 1.0 / rho ** 2) * nd - 1j * eta)


def self_block_rows(bn: BodyNodes, rows, k: float, eta: float, tol: float = 1e-13):
    """Rows ``rows`` (body-local target indices) of the self block, (len(rows), n) complex."""
    n = bn.count
    nth, order = bn.n_theta, bn.order
    per_panel = order * nth
    out = np.zeros((len(rows), n), complex)
    for ri, t in enumerate(rows):
        p = t // per_panel
        s_t = bn.s[t // nth]
        theta_t = bn.theta[t % nth]
        for i in range(bn.n_panels):
            cols = slice(i * per_panel, (i + 1) * per_panel)
            if abs(i - p) > 1:
                out[ri, cols] = pair_kernel(bn.x[t], bn.x[cols], bn.n[cols], k, eta) * bn.w[cols]
                continue
            lo, hi = bn.breaks[i], bn.breaks[i + 1]
            pan_nodes = bn.s[i * order:(i + 1) * order]
            pan_jac = bn.jac[cols].reshape(order, nth)
            pieces = []
            if i == p:
                pieces = [(s_t, lo), (s_t, hi)]
            elif i < p:
                pieces = [(hi, lo)]
            else:
                pieces = [(lo, hi)]
            acc = np.zeros((order, nth), complex)
            for (s0, e) in pieces:
                L = e - s0
                h0 = s0 - s_t  # exactly 0 on the self panel

                def fun(v, h0=h0, L=L):
                    h = h0 + L * v ** 4
                    return _integrand(bn, s_t, theta_t, h, pan_nodes, pan_jac, k, eta) * (4 * abs(L) * v ** 3)

                acc += _adaptive(fun, tol)
            out[ri, cols] = acc.reshape(-1)
        out[ri, t] += 0.5
    return out


def _rows_job(args):
    bn, rows, k, eta, tol = args
    return self_block_rows(bn, rows, k, eta, tol)


def self_block_rows_parallel(bn: BodyNodes, rows, k: float, eta: float, tol: float = 1e-13,
                             workers: int = 0):
    """``self_block_rows`` over a spawn-started process pool (rows are independent)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os

    rows = list(rows)
    workers = workers or min(len(rows), os.cpu_count() or 1)
    if workers <= 1 or len(rows) < 2:
        return self_block_rows(bn, rows, k, eta, tol)
    chunks = [rows[i::workers] for i in range(workers)]
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_rows_job, [(bn, c, k, eta, tol) for c in chunks]))
    out = np.zeros((len(rows), bn.count), complex)
    for i, part in enumerate(parts):
        out[i::workers] = part
    return out


def self_block(bn: BodyNodes, k: float, eta: float, tol: float = 1e-13, workers: int = 0):
    """The full self block.  On a body of revolution (straight axis) the block
    is circulant in theta, so only one azimuth per generating-curve node is
    integrated and the rest follow by cyclic shifts."""
    n = bn.count
    nth = bn.n_theta
    if bn.geom.axisymmetric:
        base_rows = list(range(0, n, nth))
        base = self_block_rows_parallel(bn, base_rows, k, eta, tol, workers)
        A = np.zeros((n, n), complex)
        for a, t in enumerate(base_rows):
            row = base[a].reshape(-1, nth)
            for jt in range(nth):
                A[t + jt] = np.roll(row, jt, axis=1).reshape(-1)
        return A
    return self_block_rows_parallel(bn, list(range(n)), k, eta, tol, workers)
