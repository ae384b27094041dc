"""Brute-force pin of the oracle self block on curved bodies at k != 0.

Every near-panel entry of the self block (Sec. 3.1, product integration
against the tensor Lagrange interpolant; Sec. 3.2-3.4 evaluate it with modal
Green's functions and a graded outer rule) is a plain double integral over
the panel's parameter rectangle:

    A[t, (i,l,j)] = 1/2 delta + int int P_l(s) L_j(theta)
                    [ dG/dn_y(x_t, y) |J|(s,theta) - i eta |J|_{lj} G(x_t, y) ] ds dtheta,

G = e^{ik rho}/(4 pi rho), the double layer against the interpolant of mu and
the single layer against the interpolant of mu |J| (the reading of the
oracle header).  Here that integral is evaluated directly, with none of the
oracle's machinery: the surface map is sampled, the area-weighted normal
|J| n = d_theta y x d_s y is taken by eighth-order central differences of
the map, and the rectangle is integrated by adaptive cubature: cells are
bisected along their longer side until a 12-point against 8-point tensor
Gauss-Legendre estimate is below 1e-13 of the largest entry.  The cells that
have the target's parameters (s_t, theta_t) at a corner are cut along the
diagonal into two triangles, each mapped to the unit square by Duffy's
transformation (M. G. Duffy, SIAM J. Numer. Anal. 19, 1982), whose Jacobian
vanishes at the target and cancels the 1/rho singularity.

A slip confined to the curvature (kappa) terms of the area-weighted normal,
to the cos/sin theta terms of the paper's horizontal-ring shapes, or to the
k != 0 modal derivative kernels changes these entries at O(1e-3) or more and
fails here.
"""
import numpy as np
import pytest

import scenes
from oracle.geometry import body_nodes
from oracle.selfblock import self_block_rows

CURVED = dict(base_radius=0.5, mode_cos=(0.06, 0.03), mode_sin=(0.04,), axis_length=1.0, curvature=0.35)

LD = np.longdouble
PI_LD = LD("3.14159265358979323846264338327950288")
# eighth-order central first difference: f' ~ sum_k c_k (f(x+kh) - f(x-kh)) / h
_FD = ((1, LD(4) / 5), (2, LD(-1) / 5), (3, LD(4) / 105), (4, LD(-1) / 280))
_H = LD("1e-3")


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _lagrange_poly(nodes, s):
    """P_l(s) for every node l (Lagrange basis on the panel's GL nodes), (..., n)."""
    s = np.asarray(s, float)
    out = np.ones(s.shape + (len(nodes),))
    for l in range(len(nodes)):
        for m in range(len(nodes)):
            if m != l:
                out[..., l] *= (s - nodes[m]) / (nodes[l] - nodes[m])
    return out


def _lagrange_trig(n_theta, th):
    """L_j(theta) = (1/2N)[1 + 2 sum_{m<N} cos m(theta - theta_j) + cos N(theta - theta_j)]
    (Sec. 3.1, the symmetric reading of the Nyquist term), (..., 2N)."""
    N = n_theta // 2
    d = np.asarray(th, float)[..., None] - 2 * np.pi * np.arange(n_theta) / n_theta
    out = np.ones_like(d)
    for m in range(1, N):
        out += 2.0 * np.cos(m * d)
    out += np.cos(N * d)
    return out / n_theta


def surface(body, s, th):
    """The body's reference surface y(s, theta) in extended precision, written
    from the descriptor alone (Eq. para_quasi on an arc axis; Eqs. quasiwave
    and geometries for the paper's horizontal-ring shapes)."""
    s = np.asarray(s, LD)
    th = np.asarray(th, LD)
    if body.kind == 1:
        def series(part):
            f = np.zeros_like(s)
            for om, A, B in part:
                f = f + LD(A) * np.cos(LD(om) * s) + LD(B) * np.sin(LD(om) * s)
            return f
        xc, yc, z, r = (series(p) for p in body.series)
        return np.stack([xc + r * np.cos(th), yc + r * np.sin(th), z], -1)
    u = (1 + np.sin(s)) / 2
    rho = np.ones_like(s)
    for m, a in enumerate(body.mode_cos, start=1):
        rho = rho + LD(a) * np.cos(2 * PI_LD * m * u)
    for m, b in enumerate(body.mode_sin, start=1):
        rho = rho + LD(b) * np.sin(2 * PI_LD * m * u)
    r = LD(body.base_radius) * rho * np.cos(s)
    l = LD(body.axis_length) / 2 * np.sin(s)
    kap = LD(body.curvature)
    zero = np.zeros_like(s)
    if kap == 0:
        g = np.stack([zero, zero, l], -1)
        e1 = np.stack([np.ones_like(s), zero, zero], -1)
    else:
        g = np.stack([(1 - np.cos(kap * l)) / kap, zero, np.sin(kap * l) / kap], -1)
        e1 = np.stack([np.cos(kap * l), zero, -np.sin(kap * l)], -1)
    e2 = np.stack([zero, np.ones_like(s), zero], -1)
    return g + r[..., None] * (np.cos(th)[..., None] * e1 + np.sin(th)[..., None] * e2)


def _tangents(body, s, th):
    s = np.asarray(s, LD)
    th = np.asarray(th, LD)
    ds = sum(c * (surface(body, s + k * _H, th) - surface(body, s - k * _H, th)) for k, c in _FD) / _H
    dt = sum(c * (surface(body, s, th + k * _H) - surface(body, s, th - k * _H)) for k, c in _FD) / _H
    return ds, dt


def _area_normal(body, s, th):
    """|J| n = d_theta y x d_s y (outward for both families)."""
    ds, dt = _tangents(body, s, th)
    return np.cross(dt, ds)


def _metric(body, s, th):
    """|d_s y| and |d_theta y| at one parameter point."""
    ds, dt = _tangents(body, np.array([s]), np.array([th]))
    return float(np.linalg.norm(ds.astype(float))), float(np.linalg.norm(dt.astype(float)))


def _integrand_terms(body, x_t, s, th):
    """rho and (|J| n).(y - x_t) at the points (s, th); y - x_t and the dot
    product in extended precision (the latter is O(rho^2) by cancellation)."""
    y = surface(body, s, th)
    Na = _area_normal(body, s, th)
    d = y - x_t
    rho = np.sqrt(np.sum(d * d, axis=-1))
    return rho.astype(float), np.sum(Na * d, axis=-1).astype(float)


_FAN = 4


def _quads(cells, n):
    """Tensor Gauss points of every cell, n x n per quadrilateral: a regular
    cell is one quadrilateral, a cell with the target at its corner (s0, t0)
    is cut along its diagonal into two triangles, each cut again into _FAN
    narrow triangles with the target as common vertex, each mapped to the
    unit square by Duffy's transformation (the Jacobian factor u vanishes at
    the target).  Returns s, t, weights (n_quads, n*n) and the owning cell."""
    g, w = _gl(n)
    ww = (w[:, None] * w[None, :]).ravel()
    u = np.repeat(g, n)   # first index of the tensor grid
    v = np.tile(g, n)
    S, T, W, owner = [], [], [], []
    for ci, (s0, s1, t0, t1, sing) in enumerate(cells):
        a, b = s1 - s0, t1 - t0
        if not sing:
            S.append(s0 + a * u); T.append(t0 + b * v); W.append(abs(a * b) * ww); owner.append(ci)
            continue
        # four narrow triangles along each far edge: on a skewed parametrisation
        # (the paper's shapes) the angular dependence is then resolved quickly
        for (e1s, e1t), (e2s, e2t) in (((a, 0.0), (a, b)), ((a, b), (0.0, b))):
            for f in range(_FAN):
                p1s, p1t = e1s + (e2s - e1s) * f / _FAN, e1t + (e2t - e1t) * f / _FAN
                p2s, p2t = e1s + (e2s - e1s) * (f + 1) / _FAN, e1t + (e2t - e1t) * (f + 1) / _FAN
                det = abs(p1s * p2t - p1t * p2s)
                S.append(s0 + u * (p1s + v * (p2s - p1s)))
                T.append(t0 + u * (p1t + v * (p2t - p1t)))
                W.append(det * u * ww)
                owner.append(ci)
    return np.array(S), np.array(T), np.array(W), np.array(owner)


def _cells_rule(body, nth, x_t, k, pan_nodes, cells, n):
    """Integrals of P_l L_j dG/dn |J| and P_l L_j G over every cell with n x n
    Gauss points per quadrilateral, (n_cells, order, n_theta) each."""
    S, T, W, owner = _quads(cells, n)
    shp = S.shape
    rho, nd = _integrand_terms(body, x_t, S.ravel(), T.ravel())
    rho, nd = rho.reshape(shp), nd.reshape(shp)
    eikr = np.exp(1j * k * rho)
    G = W * eikr / (4 * np.pi * rho)
    dGdn = W * nd * eikr * (1j * k * rho - 1.0) / (4 * np.pi * rho ** 3)
    P = _lagrange_poly(pan_nodes, S)          # (q, p, order)
    L = _lagrange_trig(nth, T)                # (q, p, nth)
    qD = np.einsum("qp,qpl,qpj->qlj", dGdn, P, L)
    qS = np.einsum("qp,qpl,qpj->qlj", G, P, L)
    nc = len(cells)
    ID = np.zeros((nc,) + qD.shape[1:], complex)
    IS = np.zeros_like(ID)
    np.add.at(ID, owner, qD)
    np.add.at(IS, owner, qS)
    return ID, IS


def _nodes(body):
    """Panel breakpoints and Gauss-Legendre nodes in s (Sec. 3.1), own code."""
    npan, order = body.n_panels, body.order
    br = np.asarray(body.panel_breaks, float) if len(body.panel_breaks) else \
        np.linspace(-np.pi / 2, np.pi / 2, npan + 1)
    x, _ = np.polynomial.legendre.leggauss(order)
    s = np.concatenate([0.5 * (br[i] + br[i + 1]) + 0.5 * (br[i + 1] - br[i]) * x for i in range(npan)])
    return br, s


def brute_panel(body, t, panel, k, eta, tol=1e-12, max_cells=3000, rules=(10, 16)):
    """Row t (body-local node index, order panel -> GL node -> azimuth) of the
    self block restricted to the columns of ``panel``: the defining double
    integral over the panel's rectangle [lo, hi] x [theta_t - pi, theta_t + pi]
    by adaptive cubature.  A cell is accepted when the estimate |I_16 - I_10|
    (tensor Gauss 16 against 10 points) is below tol times the largest entry
    times its share of the rectangle's area (shares below 1/100 count as
    1/100), or at the rounding level of its own value; the others are
    bisected along their longer side in surface length (|d_s y| ds against
    |d_theta y| dtheta at the target).  Returns (entries, summed estimate
    relative to the largest entry)."""
    order, nth = body.order, body.n_theta
    br, snodes = _nodes(body)
    s_t = snodes[t // nth]
    th_t = 2 * np.pi * (t % nth) / nth
    x_t = surface(body, np.array([s_t]), np.array([th_t]))[0]
    lo, hi = br[panel], br[panel + 1]
    pan_nodes = snodes[panel * order:(panel + 1) * order]
    area = (hi - lo) * 2 * np.pi
    ms, mt = _metric(body, s_t, th_t)
    # cells (s0, s1, t0, t1, singular): a singular cell has the target at (s0, t0)
    if lo < s_t < hi:
        cells = [(s_t, s1, th_t, t1, True) for s1 in (lo, hi) for t1 in (th_t - np.pi, th_t + np.pi)]
    else:
        cells = [(lo, hi, th_t - np.pi, th_t + np.pi, False)]
    done_D = np.zeros((order, nth), complex)
    done_S = np.zeros((order, nth), complex)
    scale, est = None, 0.0
    while cells:
        lowD, lowS = _cells_rule(body, nth, x_t, k, pan_nodes, cells, rules[0])
        hiD, hiS = _cells_rule(body, nth, x_t, k, pan_nodes, cells, rules[1])
        nc = len(cells)
        err = np.maximum(np.abs(hiD - lowD).reshape(nc, -1).max(1), np.abs(hiS - lowS).reshape(nc, -1).max(1))
        mag = np.maximum(np.abs(hiD).reshape(nc, -1).max(1), np.abs(hiS).reshape(nc, -1).max(1))
        if scale is None:
            scale = max(np.abs(hiD.sum(0)).max(), np.abs(hiS.sum(0)).max())
        frac = np.maximum(1e-2, np.array([abs((c[1] - c[0]) * (c[3] - c[2])) / area for c in cells]))
        ok = (err <= tol * scale * frac) | (err <= 1e-15 * mag)
        if nc > max_cells:
            ok[:] = True
        done_D += hiD[ok].sum(0)
        done_S += hiS[ok].sum(0)
        est += err[ok].sum()
        nxt = []
        for c, good in zip(cells, ok):
            if good:
                continue
            s0, s1, t0, t1, sing = c
            if abs(s1 - s0) * ms >= abs(t1 - t0) * mt:
                sm = 0.5 * (s0 + s1)
                nxt += [(s0, sm, t0, t1, sing), (sm, s1, t0, t1, False)]
            else:
                tm = 0.5 * (t0 + t1)
                nxt += [(s0, s1, t0, tm, sing), (s0, s1, tm, t1, False)]
        cells = nxt
    # |J| at the panel's nodes for the single layer's interpolant of mu |J|
    S, T = np.meshgrid(pan_nodes, 2 * np.pi * np.arange(nth) / nth, indexing="ij")
    jac = np.linalg.norm(_area_normal(body, S, T).astype(float), axis=-1)
    out = (done_D - 1j * eta * jac * done_S).reshape(-1)
    col = t - panel * order * nth
    if 0 <= col < order * nth:
        out[col] += 0.5
    return out, est / scale


def _check(body, rows, k, eta):
    bn = body_nodes(body)
    A = self_block_rows(bn, rows, k, eta, tol=1e-13)
    per = bn.order * bn.n_theta
    for ri, t in enumerate(rows):
        p = t // per
        scale = np.max(np.abs(A[ri]))
        for panel in sorted({p, max(0, p - 1), min(bn.n_panels - 1, p + 1)}):
            ref, est = brute_panel(body, t, panel, k, eta)
            assert est < 1e-11
            oracle = A[ri, panel * per:(panel + 1) * per]
            err = np.max(np.abs(oracle - ref)) / scale
            assert err < 1e-12, (t, panel, err)


@pytest.mark.parametrize("k", [3.0, 10.0])
def test_arc_axis_body_entries_against_brute_force(k):
    """Curved axis (kappa = 0.35) with two profile modes: the kappa-dependent
    part of |J| n_r and the k != 0 derivative kernels."""
    body = scenes.Body(2, 6, 12, **CURVED)
    per = body.order * body.n_theta
    # a mid-panel node, the node next to the shared panel edge, a node of panel 1
    rows = [2 * body.n_theta + 3, (body.order - 1) * body.n_theta + 7, per + 2 * body.n_theta + 10]
    _check(body, rows, k, 1.0)


@pytest.mark.parametrize("k", [3.0, 10.0])
def test_conch_entries_against_brute_force(k):
    """The paper's conch (Eq. geometries, scaled by 0.5): moving ring centres
    give the b1 cos theta and b2 sin theta terms of |J| n_3."""
    body = scenes.conch(2, 6, 12, scale=0.5)
    per = body.order * body.n_theta
    rows = [3 * body.n_theta + 1, (body.order - 1) * body.n_theta + 5, per + body.n_theta + 9]
    _check(body, rows, k, 1.0)


def test_brute_force_geometry_matches_the_nodes():
    """The brute force's own surface map and area-weighted normal reproduce the
    node table (positions, |J|, outward normals) of both families."""
    for body in (scenes.Body(2, 6, 12, **CURVED), scenes.conch(2, 6, 12, scale=0.5)):
        bn = body_nodes(body)
        S, T = np.meshgrid(bn.s, bn.theta, indexing="ij")
        y = surface(body, S, T).astype(float).reshape(-1, 3)
        Na = _area_normal(body, S, T).astype(float).reshape(-1, 3)
        J = np.linalg.norm(Na, axis=-1)
        assert np.max(np.abs(bn.geom.to_world(y) - bn.x)) < 1e-14
        assert np.max(np.abs(J - bn.jac)) < 1e-13 * np.max(bn.jac)
        assert np.max(np.abs((Na / J[:, None]) @ bn.geom.R.T - bn.n)) < 1e-12


@pytest.mark.parametrize("shape,term", [("arc", 1), ("conch", 4)])
def test_planted_normal_slip_is_caught(monkeypatch, shape, term):
    """A sign slip planted in the oracle's area-weighted normal -- the kappa
    term a1 of |J| n_r on the arc axis, the sin theta term b2 of |J| n_3 on
    the conch -- moves the oracle's entries far outside the brute-force
    tolerance."""
    from oracle import geometry as og
    body = scenes.Body(2, 6, 12, **CURVED) if shape == "arc" else scenes.conch(2, 6, 12, scale=0.5)
    cls = og.BodyGeom if shape == "arc" else og.RingGeom
    orig = cls.area_normal

    def slipped(self, s):
        c = list(orig(self, s))
        c[term] = -c[term]
        return tuple(c)

    monkeypatch.setattr(cls, "area_normal", slipped)
    bn = body_nodes(body)
    t = 2 * body.n_theta + 3
    A = self_block_rows(bn, [t], 3.0, 1.0, tol=1e-13)[0, :body.order * body.n_theta]
    ref, _ = brute_panel(body, t, 0, 3.0, 1.0)
    assert np.max(np.abs(A - ref)) / np.max(np.abs(ref)) > 1e-4
