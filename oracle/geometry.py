"""Oracle geometry and Nystrom nodes (test infrastructure only).

Surface (Eq. para_quasi, generalised to a planar-arc axis with a
rotation-minimising frame e1, e2, e3):

    y(s, theta) = gamma(l(s)) + r(s) (cos theta e1 + sin theta e2),
    s in [-pi/2, pi/2],  u = (1 + sin s)/2,  l = L (u - 1/2),
    r(s) = rho(u) cos s  (closed at both poles, like the paper's shapes).

Tangents d_s, d_theta and |J| = |d_s x d_theta| (Sec. 3.1);
outward normal n = n_r e_r + n_3 e3 (n . e_theta = 0, Sec. 3.2).
Nodes: N_p uniform panels in s with N_order Gauss-Legendre nodes each, times
2N equispaced theta_j = j pi / N; weight |J| (pi/N) omega (Eq. sx).

Second family (``kind`` 1, the paper's own shapes, Eqs. quasiwave and
geometries): horizontal rings with a moving centre,

    y(s, theta) = (x_c(s) + r(s) cos theta, y_c(s) + r(s) sin theta, z(s)),

each of x_c, y_c, z, r a finite sum A cos(omega s) + B sin(omega s); the
frame is fixed (e1, e2, e3 = x, y, z).  Here d_s has an e_theta part, which
d_theta x d_s drops, so again n = n_r e_r + n_3 e3.

Both families have an area-weighted normal that is a trigonometric
polynomial of degree one in theta,
    |J| n_r = a0 + a1 cos theta,   |J| n_3 = b0 + b1 cos theta + b2 sin theta,
returned per ring by ``area_normal``.

Panels: uniform in s, or the breakpoints given in ``panel_breaks`` (dyadic
refinement toward the poles, Sec. 6.1).

Pins: tests/test_oracle_operator.py and tests/test_oracle_shapes.py (sphere area,
Gauss-Legendre exactness, divergence theorem on curved bodies and on the
paper's shapes (volumes by Cavalieri's principle), orientation, the
difference formulas of ``self_ring`` against 50-digit arithmetic).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def gauss_legendre(n: int):
    """Nodes and weights on [-1, 1] by Newton's method on P_n (own code)."""
    x = np.cos(np.pi * (np.arange(1, n + 1) - 0.25) / (n + 0.5))
    for _ in range(100):
        p0, p1 = np.ones_like(x), x.copy()
        for j in range(2, n + 1):
            p0, p1 = p1, ((2 * j - 1) * x * p1 - (j - 1) * p0) / j
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0, p1 = np.ones_like(x), x.copy()
    for j in range(2, n + 1):
        p0, p1 = p1, ((2 * j - 1) * x * p1 - (j - 1) * p0) / j
    dp = n * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


@dataclass
class BodyGeom:
    """Evaluates the reference shape of one body and maps it to world space."""

    base: float
    a: np.ndarray
    b: np.ndarray
    L: float
    kappa: float
    R: np.ndarray  # 3x3
    c: np.ndarray  # 3

    @classmethod
    def from_desc(cls, d) -> "BodyGeom":
        return cls(float(d.base_radius), np.asarray(d.mode_cos, float), np.asarray(d.mode_sin, float),
                   float(d.axis_length), float(d.curvature),
                   np.asarray(d.rotation, float).reshape(3, 3), np.asarray(d.center, float))

    # profile rho(u) and rho'(u)
    def rho(self, u):
        u = np.asarray(u, float)
        out = np.ones_like(u)
        for m, am in enumerate(self.a, start=1):
            out = out + am * np.cos(2 * np.pi * m * u)
        for m, bm in enumerate(self.b, start=1):
            out = out + bm * np.sin(2 * np.pi * m * u)
        return self.base * out

    def drho(self, u):
        u = np.asarray(u, float)
        out = np.zeros_like(u)
        for m, am in enumerate(self.a, start=1):
            out = out - am * 2 * np.pi * m * np.sin(2 * np.pi * m * u)
        for m, bm in enumerate(self.b, start=1):
            out = out + bm * 2 * np.pi * m * np.cos(2 * np.pi * m * u)
        return self.base * out

    def ring(self, s):
        """Per generating-curve parameter s (local frame): gamma, e1, e2, e3,
        r, r', l' -- everything the ring at s needs."""
        s = np.asarray(s, float)
        u = 0.5 * (1.0 + np.sin(s))
        du = 0.5 * np.cos(s)
        rr = self.rho(u) * np.cos(s)
        dr = self.drho(u) * du * np.cos(s) - self.rho(u) * np.sin(s)
        l = 0.5 * self.L * np.sin(s)
        dl = 0.5 * self.L * np.cos(s)
        k = self.kappa
        kl = k * l
        # gamma = ((1 - cos kl)/k, 0, sin(kl)/k), written without cancellation
        half = 0.5 * kl
        sinc_half = np.where(np.abs(half) > 1e-8, np.sin(half) / np.where(half == 0, 1, half), 1.0)
        sinc_full = np.where(np.abs(kl) > 1e-8, np.sin(kl) / np.where(kl == 0, 1, kl), 1.0)
        gx = 0.5 * k * l * l * sinc_half ** 2
        gz = l * sinc_full
        zero = np.zeros_like(s)
        gamma = np.stack([gx, zero, gz], -1)
        e1 = np.stack([np.cos(kl), zero, -np.sin(kl)], -1)
        e2 = np.stack([zero, np.ones_like(s), zero], -1)
        e3 = np.stack([np.sin(kl), zero, np.cos(kl)], -1)
        return dict(gamma=gamma, e1=e1, e2=e2, e3=e3, r=rr, dr=dr, dl=dl)

    def normal_parts(self, s, theta):
        """n_r, n_3 and |J| at (s, theta): d_s = A e3 + B e_r with
        A = l'(1 - kappa r cos theta), B = r';  n = (A e_r - B e3)/|.|,  |J| = r |.|."""
        g = self.ring(s)
        A = g["dl"] * (1.0 - self.kappa * g["r"] * np.cos(theta))
        B = g["dr"]
        h = np.sqrt(A * A + B * B)
        return A / h, -B / h, g["r"] * h

    def area_normal(self, s):
        """(a0, a1, b0, b1, b2) of |J| n_r = r l' (1 - kappa r cos theta),
        |J| n_3 = -r r' at generating-curve parameter s."""
        g = self.ring(np.array([s], float))
        r, dr, dl = (float(np.asarray(g[kk]).reshape(-1)[0]) for kk in ("r", "dr", "dl"))
        return r * dl, -self.kappa * r * r * dl, -r * dr, 0.0, 0.0

    @property
    def axisymmetric(self) -> bool:
        return self.kappa == 0.0

    def local_points(self, s, theta):
        g = self.ring(s)
        er = np.cos(theta)[..., None] * g["e1"] + np.sin(theta)[..., None] * g["e2"]
        return g["gamma"] + g["r"][..., None] * er

    def local_normals(self, s, theta):
        g = self.ring(s)
        er = np.cos(theta)[..., None] * g["e1"] + np.sin(theta)[..., None] * g["e2"]
        nr, n3, _ = self.normal_parts(s, theta)
        return nr[..., None] * er + n3[..., None] * g["e3"]

    def self_ring(self, s_t: float, theta_t: float, h: float):
        """Ring at s = s_t + h seen from the body's own node (s_t, theta_t).

        Returns r(s), dr = r - r~, r~, c and alpha (Sec. 3.3 notation) from
        difference formulas in h (sum-to-product identities), so that r - r~
        and c keep full relative precision as h -> 0.  With Delta = l_t - l,
        the target in the frame at l is
            a = (1 - cos k Delta)/k + r_t cos theta_t cos k Delta,
            b = r_t sin theta_t,
            c = sin(k Delta)/k - r_t cos theta_t sin k Delta.
        """
        s = s_t + h
        sh = math.sin(0.5 * h)
        mid = s_t + 0.5 * h
        u_t = 0.5 * (1.0 + math.sin(s_t))
        u = 0.5 * (1.0 + math.sin(s))
        du = math.cos(mid) * sh  # u - u_t
        # rho(u) - rho(u_t)
        drho = 0.0
        for m, am in enumerate(self.a, start=1):
            drho += am * (-2.0 * math.sin(math.pi * m * (u + u_t)) * math.sin(math.pi * m * du))
        for m, bm in enumerate(self.b, start=1):
            drho += bm * (2.0 * math.cos(math.pi * m * (u + u_t)) * math.sin(math.pi * m * du))
        drho *= self.base
        rho_t = float(self.rho(u_t))
        r_t = rho_t * math.cos(s_t)
        r = float(self.rho(u)) * math.cos(s)
        dr_t = drho * math.cos(s) + rho_t * (-2.0 * math.sin(mid) * sh)  # r - r_t
        Delta = -self.L * math.cos(mid) * sh
        kd = self.kappa * Delta
        sinc_h = math.sin(0.5 * kd) / (0.5 * kd) if abs(kd) > 1e-8 else 1.0
        sinc_f = math.sin(kd) / kd if abs(kd) > 1e-8 else 1.0
        omc_k = 0.5 * self.kappa * Delta * Delta * sinc_h ** 2  # (1 - cos k Delta)/k
        ck, sk = math.cos(kd), math.sin(kd)
        ct, st = math.cos(theta_t), math.sin(theta_t)
        a = omc_k + r_t * ct * ck
        b = r_t * st
        c = Delta * sinc_f - r_t * ct * sk
        rt = math.hypot(a, b)
        d2 = -(r_t * ct * sk) ** 2 + 2.0 * r_t * ct * ck * omc_k + omc_k ** 2  # r~^2 - r_t^2
        dr = dr_t - d2 / (rt + r_t)
        return r, dr, rt, c, math.atan2(b, a)

    def to_world(self, p):
        return p @ self.R.T + self.c

    def to_local(self, x):
        return (np.asarray(x) - self.c) @ self.R


def _series(terms, s):
    """sum A cos(omega s) + B sin(omega s) and its derivative in s."""
    s = np.asarray(s, float)
    f = np.zeros_like(s)
    df = np.zeros_like(s)
    for om, A, B in terms:
        c, sn = np.cos(om * s), np.sin(om * s)
        f = f + A * c + B * sn
        df = df + om * (B * c - A * sn)
    return f, df


def _series_drop(terms, s_t: float, h: float) -> float:
    """f(s_t) - f(s_t + h) by sum-to-product, exact in relative terms as h -> 0:
    cos w s_t - cos w s = 2 sin(w m) sin(w h/2), sin w s_t - sin w s = -2 cos(w m) sin(w h/2),
    m = s_t + h/2."""
    m = s_t + 0.5 * h
    out = 0.0
    for om, A, B in terms:
        sh = math.sin(0.5 * om * h)
        out += 2.0 * sh * (A * math.sin(om * m) - B * math.cos(om * m))
    return out


@dataclass
class RingGeom:
    """Horizontal rings of radius r(s) centred at (x_c(s), y_c(s), z(s))."""

    terms: tuple   # four lists of (omega, A, B): x_c, y_c, z, r
    R: np.ndarray
    c: np.ndarray

    @classmethod
    def from_desc(cls, d) -> "RingGeom":
        terms = tuple([tuple(map(float, t)) for t in part] for part in d.series)
        assert len(terms) == 4
        return cls(terms, np.asarray(d.rotation, float).reshape(3, 3), np.asarray(d.center, float))

    @property
    def axisymmetric(self) -> bool:
        return all(A == 0.0 and B == 0.0 for part in self.terms[:2] for (_, A, B) in part)

    def ring(self, s):
        s = np.asarray(s, float)
        xc, dxc = _series(self.terms[0], s)
        yc, dyc = _series(self.terms[1], s)
        z, dz = _series(self.terms[2], s)
        r, dr = _series(self.terms[3], s)
        zero, one = np.zeros_like(s), np.ones_like(s)
        return dict(gamma=np.stack([xc, yc, z], -1), e1=np.stack([one, zero, zero], -1),
                    e2=np.stack([zero, one, zero], -1), e3=np.stack([zero, zero, one], -1),
                    r=r, dr=dr, dz=dz, dxc=dxc, dyc=dyc)

    def normal_parts(self, s, theta):
        """d_s = A e3 + B e_r + (.) e_theta, A = z', B = r' + x_c' cos theta + y_c' sin theta;
        n = (A e_r - B e3)/|.|, |J| = r |.|."""
        g = self.ring(s)
        A = g["dz"] + 0.0 * np.asarray(theta, float)
        B = g["dr"] + g["dxc"] * np.cos(theta) + g["dyc"] * np.sin(theta)
        h = np.sqrt(A * A + B * B)
        return A / h, -B / h, g["r"] * h

    def area_normal(self, s):
        """(a0, a1, b0, b1, b2): |J| n_r = r z', |J| n_3 = -r (r' + x_c' cos theta + y_c' sin theta)."""
        g = self.ring(np.array([s], float))
        v = {kk: float(np.asarray(g[kk]).reshape(-1)[0]) for kk in ("r", "dr", "dz", "dxc", "dyc")}
        r = v["r"]
        return r * v["dz"], 0.0, -r * v["dr"], -r * v["dxc"], -r * v["dyc"]

    def self_ring(self, s_t: float, theta_t: float, h: float):
        """Ring at s = s_t + h seen from the body's own node (s_t, theta_t):
        r(s), r - r~, r~, c, alpha with the centre and radius differences taken
        by sum-to-product, so they keep relative precision as h -> 0:
            a = r_t cos theta_t + dx,  b = r_t sin theta_t + dy,  c = z(s_t) - z(s),
            r~ - r_t = (2 r_t (cos theta_t dx + sin theta_t dy) + dx^2 + dy^2)/(r~ + r_t),
        dx, dy the drops of x_c, y_c from s_t to s."""
        s = s_t + h
        r_t = float(_series(self.terms[3], s_t)[0])
        r = float(_series(self.terms[3], s)[0])
        dx = _series_drop(self.terms[0], s_t, h)
        dy = _series_drop(self.terms[1], s_t, h)
        c = _series_drop(self.terms[2], s_t, h)
        ct, st = math.cos(theta_t), math.sin(theta_t)
        a = r_t * ct + dx
        b = r_t * st + dy
        rt = math.hypot(a, b)
        drt = (2.0 * r_t * (ct * dx + st * dy) + dx * dx + dy * dy) / (rt + r_t)  # r~ - r_t
        dr = -_series_drop(self.terms[3], s_t, h) - drt
        return r, dr, rt, c, math.atan2(b, a)

    local_points = BodyGeom.local_points
    local_normals = BodyGeom.local_normals
    to_world = BodyGeom.to_world
    to_local = BodyGeom.to_local


@dataclass
class BodyNodes:
    geom: BodyGeom
    n_panels: int
    order: int
    n_theta: int
    breaks: np.ndarray      # panel breakpoints in s
    s: np.ndarray           # (n_panels*order,) node parameters, panel-major
    omega: np.ndarray       # GL weights scaled to the panels
    theta: np.ndarray       # (n_theta,)
    x: np.ndarray           # (n, 3) world positions, order panel -> l -> j
    n: np.ndarray           # (n, 3) world normals
    jac: np.ndarray         # (n,) |J|
    w: np.ndarray           # (n,) |J| (pi/N) omega

    @property
    def count(self):
        return self.x.shape[0]


def geometry(desc):
    """The geometry object of a body descriptor (``kind`` 0: arc axis, 1: horizontal rings)."""
    return RingGeom.from_desc(desc) if getattr(desc, "kind", 0) == 1 else BodyGeom.from_desc(desc)


def panel_breaks(desc) -> np.ndarray:
    """Panel breakpoints in s: ``panel_breaks`` when given, else uniform."""
    npan = desc.n_panels
    br = np.asarray(getattr(desc, "panel_breaks", ()) or (), float)
    if br.size == 0:
        return np.linspace(-np.pi / 2, np.pi / 2, npan + 1)
    assert br.size == npan + 1 and np.all(np.diff(br) > 0)
    assert abs(br[0] + np.pi / 2) < 1e-15 and abs(br[-1] - np.pi / 2) < 1e-15
    return br


def body_nodes(desc) -> BodyNodes:
    g = geometry(desc)
    npan, order, nth = desc.n_panels, desc.order, desc.n_theta
    xg, wg = gauss_legendre(order)
    breaks = panel_breaks(desc)
    s = np.concatenate([0.5 * (breaks[i] + breaks[i + 1]) + 0.5 * (breaks[i + 1] - breaks[i]) * xg
                        for i in range(npan)])
    om = np.concatenate([0.5 * (breaks[i + 1] - breaks[i]) * wg for i in range(npan)])
    theta = 2 * np.pi * np.arange(nth) / nth
    S, T = np.meshgrid(s, theta, indexing="ij")
    xl = g.local_points(S, T).reshape(-1, 3)
    nl = g.local_normals(S, T).reshape(-1, 3)
    _, _, jac = g.normal_parts(S, T)
    jac = jac.reshape(-1)
    w = jac * (2 * np.pi / nth) * np.repeat(om, nth)
    return BodyNodes(g, npan, order, nth, breaks, s, om, theta,
                     g.to_world(xl), nl @ g.R.T, jac, w)


def scene_nodes(scene):
    """All bodies' nodes, concatenated in body order."""
    return [body_nodes(b) for b in scene.bodies]
