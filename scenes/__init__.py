"""Seeded synthetic scenes: body descriptors, wavenumbers and incident directions.

This module only draws and tabulates the *inputs* of a multiple-scattering
problem.  It contains none of the method's arithmetic (no geometry
evaluation, no quadrature, no kernels): both the FP64 oracle and the CUDA
library receive the same descriptors and build everything else themselves.

A body is a rigid motion x = R x0 + c (Section 6.5, random arrays) of a
quasi-axisymmetric reference shape (Eq. para_quasi) generalised to a curved
axis.  The reference shape is described by

* ``base_radius`` and Fourier coefficients ``mode_cos``/``mode_sin`` of the
  profile rho(u) = base * (1 + sum_m a_m cos 2 pi m u + b_m sin 2 pi m u),
  u in [0, 1] the normalised axial coordinate;
* ``axis_length`` L and ``curvature`` kappa of a planar circular-arc axis;
* the discretisation: ``n_panels`` Gauss-Legendre panels of ``order`` nodes
  along the generating curve and ``n_theta`` = 2N azimuthal points
  (Section 3.1).

A body of ``kind`` 1 is one of the paper's own shapes (Eqs. quasiwave and
geometries): horizontal rings y = (x_c + r cos theta, y_c + r sin theta, z),
each of x_c, y_c, z, r given in ``series`` as (omega, A, B) triples of
A cos(omega s) + B sin(omega s), s in [-pi/2, pi/2].

``panel_breaks`` (optional) replaces the uniform panels, e.g. by dyadic
refinement toward the poles (Sec. 6.1, N_ref levels).

Seeds follow ``31380 + 1000 * config + request_id``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

MAX_MODES = 8


@dataclasses.dataclass
class Body:
    n_panels: int
    order: int
    n_theta: int
    base_radius: float = 0.5
    mode_cos: Sequence[float] = ()
    mode_sin: Sequence[float] = ()
    axis_length: float = 1.0
    curvature: float = 0.0
    rotation: Sequence[float] = (1, 0, 0, 0, 1, 0, 0, 0, 1)  # row-major 3x3
    center: Sequence[float] = (0.0, 0.0, 0.0)
    kind: int = 0
    series: Sequence = ()          # kind 1: ((omega, A, B), ...) for x_c, y_c, z, r
    panel_breaks: Sequence[float] = ()

    @property
    def n_nodes(self) -> int:
        return self.n_panels * self.order * self.n_theta

    def bound_radius(self) -> float:
        """Conservative radius of a ball about ``center`` that holds the body.

        Arc axis: |gamma(l)| <= |l| <= L/2 and r <= rho <= base*(1+sum|a|+|b|).
        Horizontal rings: |centre| <= |(X, Y, Z)| and r <= R with X = sum |A|+|B| of x_c, etc.
        """
        if self.kind == 1:
            X, Y, Z, Rr = (sum(abs(A) + abs(B) for (_, A, B) in part) for part in self.series)
            return math.sqrt(X * X + Y * Y + Z * Z) + Rr
        amp = sum(abs(a) for a in self.mode_cos) + sum(abs(b) for b in self.mode_sin)
        return 0.5 * self.axis_length + self.base_radius * (1.0 + amp)


@dataclasses.dataclass
class Scene:
    name: str
    bodies: List[Body]
    k: float
    eta: float
    directions: np.ndarray  # (R, 3) unit vectors

    @property
    def n_nodes(self) -> int:
        return sum(b.n_nodes for b in self.bodies)

    @property
    def n_rhs(self) -> int:
        return int(self.directions.shape[0])

    def pair_count(self) -> int:
        """Inter-body kernel evaluations per operator apply: N^2 - sum n_b^2."""
        n = self.n_nodes
        return n * n - sum(b.n_nodes ** 2 for b in self.bodies)


def rot_zy(t1: float, t2: float) -> List[float]:
    """R = R_z(t1) R_y(t2), row-major (Section 6.5)."""
    c1, s1, c2, s2 = math.cos(t1), math.sin(t1), math.cos(t2), math.sin(t2)
    rz = np.array([[c1, -s1, 0.0], [s1, c1, 0.0], [0.0, 0.0, 1.0]])
    ry = np.array([[c2, 0.0, s2], [0.0, 1.0, 0.0], [-s2, 0.0, c2]])
    return list((rz @ ry).reshape(-1))


def paper_direction() -> np.ndarray:
    """d = (cos t sin p, sin t sin p, cos p) with t = pi/3, p = 2 pi/3 (Section 6)."""
    t, p = math.pi / 3, 2 * math.pi / 3
    return np.array([[math.cos(t) * math.sin(p), math.sin(t) * math.sin(p), math.cos(p)]])


def fibonacci_directions(n: int, rng: Optional[np.random.Generator] = None) -> np.ndarray:
    """n unit vectors on a golden-angle (Fibonacci) spiral, optionally randomly rotated."""
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = math.pi * (3.0 - math.sqrt(5.0)) * i
    rr = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    d = np.stack([rr * np.cos(phi), rr * np.sin(phi), z], axis=1)
    if rng is not None:
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, zq = q
        rot = np.array([
            [1 - 2 * (y * y + zq * zq), 2 * (x * y - zq * w), 2 * (x * zq + y * w)],
            [2 * (x * y + zq * w), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - x * w)],
            [2 * (x * zq - y * w), 2 * (y * zq + x * w), 1 - 2 * (x * x + y * y)],
        ])
        d = d @ rot.T
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def random_bodies(rng: np.random.Generator, n_bodies: int, box: float, min_gap: float,
                  n_panels: int, order: int, n_theta: int, n_modes: int = 3,
                  mode_amp: float = 0.1, kappa_max: float = 0.5,
                  max_tries: int = 200000) -> List[Body]:
    """Seeded quasi-axisymmetric bodies placed in [0, box]^3 by rejection sampling.

    Bounding balls of radius ``bound_radius`` must be ``min_gap`` apart, so the
    true surface-to-surface gap is at least ``min_gap``.
    """
    bodies: List[Body] = []
    centers: List[np.ndarray] = []
    radii: List[float] = []
    tries = 0
    while len(bodies) < n_bodies:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place bodies with the requested gap")
        a = rng.uniform(-mode_amp, mode_amp, size=n_modes)
        b = rng.uniform(-mode_amp, mode_amp, size=n_modes)
        kappa = rng.uniform(0.0, kappa_max)
        t1, t2 = rng.uniform(0.0, 2 * math.pi, size=2)
        c = rng.uniform(0.0, box, size=3)
        body = Body(n_panels, order, n_theta, 0.5, tuple(a), tuple(b), 1.0, float(kappa),
                    tuple(rot_zy(t1, t2)), tuple(c))
        rb = body.bound_radius()
        ok = all(np.linalg.norm(c - cc) >= rb + rr + min_gap for cc, rr in zip(centers, radii))
        if ok:
            bodies.append(body)
            centers.append(c)
            radii.append(rb)
    return bodies


def config(idx: int, request_id: int = 0) -> Scene:
    """The five workloads (0-based index), seeded with 31380 + 1000*config + request_id."""
    rng = np.random.default_rng(31380 + 1000 * (idx + 1) + request_id)
    if idx == 0:
        # two straight axisymmetric bodies, centres 3 apart, 16 x 32 nodes, k = 1, d = x
        b = [Body(1, 16, 32, 0.5, (0.2,), (), 1.0, 0.0, (1, 0, 0, 0, 1, 0, 0, 0, 1), (s, 0.0, 0.0))
             for s in (-1.5, 1.5)]
        return Scene("2 axisymmetric bodies, 16x32 nodes, k=1", b, 1.0, 1.0,
                     np.array([[1.0, 0.0, 0.0]]))
    if idx == 1:
        b = random_bodies(rng, 16, 12.0, 0.5, 2, 16, 64)
        return Scene("16 quasi-axisymmetric bodies, 32x64 nodes, k=5", b, 5.0, 1.0, paper_direction())
    if idx == 2:
        b = random_bodies(rng, 100, 25.0, 0.5, 2, 12, 48)
        return Scene("100 quasi-axisymmetric bodies, 24x48 nodes, k=10, 16 RHS", b, 10.0, 1.0,
                     fibonacci_directions(16, rng))
    if idx == 3:
        b = random_bodies(rng, 1000, 60.0, 0.5, 1, 16, 32)
        return Scene("1000 quasi-axisymmetric bodies, 16x32 nodes, k=3, 4 RHS", b, 3.0, 1.0,
                     fibonacci_directions(4, rng))
    if idx == 4:
        return serving_request(request_id)
    raise ValueError(idx)


def serving_request(request_id: int, max_bodies: int = 500) -> Scene:
    """One request of the serving stream: 10..max_bodies bodies (500 in the
    full stream), {16x32, 24x48} nodes, k ~ U[1, 15], 1..16 RHS; box side
    60 (N_b/1000)^(1/3), at least 12."""
    rng = np.random.default_rng(31380 + 5000 + request_id)
    nb = int(rng.integers(10, max_bodies + 1))
    disc = (1, 16, 32) if rng.integers(0, 2) == 0 else (2, 12, 48)
    k = float(rng.uniform(1.0, 15.0))
    r = int(rng.integers(1, 17))
    box = max(12.0, 60.0 * (nb / 1000.0) ** (1.0 / 3.0))
    b = random_bodies(rng, nb, box, 0.5, *disc)
    return Scene(f"serving request {request_id}", b, k, 1.0, fibonacci_directions(r, rng))


def reduced(idx: int, n_copies: int) -> Scene:
    """A few rigid copies of workload ``idx``'s first seeded body, with that
    workload's discretisation, wavenumber and incident directions: each copy
    gets a seeded rotation R_z R_y (Sec. 6.5) and a centre on a line, bounding
    balls 1.0 apart.  Congruent copies share one self block, so an oracle
    dense solve stays affordable at the full discretisation."""
    base = config(idx)
    b0 = base.bodies[0]
    rng = np.random.default_rng(31380 + 77 * (idx + 1))
    rb = b0.bound_radius()
    bodies = []
    for i in range(n_copies):
        t1, t2 = rng.uniform(0.0, 2 * math.pi, size=2)
        jitter = rng.uniform(-0.3, 0.3, size=2)
        c = (i * (2 * rb + 1.0), float(jitter[0]), float(jitter[1]))
        bodies.append(dataclasses.replace(b0, rotation=tuple(rot_zy(t1, t2)), center=c))
    return Scene(f"{n_copies} copies of body 0 of workload {idx} ({base.name})", bodies, base.k, base.eta,
                 base.directions)


@dataclasses.dataclass
class LatticeScene(Scene):
    """A regular array of one body: ``dims`` copies along the rows of
    ``basis`` (Sec. 4, regular P x Q x R arrays); ``bodies`` lists them in
    the order p, q, r (body index (p Q + q) R + r)."""
    body: Optional[Body] = None
    dims: tuple = (1, 1, 1)
    basis: Optional[np.ndarray] = None


def lattice_scene(name: str, body: Body, dims, basis, k: float, eta: float,
                  directions: np.ndarray) -> LatticeScene:
    basis = np.asarray(basis, dtype=np.float64).reshape(3, 3)
    c0 = np.asarray(body.center, dtype=np.float64)
    bodies = []
    for p in range(dims[0]):
        for q in range(dims[1]):
            for r in range(dims[2]):
                c = c0 + p * basis[0] + q * basis[1] + r * basis[2]
                bodies.append(dataclasses.replace(body, center=tuple(float(v) for v in c)))
    return LatticeScene(name, bodies, k, eta, directions, body=body, dims=tuple(int(v) for v in dims),
                        basis=basis)


def paper_cubic(P: int = 10, k: float = 2.0, order: int = 16, n_theta: int = 6) -> LatticeScene:
    """P^3 quasi-ellipsoids (Eq. quasiellipsoid) on a cubic lattice of spacing
    0.5, the regular-array experiment of Sec. 6 (Table tab:multibody_cubic:
    N_p = 1, 16 x N_f = 6 nodes, 10^3 bodies in [-1, 4]^3, surface gaps above
    0.05).  Reading: the scale 0.04 keeps bounding balls 0.087 apart; the
    incident direction is the paper's d(pi/3, 2 pi/3)."""
    b = quasi_ellipsoid(1, order, n_theta, scale=0.04, center=(-0.75, -0.75, -0.75))
    return lattice_scene(f"{P}^3 quasi-ellipsoids, 16x{n_theta} nodes, k={k:g}", b, (P, P, P),
                         0.5 * np.eye(3), k, 1.0, paper_direction())


def lattice_of_workload(idx: int, dims=(10, 10, 10), gap: float = 0.5) -> LatticeScene:
    """The first seeded body of workload ``idx`` repeated on a cubic lattice
    whose bounding balls are ``gap`` apart, with that workload's wavenumber
    and incident directions (e.g. 10^3 copies of the 1000-body workload's
    body: the same N = 512,000, k = 3 and 4 right-hand sides, in the
    translation-invariant arrangement of Sec. 4)."""
    base = config(idx)
    b0 = dataclasses.replace(base.bodies[0], center=(0.0, 0.0, 0.0))
    h = 2.0 * b0.bound_radius() + gap
    return lattice_scene(f"{dims[0]}x{dims[1]}x{dims[2]} lattice of body 0 of workload {idx} ({base.name})", b0,
                         dims, h * np.eye(3), base.k, base.eta, base.directions)


def small_scene(n_bodies: int = 3, n_panels: int = 1, order: int = 8, n_theta: int = 16,
                k: float = 2.0, eta: float = 1.0, n_rhs: int = 1, seed: int = 7,
                box: float = 6.0) -> Scene:
    """A few small random bodies, for parity tests the oracle finishes in seconds."""
    rng = np.random.default_rng(seed)
    b = random_bodies(rng, n_bodies, box, 0.5, n_panels, order, n_theta)
    d = paper_direction() if n_rhs == 1 else fibonacci_directions(n_rhs, rng)
    return Scene(f"small {n_bodies} bodies", b, k, eta, d)


def sphere(radius: float, n_panels: int, order: int, n_theta: int,
           center=(0.0, 0.0, 0.0)) -> Body:
    """rho = a, L = 2a: r(s) = a cos s, axial coordinate a sin s -- a sphere."""
    return Body(n_panels, order, n_theta, radius, (), (), 2.0 * radius, 0.0,
                (1, 0, 0, 0, 1, 0, 0, 0, 1), tuple(center))


def rhs_seeded(n: int, r: int, seed: int) -> np.ndarray:
    """A seeded complex [n, r] array with entries ~ N(0,1) + i N(0,1)."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, r)) + 1j * rng.normal(size=(n, r))


# ---------------------------------------------------------------------------
# The paper's named shapes (Eqs. quasiwave and geometries), as horizontal-ring
# series; ``scale`` multiplies every length (the factor a of Sec. 6.5).

def _ring_body(series, n_panels, order, n_theta, scale, breaks=(), **kw) -> Body:
    sc = tuple(tuple((om, scale * A, scale * B) for (om, A, B) in part) for part in series)
    return Body(n_panels, order, n_theta, kind=1, series=sc, panel_breaks=tuple(breaks), **kw)


def quasi_wave(n_panels=8, order=16, n_theta=40, scale=1.0, **kw) -> Body:
    """x = 0.2 cos 4t + cos t cos phi, y = cos t sin phi, z = 2 sin t."""
    return _ring_body((((4.0, 0.2, 0.0),), (), ((1.0, 0.0, 2.0),), ((1.0, 1.0, 0.0),)),
                      n_panels, order, n_theta, scale, **kw)


def quasi_ellipsoid(n_panels=6, order=16, n_theta=40, scale=1.0, **kw) -> Body:
    """x = cos t + 2 cos t cos phi, y = 2 cos t sin phi, z = 3 sin t."""
    return _ring_body((((1.0, 1.0, 0.0),), (), ((1.0, 0.0, 3.0),), ((1.0, 2.0, 0.0),)),
                      n_panels, order, n_theta, scale, **kw)


def spiral(n_panels=8, order=16, n_theta=40, scale=1.0, **kw) -> Body:
    """x = 0.05 cos 4 pi t + 1.5 cos t cos phi, y = 0.1 sin 4 pi t + 1.5 cos t sin phi, z = 2 sin t."""
    w = 4.0 * math.pi
    return _ring_body((((w, 0.05, 0.0),), ((w, 0.0, 0.1),), ((1.0, 0.0, 2.0),), ((1.0, 1.5, 0.0),)),
                      n_panels, order, n_theta, scale, **kw)


def conch(n_panels=6, order=16, n_theta=40, scale=1.0, **kw) -> Body:
    """x = (0.2 + 0.1 sin 8t) cos t + cos t cos phi, y = (0.2 + 0.1 sin 8t) sin t + cos t sin phi,
    z = 1.5 sin t; the centre products expanded: sin 8t cos t = (sin 9t + sin 7t)/2,
    sin 8t sin t = (cos 7t - cos 9t)/2."""
    return _ring_body((((1.0, 0.2, 0.0), (9.0, 0.0, 0.05), (7.0, 0.0, 0.05)),
                       ((1.0, 0.0, 0.2), (7.0, 0.05, 0.0), (9.0, -0.05, 0.0)),
                       ((1.0, 0.0, 1.5),), ((1.0, 1.0, 0.0),)),
                      n_panels, order, n_theta, scale, **kw)


def dyadic_breaks(n_uniform: int, n_ref: int) -> tuple:
    """n_uniform equal panels in s, the two end panels then bisected n_ref times
    toward the poles: n_uniform + 2 n_ref panels (Sec. 6.1, N_ref)."""
    if n_uniform < 2:
        raise ValueError("dyadic refinement needs at least two uniform panels")
    w = math.pi / n_uniform
    left = [-math.pi / 2] + [-math.pi / 2 + w / 2 ** (n_ref - i) for i in range(n_ref)]
    inner = [-math.pi / 2 + w * i for i in range(1, n_uniform)]
    right = [math.pi / 2 - w / 2 ** (i + 1) for i in range(n_ref)] + [math.pi / 2]
    return tuple(left + inner + right)
