"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module holds geometry only: grids, body circles, boundary-condition kinds and
the seeded random draws of the parametric studies.  It contains none of the
method's arithmetic (no mesh rules, no element matrices, no solve), so both the
GPU library and the CPU oracle can take their inputs from here without sharing
any computation.

The layouts stand in for the paper's five-cylinder study (Results section,
"Potential Flow Interferences in a Multiple-Body System" and "Effect of Gap Ratio",
Table 1), whose exact cylinder positions are only given in figures that are not
available.  The single-cylinder case stands in for the Validation section.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Side order used everywhere: left (x = x0), right (x = x1), bottom (y = y0), top (y = y1).
BC_DIRICHLET_UY = 0   # psi = U * y prescribed on the side (uniform stream)
BC_NATURAL = 1        # zero normal derivative of psi (inlet / outlet)
ALL_DIRICHLET = (BC_DIRICHLET_UY,) * 4


@dataclass
class Case:
    """One geometric variant: background grid, circular bodies and side BCs."""
    x0: float
    x1: float
    y0: float
    y1: float
    nx: int
    ny: int
    bodies: np.ndarray                 # (n_bodies, 3) rows of (cx, cy, r), float64
    sweeps: int
    bc: tuple = ALL_DIRICHLET
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def grid(self):
        return (self.x0, self.x1, self.y0, self.y1, self.nx, self.ny)

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1)


def five_cylinders(delta: float, D: float = 1.0, jitter=None) -> np.ndarray:
    """Five cylinders of diameter D: two streamwise at (-5D, 0), (5D, 0) and three
    transverse at x = 0, y = 0 and y = -/+ (D + delta*D), i.e. surface gap delta*D
    between the middle and each outer transverse cylinder.

    Body order: 0 = (-5D, 0), 1 = (0, 0), 2 = (5D, 0), 3 = bottom transverse,
    4 = top transverse.  The transverse-gap flow is psi[4] - psi[3].
    """
    r = 0.5 * D
    c = np.array([[-5 * D, 0.0], [0.0, 0.0], [5 * D, 0.0],
                  [0.0, -(D + delta * D)], [0.0, D + delta * D]], dtype=np.float64)
    if jitter is not None:
        c = c + np.asarray(jitter, dtype=np.float64).reshape(5, 2)
    return np.concatenate([c, np.full((5, 1), r)], axis=1)


def single_cylinder(nx: int = 128, ny: int = 64, sweeps: int = 50, a: float = 0.5) -> Case:
    """One cylinder of radius a at the origin in [-10,10]x[-5,5]."""
    return Case(-10.0, 10.0, -5.0, 5.0, nx, ny, np.array([[0.0, 0.0, a]]), sweeps,
                name=f"single_cylinder_{nx}x{ny}")


def five_cylinder_case(delta: float, nx: int = 2048, ny: int = 1024, sweeps: int = 200,
                       jitter=None) -> Case:
    """Five-cylinder layout in [-20,20]x[-10,10] with psi = U*y on all four sides."""
    return Case(-20.0, 20.0, -10.0, 10.0, nx, ny, five_cylinders(delta, jitter=jitter),
                sweeps, name=f"five_cyl_d{delta:g}_{nx}x{ny}", meta={"delta": delta})


FIVE_CYL_DELTAS = (0.1, 0.25, 0.5, 1.0, 2.0)


def _min_gap(bodies: np.ndarray) -> float:
    g = np.inf
    for a in range(len(bodies)):
        for b in range(a + 1, len(bodies)):
            d = np.hypot(*(bodies[a, :2] - bodies[b, :2])) - bodies[a, 2] - bodies[b, 2]
            g = min(g, d)
    return g


def parametric_sweep(n_variants: int = 256, seed: int = 0, jitter_sigma: float = 0.05,
                     nx_choices=tuple(range(256, 1025, 32)), sweeps: int = 200,
                     min_gap: float = 0.05, D: float = 1.0) -> list:
    """Batched parametric sweep: delta ~ U[0.1, 2.0], every centre jittered by
    N(0, sigma^2 D^2) per coordinate, nx uniform over nx_choices, ny = nx/2, domain
    [-20,20]x[-10,10].  A variant's jitter is redrawn while any surface gap is below
    min_gap*D or any body comes within 2D of the outer boundary."""
    rng = np.random.default_rng(seed)
    cases = []
    for v in range(n_variants):
        delta = float(rng.uniform(0.1, 2.0))
        nx = int(rng.choice(np.asarray(nx_choices)))
        while True:
            jit = rng.normal(0.0, jitter_sigma * D, size=(5, 2)) if jitter_sigma > 0 else None
            bodies = five_cylinders(delta, D, jit)
            ok = _min_gap(bodies) >= min_gap * D
            ok &= bool(np.all(np.abs(bodies[:, 0]) + bodies[:, 2] <= 20.0 - 2 * D))
            ok &= bool(np.all(np.abs(bodies[:, 1]) + bodies[:, 2] <= 10.0 - 2 * D))
            if ok:
                break
        cases.append(Case(-20.0, 20.0, -10.0, 10.0, nx, nx // 2, bodies, sweeps,
                          name=f"sweep{seed}_{v}", meta={"delta": delta}))
    return cases


def gradient_study(n_variants: int = 64, seed: int = 1, nx: int = 1024, sweeps: int = 200) -> list:
    """Differentiation study: delta ~ U[0.1, 2.0], no jitter, nx x nx/2 grids."""
    rng = np.random.default_rng(seed)
    return [five_cylinder_case(float(rng.uniform(0.1, 2.0)), nx, nx // 2, sweeps)
            for _ in range(n_variants)]


PAPER_TABLE1_DELTAS = (0.3, 0.4, 0.5, 0.6, 0.7)


def paper_channel_case(delta: float, nx: int = 403, ny: int = 201, sweeps: int = 60) -> Case:
    """The paper's channel layout (Results section, Table 1): [0,1]x[0,0.5] with walls
    psi = 0 (bottom) and psi = U/2 (top) and natural inlet and outlet; three cylinders of
    diameter 0.2 on the axis y = 0.25 and two of diameter 0.1 above and below it with
    centre distance h_c = delta * h_d (h_d = 0.5, the channel height).  The x positions
    are assumed (the paper gives them only in a figure); the grid is chosen so that no
    node lies exactly on a circle.  With U = 2 the walls carry psi = 0 and 1."""
    hd, yc = 0.5, 0.25
    hc = delta * hd
    bodies = np.array([[0.15, yc, 0.1], [0.55, yc, 0.1], [0.85, yc, 0.1],
                       [0.35, yc - hc / 2, 0.05], [0.35, yc + hc / 2, 0.05]])
    return Case(0.0, 1.0, 0.0, 0.5, nx, ny, bodies, sweeps, bc=(BC_NATURAL, BC_NATURAL, BC_DIRICHLET_UY, BC_DIRICHLET_UY),
                name=f"paper_channel_d{delta:g}", meta={"delta": delta})


@dataclass
class PolygonBody:
    """A polygonal body: vertices counter-clockwise, the reference point of the polar
    angle of the surface velocity, and the trailing-edge vertex that carries the Kutta
    condition (-1: none).  `meta` records how the shape was generated."""
    vertices: np.ndarray
    ref: tuple = (0.0, 0.0)
    kutta: int = -1
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.vertices = np.asarray(self.vertices, dtype=np.float64).reshape(-1, 2)


def ellipse_body(a: float, b: float, n: int, cx: float = 0.0, cy: float = 0.0, angle: float = 0.0) -> PolygonBody:
    """n vertices on the ellipse x = a cos t, y = b sin t, turned by `angle` and shifted."""
    t = 2.0 * np.pi * np.arange(n) / n
    x = a * np.cos(t)
    y = b * np.sin(t)
    c, s = np.cos(angle), np.sin(angle)
    return PolygonBody(np.stack([cx + c * x - s * y, cy + s * x + c * y], axis=1), ref=(cx, cy),
                       meta={"a": a, "b": b, "angle": angle})


def joukowski_airfoil(k: float, m: float, n: int, alpha: float = 0.0, shift=(0.0, 0.0)) -> PolygonBody:
    """Symmetric Joukowski airfoil: the circle of radius R = k + m about (-m, 0), mapped by
    z = zeta + k^2 / zeta, turned by -alpha (a stream along +x then meets it at angle of
    attack alpha) and shifted; n vertices counter-clockwise from the trailing edge
    (z = 2k before the turn), which carries the Kutta condition.  Chord about 4k,
    thickness about 1.3 m/k of the chord."""
    R = k + m
    th = 2.0 * np.pi * np.arange(n) / n
    zeta = -m + R * np.exp(1j * th)
    z = zeta + k * k / zeta
    z = z * np.exp(-1j * alpha) + complex(*shift)
    return PolygonBody(np.stack([z.real, z.imag], axis=1), ref=tuple(shift), kutta=0,
                       meta={"k": k, "m": m, "R": R, "alpha": alpha, "shift": tuple(shift)})


def airfoil_case(nx: int = 256, alpha_deg: float = 6.0, sweeps: int = None, kutta: bool = True):
    """One Joukowski airfoil (chord about 2, 12% thick, 400 vertices) at angle of attack
    alpha in [-3,3]x[-1.5,1.5] with psi = U*y on all sides: (Case without circles, the
    polygon list)."""
    af = joukowski_airfoil(0.5, 0.08, 400, alpha=np.radians(alpha_deg))
    if not kutta:
        af.kutta = -1
    c = Case(-3.0, 3.0, -1.5, 1.5, nx, nx // 2, np.zeros((0, 3)), nx // 4 if sweeps is None else sweeps,
             name=f"airfoil_{alpha_deg:g}deg_{nx}x{nx // 2}", meta={"alpha_deg": alpha_deg})
    return c, [af]


def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded standard-normal float64 vector (used as an operator input)."""
    return np.random.default_rng(seed).standard_normal(n)
