"""Oracle (test infrastructure only): polygonal immersed bodies and the Kutta condition.

Section "Body-Conforming Grid Generation" takes each immersed body as a closed boundary
curve; section "Boundary Conditions" adds, for bodies with corners or sharp trailing
edges, the Kutta condition: an additional point in the fluid region, placed so that the
flow leaves the trailing edge tangentially to the line from the trailing edge to that
point, is held at the body's stream-function value (a nearby fluid node may be moved
onto the line).  Section "Matrix-Free Conjugate Gradient with Multiple Constraint
Enforcement" counts the Kutta condition in the body's single constraint.

Readings taken where the paper is silent (the same rules are in the CUDA library):
  * a polygon is given by its vertices in counter-clockwise order; a node is inside iff
    the crossing-number test counts an odd number of edge crossings of the ray to +x,
    with the edge (a, b) crossed when (a_y > y) != (b_y > y) and
    x < a_x + ((y - a_y) (b_x - a_x)) / (b_y - a_y);
  * an "immediately inside" node moves to the nearest point of the polygon boundary:
    per edge t = ((p - a).(b - a)) / |b - a|^2 clamped to [0, 1], q = a + t (b - a),
    the first edge (in vertex order) with the smallest |p - q|^2 wins;
  * Kutta condition at vertex T: the wake direction w is the unit bisector of the two
    edges meeting at T, pointing out of the body ((T - prev)/|T - prev| +
    (T - next)/|T - next|, normalised); the fluid node nearest to W = T + h w (h the grid
    spacing in x, first in row-major order on ties) moves onto W and is held at the
    body's stream-function value: that equation replaces the body's zero-circulation
    equation (its collapsed row), so the circulation around the body is whatever makes
    the body streamline leave the trailing edge along w (`oracle.system.kutta_rows`).
    (Holding W at the body's value while keeping the collapsed row would only enlarge the
    body and keep the circulation at zero.)  The trailing edge itself is not a mesh node
    when the body is thinner than the grid near it; the body nodes are projected as
    everywhere else;
  * boundary edges of a body (for the surface velocity) never include the wake node;
    the polar angle of an edge midpoint is taken about the body's reference point.

Polygons are any objects with `vertices` ((n, 2), counter-clockwise), `ref` (the
reference point) and `kutta` (vertex index or -1); the seeded geometry generators live
in the shared input module.  Every expression is a sequence of individually rounded
IEEE float64 operations (numpy applies no fused multiply-add), so the classification and
the coordinates can be reproduced bit for bit.
"""
from __future__ import annotations

import numpy as np


def signed_area(v):
    x, y = v[:, 0], v[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def inside_polygon(px, py, v):
    """Crossing-number test of the points (px, py) (arrays) against polygon v."""
    px = np.asarray(px, dtype=np.float64)
    py = np.asarray(py, dtype=np.float64)
    inside = np.zeros(px.shape, dtype=bool)
    n = len(v)
    for e in range(n):
        ax, ay = v[e]
        bx, by = v[(e + 1) % n]
        straddle = (ay > py) != (by > py)
        if not np.any(straddle):
            continue
        with np.errstate(divide="ignore", invalid="ignore"):
            xint = ax + ((py - ay) * (bx - ax)) / (by - ay)
        inside ^= straddle & (px < xint)
    return inside


def nearest_on_polygon(px, py, v):
    """Nearest point of the polygon boundary to each point (arrays), first edge on ties."""
    px = np.asarray(px, dtype=np.float64)
    py = np.asarray(py, dtype=np.float64)
    best = np.full(px.shape, np.inf)
    qx = np.zeros(px.shape)
    qy = np.zeros(px.shape)
    n = len(v)
    for e in range(n):
        ax, ay = v[e]
        bx, by = v[(e + 1) % n]
        dx = bx - ax
        dy = by - ay
        num = (px - ax) * dx + (py - ay) * dy
        den = dx * dx + dy * dy
        t = num / den
        t = np.where(t < 0.0, 0.0, np.where(t > 1.0, 1.0, t))
        cx = ax + t * dx
        cy = ay + t * dy
        ex = px - cx
        ey = py - cy
        d2 = ex * ex + ey * ey
        better = d2 < best
        best = np.where(better, d2, best)
        qx = np.where(better, cx, qx)
        qy = np.where(better, cy, qy)
    return qx, qy


def kutta_points(poly, h):
    """Trailing edge T, unit wake direction w and wake point W = T + h w."""
    v = poly.vertices
    n = len(v)
    k = poly.kutta
    T = v[k]
    a = T - v[(k - 1) % n]
    b = T - v[(k + 1) % n]
    la = np.sqrt(a[0] * a[0] + a[1] * a[1])
    lb = np.sqrt(b[0] * b[0] + b[1] * b[1])
    wx = a[0] / la + b[0] / lb
    wy = a[1] / la + b[1] / lb
    lw = np.sqrt(wx * wx + wy * wy)
    wx = wx / lw
    wy = wy / lw
    return T, (wx, wy), (T[0] + h * wx, T[1] + h * wy)


def nearest_node(xg, yg, mask, X, Y):
    """Flat index of the node under `mask` nearest to (X, Y), first in row-major order."""
    ex = xg - X
    ey = yg - Y
    d2 = np.where(mask, ex * ex + ey * ey, np.inf)
    return int(np.argmin(d2.ravel()))


def joukowski_psi(x, y, poly, U=1.0, kutta=True):
    """Exact stream function of the uniform stream U (along +x) past the Joukowski airfoil
    described by poly.meta (k, m, R = k + m, alpha, shift: the circle of radius R about
    (-m, 0) mapped by z = zeta + k^2 / zeta, turned by -alpha and shifted), with the
    circulation of the Kutta condition (or none):
    psi = Im{U [(zeta - zc) e^{-i alpha} + R^2 e^{i alpha} / (zeta - zc)]} - (Gamma / 2 pi) ln|zeta - zc|,
    zeta the exterior inverse of the map, zc = -m, Gamma = -4 pi U R sin(alpha).
    Returns (psi at the points, psi on the body)."""
    k, m, R, alpha = (poly.meta[s] for s in ("k", "m", "R", "alpha"))
    sx, sy = poly.meta["shift"]
    z = ((np.asarray(x) - sx) + 1j * (np.asarray(y) - sy)) * np.exp(1j * alpha)
    root = np.sqrt(z * z - 4.0 * k * k)
    z1 = 0.5 * (z + root)
    z2 = 0.5 * (z - root)
    zeta = np.where(np.abs(z1 + m) >= np.abs(z2 + m), z1, z2)
    w = zeta + m
    gamma = -4.0 * np.pi * U * R * np.sin(alpha) if kutta else 0.0
    psi = np.imag(U * (w * np.exp(-1j * alpha) + R * R * np.exp(1j * alpha) / w)) - gamma / (2 * np.pi) * np.log(np.abs(w))
    return psi, -gamma / (2 * np.pi) * np.log(R)


def ellipse_psi(x, y, a, b, U=1.0, alpha=0.0):
    """Exact stream function of the uniform stream U (along +x) past the ellipse
    x^2/a^2 + y^2/b^2 = 1 (a > b) turned by -alpha, without circulation: the circle of
    radius R = (a + b)/2 maps onto it by z = zeta + k^2/zeta with k^2 = R (a - b)/2, and
    psi = Im{U (zeta e^{-i alpha} + R^2 e^{i alpha} / zeta)} (zero on the body)."""
    R = 0.5 * (a + b)
    k2 = R * 0.5 * (a - b)
    z = (np.asarray(x) + 1j * np.asarray(y)) * np.exp(1j * alpha)
    root = np.sqrt(z * z - 4.0 * k2)
    z1 = 0.5 * (z + root)
    z2 = 0.5 * (z - root)
    zeta = np.where(np.abs(z1) >= np.abs(z2), z1, z2)
    return np.imag(U * (zeta * np.exp(-1j * alpha) + R * R * np.exp(1j * alpha) / zeta))
