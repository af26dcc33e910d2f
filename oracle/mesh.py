"""Oracle: body-conforming Q4 grid from a Cartesian background grid (float64).

Follows the section "Body-Conforming Grid Generation": a uniform background grid
covers the domain; grid points immediately inside an immersed boundary are moved
onto it, each receiving the displacement d = x_boundary - x_grid; the displacement
is propagated into the domain by a Laplace problem for d with d = d_i on the
bodies and d = 0 on the grid-aligned outer boundary; finally x_new = x_old + d.

Readings taken where the paper is silent:
  * "immediately inside" = an inside node that is a corner of at least one active
    cell, where a cell is active iff at least one corner lies outside every body;
    a node is inside body k iff (x-cx)^2 + (y-cy)^2 <= r^2 (ties count as inside);
  * the surface point is the radial projection c + r (x - c)/|x - c| and every cell
    stays a quadrilateral (the node splitting and the triangle / pentagon cells are the
    mixed-cell mesh of `oracle.cutmesh`);
  * the Laplace problem for d is approximated by a fixed number S of Jacobi sweeps
    on the logical grid, d_n <- (d_W + d_E + d_S + d_N) / 4 summed in that order,
    over nodes that are outside every body and not on the outer ring.

Polygonal bodies and the Kutta condition (the wake point held at the body's value)
follow `oracle.shapes`; they are appended after the circles, so body k < n_circles is
a circle and the others are polygons in the given order.

Every expression is written so that it is a sequence of individually rounded IEEE
float64 operations (numpy applies no fused multiply-add), which makes the result
reproducible bit for bit by any implementation that performs the same operations.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import shapes as SH

FREE, DIRICHLET, BODY, INACTIVE = 0, 1, 2, 3
BC_DIRICHLET_UY, BC_NATURAL = 0, 1


class MeshError(ValueError):
    pass


@dataclass
class Mesh:
    nx: int
    ny: int
    x: np.ndarray        # (ny+1, nx+1) final node x
    y: np.ndarray        # (ny+1, nx+1) final node y
    xg: np.ndarray       # background grid x
    yg: np.ndarray       # background grid y
    kind: np.ndarray     # (ny+1, nx+1) int8: FREE / DIRICHLET / BODY / INACTIVE
    body: np.ndarray     # (ny+1, nx+1) int32: body index for BODY nodes (and inside nodes), else -1
    active: np.ndarray   # (ny, nx) bool: cell (i, j) active
    bodies: np.ndarray   # (n_bodies, 3): circles (cx, cy, r); polygons (ref x, ref y, 0)
    bc: tuple
    dx0: np.ndarray      # initial (projection) displacement, before smoothing
    dy0: np.ndarray
    polygons: tuple = ()          # polygon bodies (after the circles)
    wake: np.ndarray = None       # (ny+1, nx+1) bool: Kutta wake nodes (held at their body's value)
    wake_node: tuple = ()         # per polygon: flat index of its wake node, or -1
    cut_points: np.ndarray = None  # mixed-cell mesh (`oracle.cutmesh`): (4, ny+1, nx+1, 2) surface points

    @property
    def n_nodes(self):
        return (self.nx + 1) * (self.ny + 1)


def body_boxes(bodies, polygons):
    """Axis-aligned bounding box (xmin, xmax, ymin, ymax) of every body."""
    out = [(cx - r, cx + r, cy - r, cy + r) for cx, cy, r in np.asarray(bodies).reshape(-1, 3)]
    for p in polygons:
        v = p.vertices
        out.append((v[:, 0].min(), v[:, 0].max(), v[:, 1].min(), v[:, 1].max()))
    return out


def validate_inputs(grid, bodies, polygons=()):
    """Host checks: positive sizes, bodies disjoint and at least 2h inside the box.
    Polygons need at least 3 vertices in counter-clockwise order, and their bounding
    boxes may not overlap any other body's (a conservative disjointness test)."""
    x0, x1, y0, y1, nx, ny = grid
    if nx < 2 or ny < 2 or not (x1 > x0) or not (y1 > y0):
        raise MeshError("invalid grid")
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    for k, p in enumerate(polygons):
        if len(p.vertices) < 3 or not (SH.signed_area(p.vertices) > 0):
            raise MeshError(f"polygon {k}: needs >= 3 vertices in counter-clockwise order")
        if p.kutta >= len(p.vertices):
            raise MeshError(f"polygon {k}: Kutta vertex out of range")
    nc = len(np.asarray(bodies).reshape(-1, 3))
    boxes = body_boxes(bodies, polygons)
    for k, (bx0, bx1, by0, by1) in enumerate(boxes[nc:], start=nc):
        if bx0 < x0 + 2 * hx or bx1 > x1 - 2 * hx or by0 < y0 + 2 * hy or by1 > y1 - 2 * hy:
            raise MeshError(f"body {k} is within 2h of the outer boundary")
        for c, (cx0, cx1, cy0, cy1) in enumerate(boxes):
            if c != k and not (bx1 < cx0 or cx1 < bx0 or by1 < cy0 or cy1 < by0):
                raise MeshError(f"bodies {k} and {c} have overlapping bounding boxes")
    b = np.asarray(bodies, dtype=np.float64).reshape(-1, 3)
    for k, (cx, cy, r) in enumerate(b):
        if not (r > 0):
            raise MeshError(f"body {k}: radius must be positive")
        if cx - r < x0 + 2 * hx or cx + r > x1 - 2 * hx or cy - r < y0 + 2 * hy or cy + r > y1 - 2 * hy:
            raise MeshError(f"body {k} is within 2h of the outer boundary")
    for a in range(len(b)):
        for c in range(a + 1, len(b)):
            ddx = b[a, 0] - b[c, 0]
            ddy = b[a, 1] - b[c, 1]
            if ddx * ddx + ddy * ddy <= (b[a, 2] + b[c, 2]) ** 2:
                raise MeshError(f"bodies {a} and {c} overlap or touch")
    return b


def background_grid(grid):
    """Uniform background grid: x = x0 + i*hx, y = y0 + j*hy (one multiply, one add)."""
    x0, x1, y0, y1, nx, ny = grid
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    xs = x0 + np.arange(nx + 1, dtype=np.float64) * hx
    ys = y0 + np.arange(ny + 1, dtype=np.float64) * hy
    xg, yg = np.meshgrid(xs, ys)          # (ny+1, nx+1), row j, column i
    return xg, yg


def classify(xg, yg, bodies, polygons=()):
    """Inside test of every node against every body; returns body index or -1."""
    body = np.full(xg.shape, -1, dtype=np.int32)
    for k, (cx, cy, r) in enumerate(bodies):
        dx = xg - cx
        dy = yg - cy
        inside = (dx * dx + dy * dy) <= r * r
        if np.any(inside & (body >= 0)):
            raise MeshError("node inside two bodies")
        body[inside] = k
    for q, p in enumerate(polygons):
        k = len(bodies) + q
        inside = SH.inside_polygon(xg, yg, p.vertices)
        if np.any(inside & (body >= 0)):
            raise MeshError("node inside two bodies")
        body[inside] = k
    return body


def node_kinds(body, bc):
    """Active cells, and FREE / DIRICHLET / BODY / INACTIVE per node."""
    ny1, nx1 = body.shape
    outside = body < 0
    active = outside[:-1, :-1] | outside[:-1, 1:] | outside[1:, :-1] | outside[1:, 1:]
    corner_of_active = np.zeros(body.shape, dtype=bool)
    corner_of_active[:-1, :-1] |= active
    corner_of_active[:-1, 1:] |= active
    corner_of_active[1:, :-1] |= active
    corner_of_active[1:, 1:] |= active
    kind = np.full(body.shape, FREE, dtype=np.int8)
    kind[~outside & corner_of_active] = BODY
    kind[~outside & ~corner_of_active] = INACTIVE
    left, right, bottom, top = bc
    ring = np.zeros(body.shape, dtype=bool)
    if left == BC_DIRICHLET_UY:
        ring[:, 0] = True
    if right == BC_DIRICHLET_UY:
        ring[:, -1] = True
    if bottom == BC_DIRICHLET_UY:
        ring[0, :] = True
    if top == BC_DIRICHLET_UY:
        ring[-1, :] = True
    kind[ring & outside] = DIRICHLET
    return kind, active


def project(xg, yg, body, kind, bodies, polygons=()):
    """Initial displacement: radial projection of every BODY node onto its circle, or
    the nearest point of its polygon."""
    dx0 = np.zeros_like(xg)
    dy0 = np.zeros_like(yg)
    for q, p in enumerate(polygons):
        m = (kind == BODY) & (body == len(bodies) + q)
        qx, qy = SH.nearest_on_polygon(xg[m], yg[m], p.vertices)
        dx0[m] = qx - xg[m]
        dy0[m] = qy - yg[m]
    for k, (cx, cy, r) in enumerate(bodies):
        m = (kind == BODY) & (body == k)
        ex = xg[m] - cx
        ey = yg[m] - cy
        rho = np.sqrt(ex * ex + ey * ey)
        if np.any(rho == 0.0):
            raise MeshError("grid node at a body centre")
        xb = cx + (r * ex) / rho
        yb = cy + (r * ey) / rho
        dx0[m] = xb - xg[m]
        dy0[m] = yb - yg[m]
    return dx0, dy0


def smoothing_mask(kind, body, wake=None):
    """Nodes updated by the Jacobi sweeps: outside every body, not on the outer ring and
    not a Kutta wake node (which keeps its position on the wake line)."""
    m = body < 0
    if wake is not None:
        m = m & ~wake
    m[0, :] = False
    m[-1, :] = False
    m[:, 0] = False
    m[:, -1] = False
    return m


def jacobi_sweeps(d, mask, sweeps):
    """S Jacobi sweeps of the 5-point Laplacian for one displacement component.
    Every node under `mask` has four non-inactive neighbours (an outside node makes
    all four of its cells active), so the neighbour average divides by 4; the sum is
    taken in the order W, E, S, N."""
    d = d.copy()
    for _ in range(sweeps):
        s = ((d[1:-1, :-2] + d[1:-1, 2:]) + d[:-2, 1:-1]) + d[2:, 1:-1]
        new = s / 4.0
        inner = mask[1:-1, 1:-1]
        d[1:-1, 1:-1] = np.where(inner, new, d[1:-1, 1:-1])
    return d


def kutta_nodes(xg, yg, body, kind, dx0, dy0, bodies, polygons, hx):
    """Kutta condition of every polygon that asks for it: the fluid node nearest to the
    wake point W = T + hx w (T the trailing edge, w the bisector) moves onto W (it stays
    a fluid node; the solve holds it at the body's value, `oracle.system.kutta_rows`).  Returns the wake-node mask and, per polygon, the
    flat index of its wake node (-1 without a Kutta condition)."""
    wake = np.zeros(xg.shape, dtype=bool)
    wake_node = []
    for q, p in enumerate(polygons):
        if p.kutta < 0:
            wake_node.append(-1)
            continue
        k = len(bodies) + q
        T, _, W = SH.kutta_points(p, hx)
        nw = SH.nearest_node(xg, yg, kind == FREE, W[0], W[1])
        j, i = divmod(nw, xg.shape[1])
        dx0[j, i] = W[0] - xg[j, i]
        dy0[j, i] = W[1] - yg[j, i]
        wake[j, i] = True
        wake_node.append(nw)
    return wake, tuple(wake_node)


def build_mesh(grid, bodies, sweeps, bc=(0, 0, 0, 0), polygons=()) -> Mesh:
    """Background grid -> classify -> project (and Kutta points) -> S smoothing sweeps ->
    x = x_grid + d."""
    polygons = tuple(polygons)
    bodies = validate_inputs(grid, bodies, polygons)
    x0, x1, y0, y1, nx, ny = grid
    xg, yg = background_grid(grid)
    body = classify(xg, yg, bodies, polygons)
    kind, active = node_kinds(body, bc)
    dx0, dy0 = project(xg, yg, body, kind, bodies, polygons)
    wake, wake_node = kutta_nodes(xg, yg, body, kind, dx0, dy0, bodies, polygons, (x1 - x0) / nx)
    mask = smoothing_mask(kind, body, wake)
    dx = jacobi_sweeps(dx0, mask, sweeps)
    dy = jacobi_sweeps(dy0, mask, sweeps)
    rows = np.concatenate([bodies, np.array([[p.ref[0], p.ref[1], 0.0] for p in polygons]).reshape(-1, 3)])
    return Mesh(nx, ny, xg + dx, yg + dy, xg, yg, kind, body, active, rows, tuple(bc), dx0, dy0, polygons, wake,
                wake_node)


def cell_coords(mesh: Mesh):
    """(ny, nx, 4, 2) corner coordinates of every cell, corners counter-clockwise
    (i,j), (i+1,j), (i+1,j+1), (i,j+1)."""
    X, Y = mesh.x, mesh.y
    cx = np.stack([X[:-1, :-1], X[:-1, 1:], X[1:, 1:], X[1:, :-1]], axis=-1)
    cy = np.stack([Y[:-1, :-1], Y[:-1, 1:], Y[1:, 1:], Y[1:, :-1]], axis=-1)
    return np.stack([cx, cy], axis=-1)


def cell_nodes(nx, ny):
    """(ny, nx, 4) logical node indices n = j*(nx+1) + i of the four corners."""
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    n0 = j * (nx + 1) + i
    return np.stack([n0, n0 + 1, n0 + 1 + (nx + 1), n0 + (nx + 1)], axis=-1)
