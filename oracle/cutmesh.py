"""Oracle (test infrastructure only): the mixed-cell body-conforming mesh with node
splitting, triangle and pentagon cells and boundary-point redistribution (float64).

Section "Body-Conforming Grid Generation" fixes the steps: grid points just inside a
body move onto its surface; a point that meets the surface at two distinct places is
split (a node-splitting event); the surface displacements are propagated into the
domain by a Laplace problem; the split points turn neighbouring exterior cells into
triangles and pentagons, and a pentagon is divided into a triangle and a quadrilateral
by joining its first split point to the background node opposite; finally the surface
points are redistributed to a prescribed minimum spacing.  The section shows these
steps on a figure only, so every rule below is a reading:

  * node kinds are those of `oracle.mesh` (inside test <= r^2, BODY = an inside corner of
    an active cell, a cell being active iff a corner lies outside every body);
  * a BODY node g of circle (c, r) and an outside 4-neighbour k define the surface point
    P(g, k) where the grid edge g-k crosses the circle: on a horizontal edge
    P = (cx +- sqrt(r^2 - (y_g - cy)^2), y_g), on a vertical edge
    P = (x_g, cy +- sqrt(r^2 - (x_g - cx)^2)), the sign that of k - g.  A node with two or
    more outside neighbours is thereby split into that many surface points;
  * the Laplace problem is solved by the Jacobi sweeps of `oracle.mesh`
    (d_n <- (d_W + d_E + d_S + d_N) / 4, summed in that order), in which a BODY neighbour m
    of the updated node n contributes the displacement P(m, n) - x_m of the surface point
    on their common edge; BODY nodes keep their background position;
  * a cut cell (an active cell with an inside corner) is the polygon walked
    counter-clockwise from corner 0: every outside corner a, and after it the surface
    point on edge a (corner a -> a+1) when exactly one end of that edge is inside.  Three
    vertices make a linear triangle, four a Q4 element; five (one inside corner m) make the
    triangle (P+, c_{m+1}, c_{m+2}) and the quadrilateral (P+, c_{m+2}, c_{m+3}, P-), P+ the
    point on edge m and P- the point on edge m-1.  A cell with two diagonal inside corners,
    or with inside corners of two bodies, is refused (MeshError);
  * every vertex of a piece stands for a cell corner: an outside corner for itself, a
    surface point for the inside corner it came from; the cell's 4x4 matrix is the sum of
    its pieces' element matrices scattered by that map.  All surface points of a body take
    the body's single value C_k, so the split copies share its unknown;
  * redistribution, with minimum spacing s_min = sigma * min(hx, hy), runs once after the
    smoothing: the chord (A, B) of every cut cell (its two surface points, in the order its
    boundary runs counter-clockwise) with 0 < L = |B - A| < s_min pushes A by -f (B - A) and B by +f (B - A),
    f = ((s_min - L) * 0.5) / L; a point adds the pushes of its two cells (the cell below, or
    to the left of, its edge first) and, if pushed at all, is projected radially back onto
    the circle, c + r (Q - c) / |Q - c|.  sigma = 0 leaves every point in place;
  * min det J of a piece: the smallest Jacobian determinant at the 2x2 Gauss points for a
    quadrilateral, twice the signed area for a triangle (its reference triangle has area 1/2);
  * element velocity of a cut cell: the area-weighted mean of its pieces' gradients (the
    triangle's constant gradient, the quadrilateral's at its centre), u = dpsi/dy,
    v = -dpsi/dx; surface tangential velocity: one chord per cut cell, u_t = (psi_c - C) / d
    with psi_c the mean of the polygon's vertex values and d the distance from the mean of
    its vertices to the chord line, theta the polar angle of the chord midpoint; chords of
    zero length are not listed.

Polygonal bodies (`oracle.shapes`, after the circles) take the same steps, with these
readings for their surface points and the Kutta condition:
  * on a row the crossings of the polygon's edges are those of the inside test,
    x = a_x + ((y - a_y)(b_x - a_x)) / (b_y - a_y) for an edge with (a_y > y) != (b_y > y),
    and the surface point is the one nearest the inside node with x_g < x <= x_k (towards
    +x) or x_k < x <= x_g (towards -x); the inside test counts an odd number of them there;
  * on a column the same with x and y exchanged; should rounding near a vertex leave no
    crossing in that range, the crossing nearest the range (the first edge on ties) is
    clipped onto it, and without any crossing on the line the edge's midpoint is taken;
  * a redistributed point of a polygon moves to the nearest point of its boundary
    (`oracle.shapes.nearest_on_polygon`) instead of the radial projection;
  * the Kutta wake node moves onto its point as on the Q4 mesh and keeps that position.

Every mesh expression is a sequence of individually rounded IEEE float64 operations, so
the surface points and the node coordinates are reproducible bit for bit.
"""
from __future__ import annotations

import numpy as np

from . import shapes as SH
from .element import q4_stiffness, shape_derivatives
from .mesh import (BODY, FREE, Mesh, MeshError, background_grid, cell_coords, cell_nodes, classify,
                   kutta_nodes, node_kinds, smoothing_mask, validate_inputs)

DIRS = ((1, 0), (0, 1), (-1, 0), (0, -1))       # E, N, W, S as (di, dj)
CI = (0, 1, 1, 0)                               # corner a of cell (i, j) is node (i + CI[a], j + CJ[a])
CJ = (0, 0, 1, 1)


# ---------------------------------------------------------------- elements
def p1_stiffness(xy):
    """Linear triangle: K_ab = (b_a b_b + c_a c_b) / (4 A) with b_a = y_{a+1} - y_{a+2},
    c_a = x_{a+2} - x_{a+1} (indices mod 3) and 2A = (x1 - x0)(y2 - y0) - (x2 - x0)(y1 - y0).
    Returns (K (3, 3), 2A)."""
    xy = np.asarray(xy, dtype=np.float64)
    x, y = xy[:, 0], xy[:, 1]
    two_a = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0])
    b = np.array([y[1] - y[2], y[2] - y[0], y[0] - y[1]])
    c = np.array([x[2] - x[1], x[0] - x[2], x[1] - x[0]])
    K = (np.outer(b, b) + np.outer(c, c)) / (2.0 * two_a)
    return K, two_a


def piece_stiffness(verts):
    """(K, min det J) of one piece: a triangle (3 vertices) or a Q4 element (4)."""
    verts = np.asarray(verts, dtype=np.float64)
    if len(verts) == 3:
        return p1_stiffness(verts)
    K, dm = q4_stiffness(verts)
    return K, float(dm)


def signed_area(verts):
    """Shoelace area of a polygon (positive when counter-clockwise)."""
    v = np.asarray(verts, dtype=np.float64)
    x, y = v[:, 0], v[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


# ---------------------------------------------------------------- surface points
def neighbour_outside(outside, d):
    """Mask of nodes whose neighbour in direction d lies outside every body."""
    m = np.zeros_like(outside)
    if d == 0:
        m[:, :-1] = outside[:, 1:]
    elif d == 1:
        m[:-1, :] = outside[1:, :]
    elif d == 2:
        m[:, 1:] = outside[:, :-1]
    else:
        m[1:, :] = outside[:-1, :]
    return m


def polygon_crossing(v, xg, yg, xk, yk, d):
    """Surface point of a polygon on the grid edge from the inside node (xg, yg) to its
    outside neighbour (xk, yk) in direction d (readings in the module header)."""
    row = d in (0, 2)
    c = yg if row else xg                     # the grid line
    g, k = (xg, xk) if row else (yg, yk)      # positions along it
    up = k > g
    lo, hi = (g, k) if up else (k, g)
    n = len(v)
    best, fb, fbd, anyx = None, 0.0, np.inf, False
    for e in range(n):
        ax, ay = v[e]
        bx, by = v[(e + 1) % n]
        if row:
            if (ay > c) == (by > c):
                continue
            t = ax + ((c - ay) * (bx - ax)) / (by - ay)
        else:
            if (ax > c) == (bx > c):
                continue
            t = ay + ((c - ax) * (by - ay)) / (bx - ax)
        anyx = True
        if (g < t <= k) if up else (k < t <= g):
            best = t if best is None else (min(best, t) if up else max(best, t))
        else:
            dist = lo - t if t < lo else t - hi
            if dist < fbd:
                fbd, fb = dist, t
    if best is not None:
        s = best
    elif anyx:
        s = min(max(fb, lo), hi)
    else:
        s = (g + k) * 0.5
    return (s, yg) if row else (xg, s)


def surface_points(xg, yg, kind, body, bodies, polygons=()):
    """P[d, j, i] = (x, y) of the surface point of BODY node (i, j) on its edge towards the
    outside neighbour in direction d (E, N, W, S); NaN where there is none."""
    P = np.full((4,) + xg.shape + (2,), np.nan)
    outside = body < 0
    for d in range(4):
        m = (kind == BODY) & neighbour_outside(outside, d)
        di, dj = DIRS[d]
        for q, poly in enumerate(polygons):
            js, is_ = np.nonzero(m & (body == len(bodies) + q))
            for j, i in zip(js.tolist(), is_.tolist()):
                P[d, j, i] = polygon_crossing(poly.vertices, xg[j, i], yg[j, i], xg[j + dj, i + di],
                                              yg[j + dj, i + di], d)
        for k, (cx, cy, r) in enumerate(bodies):
            mk = m & (body == k)
            if d in (0, 2):
                e = yg[mk] - cy
                s = np.sqrt(r * r - e * e)
                P[d][mk, 0] = cx + s if d == 0 else cx - s
                P[d][mk, 1] = yg[mk]
            else:
                e = xg[mk] - cx
                s = np.sqrt(r * r - e * e)
                P[d][mk, 0] = xg[mk]
                P[d][mk, 1] = cy + s if d == 1 else cy - s
    return P


def jacobi_sweeps_cut(d, Pc, grid_c, isbody, mask, sweeps):
    """S Jacobi sweeps of one displacement component (as `oracle.mesh.jacobi_sweeps`) in
    which a BODY neighbour contributes the displacement of its surface point on the common
    edge: Pc[dir] - grid_c, the component of P towards the updated node."""
    D = [Pc[k] - grid_c for k in range(4)]
    d = d.copy()
    ib = isbody
    for _ in range(sweeps):
        w = np.where(ib[1:-1, :-2], D[0][1:-1, :-2], d[1:-1, :-2])     # west neighbour, its E point
        e = np.where(ib[1:-1, 2:], D[2][1:-1, 2:], d[1:-1, 2:])        # east neighbour, its W point
        s = np.where(ib[:-2, 1:-1], D[1][:-2, 1:-1], d[:-2, 1:-1])     # south neighbour, its N point
        n = np.where(ib[2:, 1:-1], D[3][2:, 1:-1], d[2:, 1:-1])        # north neighbour, its S point
        new = (((w + e) + s) + n) / 4.0
        inner = mask[1:-1, 1:-1]
        d[1:-1, 1:-1] = np.where(inner, new, d[1:-1, 1:-1])
    return d


# ---------------------------------------------------------------- cut cells
def cell_inside(body, j, i):
    return [body[j + CJ[a], i + CI[a]] >= 0 for a in range(4)]


def edge_point(inside, a):
    """(corner, direction) of the surface point on edge a of a cell, or None."""
    b = (a + 1) % 4
    if inside[a] == inside[b]:
        return None
    return (a, a) if inside[a] else (b, (a + 2) % 4)


def cut_polygon(mesh: Mesh, j, i, P=None):
    """Walk of cut cell (i, j): list of (xy, corner, point id) with point id = (corner, dir)
    for surface points and None for outside corners."""
    P = mesh.cut_points if P is None else P
    inside = cell_inside(mesh.body, j, i)
    if inside[0] == inside[2] and inside[1] == inside[3] and inside[0] != inside[1]:
        raise MeshError(f"cell ({i}, {j}) has two diagonal inside corners")
    bs = {int(mesh.body[j + CJ[a], i + CI[a]]) for a in range(4) if inside[a]}
    if len(bs) > 1:
        raise MeshError(f"cell ({i}, {j}) has inside corners of two bodies")
    out = []
    for a in range(4):
        if not inside[a]:
            out.append((np.array([mesh.x[j + CJ[a], i + CI[a]], mesh.y[j + CJ[a], i + CI[a]]]), a, None))
        ep = edge_point(inside, a)
        if ep is not None:
            g, d = ep
            out.append((P[d, j + CJ[g], i + CI[g]].copy(), g, (g, d)))
    return out


def cut_pieces(mesh: Mesh, j, i):
    """Pieces of cut cell (i, j): list of (vertices (n, 2), corners (n,))."""
    poly = cut_polygon(mesh, j, i)
    if len(poly) in (3, 4):
        return [(np.array([p[0] for p in poly]), [p[1] for p in poly])]
    inside = cell_inside(mesh.body, j, i)
    m = inside.index(True)
    P = mesh.cut_points
    node = (j + CJ[m], i + CI[m])
    p_next = P[m, node[0], node[1]]                       # on edge m, towards corner m+1
    p_prev = P[(m + 1) % 4, node[0], node[1]]             # on edge m-1, towards corner m-1

    def corner(a):
        a %= 4
        return np.array([mesh.x[j + CJ[a], i + CI[a]], mesh.y[j + CJ[a], i + CI[a]]])
    tri = (np.array([p_next, corner(m + 1), corner(m + 2)]), [m, (m + 1) % 4, (m + 2) % 4])
    quad = (np.array([p_next, corner(m + 2), corner(m + 3), p_prev]), [m, (m + 2) % 4, (m + 3) % 4, m])
    return [tri, quad]


def cut_cell_matrix(mesh: Mesh, j, i):
    """(4x4 matrix on the cell's corners, min det J over the pieces)."""
    M = np.zeros((4, 4))
    dm = np.inf
    for verts, cmap in cut_pieces(mesh, j, i):
        K, d = piece_stiffness(verts)
        dm = min(dm, float(d))
        for a in range(len(cmap)):
            for b in range(len(cmap)):
                M[cmap[a], cmap[b]] += K[a, b]
    return M, dm


def cut_cells(mesh: Mesh):
    """(j, i) of every cut cell, row-major."""
    ins = mesh.body >= 0
    any_in = ins[:-1, :-1] | ins[:-1, 1:] | ins[1:, :-1] | ins[1:, 1:]
    js, is_ = np.nonzero(mesh.active & any_in)
    return list(zip(js.tolist(), is_.tolist()))


def chord(mesh: Mesh, j, i, P=None):
    """The two surface points of cut cell (i, j), each as (xy, corner, point id), in the
    order the cell's boundary runs counter-clockwise (the chord from the first to the second
    is an edge of the cell polygon)."""
    poly = cut_polygon(mesh, j, i, P)
    k = [q for q, p in enumerate(poly) if p[2] is not None]
    if k[0] == 0 and k[1] == len(poly) - 1:
        return poly[k[1]], poly[k[0]]
    return poly[k[0]], poly[k[1]]


# ---------------------------------------------------------------- redistribution
def point_cells(i, j, d):
    """The two cells sharing the edge of point (i, j, d): below then above (horizontal
    edge), left then right (vertical edge)."""
    if d == 0:
        return (i, j - 1), (i, j)
    if d == 2:
        return (i - 1, j - 1), (i - 1, j)
    if d == 1:
        return (i - 1, j), (i, j)
    return (i - 1, j - 1), (i, j - 1)


def redistribute(mesh: Mesh, sigma, hx, hy):
    """One pass of the minimum-spacing rule on mesh.cut_points (returns the new array);
    hx = (x1 - x0) / nx and hy = (y1 - y0) / ny are the grid spacings."""
    P0 = mesh.cut_points
    P1 = P0.copy()
    if sigma <= 0:
        return P1
    smin = sigma * min(hx, hy)
    push = {}                                        # (cell i, cell j) -> {point id: (mx, my)}
    for (j, i) in cut_cells(mesh):
        (A, _, ida), (B, _, idb) = chord(mesh, j, i, P0)
        ex = B[0] - A[0]
        ey = B[1] - A[1]
        L = np.sqrt(ex * ex + ey * ey)
        if L > 0.0 and L < smin:
            f = ((smin - L) * 0.5) / L
            mx = f * ex
            my = f * ey
            push[(i, j)] = {ida: (-mx, -my), idb: (mx, my)}
    for d in range(4):
        js, is_ = np.nonzero(~np.isnan(P0[d][..., 0]))
        for j, i in zip(js.tolist(), is_.tolist()):
            moved = False
            qx, qy = P0[d, j, i, 0], P0[d, j, i, 1]
            for cell in point_cells(i, j, d):
                pc = push.get(cell)
                mx, my = 0.0, 0.0
                if pc is not None:
                    ci, cj = cell
                    a = (i - ci) + 3 * (j - cj) - 2 * (i - ci) * (j - cj)   # corner index of node in cell
                    key = (a, d)
                    if key in pc:
                        mx, my = pc[key]
                        moved = True
                qx = qx + mx
                qy = qy + my
            if moved:
                k = mesh.body[j, i]
                nc = len(mesh.bodies) - len(mesh.polygons)
                if k >= nc:
                    px, py = SH.nearest_on_polygon(np.array([qx]), np.array([qy]), mesh.polygons[k - nc].vertices)
                    P1[d, j, i, 0] = px[0]
                    P1[d, j, i, 1] = py[0]
                    continue
                cx, cy, r = mesh.bodies[k]
                ux = qx - cx
                uy = qy - cy
                rho = np.sqrt(ux * ux + uy * uy)
                P1[d, j, i, 0] = cx + (r * ux) / rho
                P1[d, j, i, 1] = cy + (r * uy) / rho
    return P1


# ---------------------------------------------------------------- the mesh
def build_cut_mesh(grid, bodies, sweeps, bc=(0, 0, 0, 0), sigma=0.0, polygons=()) -> Mesh:
    """Background grid -> classify -> surface points (node splitting) and Kutta wake points
    -> S smoothing sweeps with the points' displacements as data -> x = x_grid + d ->
    redistribution.  Circles, then polygons.  BODY nodes keep their background
    coordinates; their surface points are mesh.cut_points[d, j, i]."""
    polygons = tuple(polygons)
    bodies = validate_inputs(grid, bodies, polygons)
    xg, yg = background_grid(grid)
    body = classify(xg, yg, bodies, polygons)
    kind, active = node_kinds(body, bc)
    P = surface_points(xg, yg, kind, body, bodies, polygons)
    dx0 = np.zeros_like(xg)
    dy0 = np.zeros_like(yg)
    wake, wake_node = kutta_nodes(xg, yg, body, kind, dx0, dy0, bodies, polygons, (grid[1] - grid[0]) / grid[4])
    mask = smoothing_mask(kind, body, wake)
    isbody = kind == BODY
    dx = jacobi_sweeps_cut(dx0, P[..., 0], xg, isbody, mask, sweeps)
    dy = jacobi_sweeps_cut(dy0, P[..., 1], yg, isbody, mask, sweeps)
    rows = np.concatenate([bodies, np.array([[p.ref[0], p.ref[1], 0.0] for p in polygons]).reshape(-1, 3)])
    m = Mesh(grid[4], grid[5], xg + dx, yg + dy, xg, yg, kind, body, active, rows, tuple(bc), dx0, dy0,
             polygons, wake, wake_node, P)
    for (j, i) in cut_cells(m):                     # refuse saddles and two-body cells early
        cut_polygon(m, j, i)
    x0, x1, y0, y1, nx, ny = grid
    m.cut_points = redistribute(m, sigma, (x1 - x0) / nx, (y1 - y0) / ny)
    return m


def element_matrices(mesh: Mesh):
    """K_e (E_active, 4, 4), corner node indices and min det J of every active cell:
    Q4 on the cell's corners, or the cut-cell matrix."""
    xy = cell_coords(mesh)[mesh.active]
    cells = cell_nodes(mesh.nx, mesh.ny)[mesh.active]
    Ke, detmin = q4_stiffness(xy)
    Ke = Ke.copy()
    detmin = np.array(detmin, dtype=np.float64).copy()
    pos = -np.ones((mesh.ny, mesh.nx), dtype=np.int64)
    pos[mesh.active] = np.arange(int(mesh.active.sum()))
    for (j, i) in cut_cells(mesh):
        M, dm = cut_cell_matrix(mesh, j, i)
        Ke[pos[j, i]] = M
        detmin[pos[j, i]] = dm
    return Ke, cells, detmin


# ---------------------------------------------------------------- outputs
def velocity_field(mesh: Mesh, psi: np.ndarray):
    """(u, v) = (dpsi/dy, -dpsi/dx) per active cell (row-major): at the centre of an uncut
    cell, the area-weighted mean of the pieces' gradients on a cut cell."""
    from .potential import element_gradient
    fx, fy, _, _ = element_gradient(mesh, psi)
    fx, fy = fx.copy(), fy.copy()
    pos = -np.ones((mesh.ny, mesh.nx), dtype=np.int64)
    pos[mesh.active] = np.arange(int(mesh.active.sum()))
    P = psi.reshape(mesh.ny + 1, mesh.nx + 1)
    for (j, i) in cut_cells(mesh):
        gx = gy = wsum = 0.0
        for verts, cmap in cut_pieces(mesh, j, i):
            vals = np.array([P[j + CJ[a], i + CI[a]] for a in cmap])
            if len(cmap) == 3:
                K, two_a = p1_stiffness(verts)
                x, y = verts[:, 0], verts[:, 1]
                b = np.array([y[1] - y[2], y[2] - y[0], y[0] - y[1]])
                c = np.array([x[2] - x[1], x[0] - x[2], x[1] - x[0]])
                px, py, w = (b @ vals) / two_a, (c @ vals) / two_a, 0.5 * two_a
            else:
                dxi, deta = shape_derivatives(0.0, 0.0)
                x, y = verts[:, 0], verts[:, 1]
                j00, j01, j10, j11 = x @ dxi, y @ dxi, x @ deta, y @ deta
                det = j00 * j11 - j01 * j10
                px = ((j11 * dxi - j01 * deta) / det) @ vals
                py = ((-j10 * dxi + j00 * deta) / det) @ vals
                w = 4.0 * det
            gx += w * px
            gy += w * py
            wsum += w
        fx[pos[j, i]] = gx / wsum
        fy[pos[j, i]] = gy / wsum
    return fy, -fx


def surface_velocity(mesh: Mesh, psi: np.ndarray, C: np.ndarray, k: int):
    """theta_deg, u_t of body k: one chord per cut cell of the body (row-major), zero-length
    chords skipped."""
    P = psi.reshape(mesh.ny + 1, mesh.nx + 1)
    cx, cy, _ = mesh.bodies[k]
    th, ut = [], []
    for (j, i) in cut_cells(mesh):
        inside = cell_inside(mesh.body, j, i)
        a_in = inside.index(True)
        if mesh.body[j + CJ[a_in], i + CI[a_in]] != k:
            continue
        poly = cut_polygon(mesh, j, i)
        (A, _, _), (B, _, _) = chord(mesh, j, i)
        if A[0] == B[0] and A[1] == B[1]:
            continue
        vals = np.array([P[j + CJ[a], i + CI[a]] for _, a, _ in poly])
        V = np.array([p[0] for p in poly])
        psic = vals.mean()
        gx, gy = V[:, 0].mean(), V[:, 1].mean()
        ex, ey = B[0] - A[0], B[1] - A[1]
        dnc = abs(ex * (gy - A[1]) - ey * (gx - A[0])) / np.hypot(ex, ey)
        ut.append((psic - C[k]) / dnc)
        t = np.degrees(np.arctan2(0.5 * (A[1] + B[1]) - cy, 0.5 * (A[0] + B[0]) - cx))
        th.append(t + 360.0 if t < 0 else t)
    return np.array(th), np.array(ut)


__all__ = ["build_cut_mesh", "element_matrices", "surface_points", "cut_cells", "cut_pieces", "cut_polygon",
           "cut_cell_matrix", "chord", "redistribute", "p1_stiffness", "piece_stiffness", "signed_area",
           "velocity_field", "surface_velocity", "FREE", "BODY"]
