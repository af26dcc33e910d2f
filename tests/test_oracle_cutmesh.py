"""Pins of the mixed-cell mesh oracle (`oracle.cutmesh`: node splitting, triangle and
pentagon cells, boundary-point redistribution) against what geometry and the
mathematics fix, independently of the oracle's own formulas:

* hand-built layouts where the split points, the cell polygons and the pentagon's
  triangle + quadrilateral are written out by hand;
* the linear triangle against the textbook right-triangle stiffness;
* the tiling identity: the signed areas of all pieces add up to the box minus the polygons
  of surface chords (a gap, an overlap or a mis-ordered vertex anywhere breaks it), and each
  chord polygon is inscribed in its circle;
* the linear patch test piece by piece around every FREE node;
* the closed-form cylinder psi = U y (1 - a^2/rho^2) converging under refinement, and the
  signed surface velocity approaching 2 U sin(theta);
* redistribution: sigma = 0 is the identity, every point stays on its circle, the short
  chords lengthen."""
import numpy as np
import pytest

from oracle import cutmesh as CM, mesh as M, solve as SV, system as S
from paper_2512_12232_gb300 import workloads as W

SQ = np.sqrt


def test_p1_right_triangle_closed_form():
    a, b = 0.7, 0.3
    K, two_a = CM.p1_stiffness([(0.0, 0.0), (a, 0.0), (0.0, b)])
    assert two_a == pytest.approx(a * b)
    ref = 0.5 * np.array([[b / a + a / b, -b / a, -a / b],
                          [-b / a, b / a, 0.0],
                          [-a / b, 0.0, a / b]])
    np.testing.assert_allclose(K, ref, rtol=1e-14, atol=1e-14)
    # rigid motions leave it unchanged
    th = 0.37
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    xy = np.array([(0.0, 0.0), (a, 0.0), (0.0, b)]) @ R.T + np.array([2.0, -1.0])
    K2, _ = CM.p1_stiffness(xy)
    np.testing.assert_allclose(K2, ref, rtol=1e-13, atol=1e-13)


def single_inside_node_mesh(S=0, sigma=0.0):
    """h = 1, circle (4.2, 4.3) r = 0.45: node (4, 4) alone is inside, with four outside
    neighbours, so it splits into four points and its four cells are pentagons."""
    return CM.build_cut_mesh((0.0, 8.0, 0.0, 8.0, 8, 8), np.array([[4.2, 4.3, 0.45]]), S, sigma=sigma)


def test_node_split_into_four_points_and_four_pentagons():
    m = single_inside_node_mesh()
    assert (m.body >= 0).sum() == 1 and m.kind[4, 4] == M.BODY
    r2 = 0.45 * 0.45
    pts = {d: m.cut_points[d, 4, 4] for d in range(4)}
    np.testing.assert_allclose(pts[0], (4.2 + SQ(r2 - 0.09), 4.0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(pts[1], (4.0, 4.3 + SQ(r2 - 0.04)), rtol=0, atol=1e-15)
    np.testing.assert_allclose(pts[2], (4.2 - SQ(r2 - 0.09), 4.0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(pts[3], (4.0, 4.3 - SQ(r2 - 0.04)), rtol=0, atol=1e-15)
    assert np.isnan(m.cut_points[:, 3, 3]).all()       # an outside node has none
    assert CM.cut_cells(m) == [(3, 3), (3, 4), (4, 3), (4, 4)]
    # cell (4, 4): corner 0 = node (4, 4) inside, pentagon P_E, (5,4), (5,5), (4,5), P_N
    tri, quad = CM.cut_pieces(m, 4, 4)
    np.testing.assert_array_equal(tri[0], [pts[0], (5.0, 4.0), (5.0, 5.0)])
    assert tri[1] == [0, 1, 2]
    np.testing.assert_array_equal(quad[0], [pts[0], (5.0, 5.0), (4.0, 5.0), pts[1]])
    assert quad[1] == [0, 2, 3, 0]
    # cell (3, 3): node (4, 4) is its corner 2; P+ on edge 2 (towards (3, 4)) is the W point
    tri, quad = CM.cut_pieces(m, 3, 3)
    np.testing.assert_array_equal(tri[0], [pts[2], (3.0, 4.0), (3.0, 3.0)])
    np.testing.assert_array_equal(quad[0], [pts[2], (3.0, 3.0), (4.0, 3.0), pts[3]])
    for (j, i) in CM.cut_cells(m):
        for verts, _ in CM.cut_pieces(m, j, i):
            assert CM.signed_area(verts) > 0


def l_shaped_mesh(S=0, sigma=0.0):
    """h = 1, circle (4.3, 4.3) r = 0.85: nodes (4,4), (5,4), (4,5) inside, (5,5) outside."""
    return CM.build_cut_mesh((0.0, 9.0, 0.0, 9.0, 9, 9), np.array([[4.3, 4.3, 0.85]]), S, sigma=sigma)


def test_triangle_quadrilateral_and_pentagon_cells_by_hand():
    m = l_shaped_mesh()
    assert sorted(zip(*np.nonzero(m.body >= 0))) == [(4, 4), (4, 5), (5, 4)]
    r2 = 0.85 * 0.85
    s = SQ(r2 - 0.49)
    # cell (4, 4): three inside corners -> triangle P((5,4), N), (5,5), P((4,5), E)
    poly = CM.cut_polygon(m, 4, 4)
    assert len(poly) == 3
    np.testing.assert_allclose(poly[0][0], (5.0, 4.3 + s), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(poly[1][0], (5.0, 5.0))
    np.testing.assert_allclose(poly[2][0], (4.3 + s, 5.0), rtol=0, atol=1e-15)
    assert [p[1] for p in poly] == [1, 2, 3]
    # cell (4, 3): corners (4,3) out, (5,3) out, (5,4) in, (4,4) in -> quadrilateral
    poly = CM.cut_polygon(m, 3, 4)
    assert len(poly) == 4
    np.testing.assert_array_equal(poly[0][0], (4.0, 3.0))
    np.testing.assert_array_equal(poly[1][0], (5.0, 3.0))
    s5 = SQ(r2 - 0.49)                                 # node (5, 4): x - cx = 0.7
    s4 = SQ(r2 - 0.09)                                 # node (4, 4): x - cx = -0.3
    np.testing.assert_allclose(poly[2][0], (5.0, 4.3 - s5), rtol=0, atol=1e-15)
    np.testing.assert_allclose(poly[3][0], (4.0, 4.3 - s4), rtol=0, atol=1e-15)
    assert [p[1] for p in poly] == [0, 1, 2, 3]
    # cell (3, 3): only (4, 4) inside -> pentagon
    assert len(CM.cut_polygon(m, 3, 3)) == 5
    M4, dm = CM.cut_cell_matrix(m, 4, 4)
    np.testing.assert_allclose(M4[0], 0.0)             # corner 0 = node (4, 4) takes no part
    np.testing.assert_allclose(M4.sum(axis=1), 0.0, atol=1e-14)
    np.testing.assert_allclose(M4, M4.T, atol=0)
    assert dm > 0


def chord_polygon_area(m, k):
    """Signed area of the loop of chords around body k (negative: clockwise around it)."""
    tot = 0.0
    for (j, i) in CM.cut_cells(m):
        ins = CM.cell_inside(m.body, j, i)
        a = ins.index(True)
        if m.body[j + CM.CJ[a], i + CM.CI[a]] != k:
            continue
        (A, _, _), (B, _, _) = CM.chord(m, j, i)
        tot += 0.5 * (A[0] * B[1] - B[0] * A[1])
    return tot


@pytest.mark.parametrize("S,sigma", [(0, 0.0), (30, 0.0), (30, 0.4)])
def test_pieces_tile_the_box_minus_the_chord_polygons(S, sigma):
    c = W.five_cylinder_case(0.5, 160, 80, S)
    m = CM.build_cut_mesh(c.grid, c.bodies, c.sweeps, c.bc, sigma=sigma)
    x0, x1, y0, y1, nx, ny = c.grid
    total = 0.0
    cut = set(CM.cut_cells(m))
    for j, i in zip(*np.nonzero(m.active)):
        if (j, i) in cut:
            for verts, _ in CM.cut_pieces(m, j, i):
                a = CM.signed_area(verts)
                assert a > 0
                total += a
        else:
            xy = M.cell_coords(m)[j, i]
            total += CM.signed_area(xy)
    holes = [chord_polygon_area(m, k) for k in range(len(c.bodies))]
    assert total == pytest.approx((x1 - x0) * (y1 - y0) + sum(holes), rel=1e-13)
    h = max((x1 - x0) / nx, (y1 - y0) / ny)
    for k, (_, _, r) in enumerate(c.bodies):
        enclosed = -holes[k]
        assert 0 < np.pi * r * r - enclosed <= np.pi * h * h, (k, np.pi * r * r - enclosed)


def test_linear_patch_test_piece_by_piece():
    """Around every FREE node the pieces reproduce a linear field: the rows of the piece
    matrices, applied to the field's values at the piece vertices, sum to zero."""
    c = W.five_cylinder_case(0.25, 128, 64, 24)
    m = CM.build_cut_mesh(c.grid, c.bodies, c.sweeps, c.bc, sigma=0.3)
    lin = lambda xy: 0.3 + 1.7 * xy[:, 0] - 0.9 * xy[:, 1]
    y = np.zeros((m.ny + 1, m.nx + 1))
    cut = set(CM.cut_cells(m))
    for j, i in zip(*np.nonzero(m.active)):
        if (j, i) in cut:
            pieces = CM.cut_pieces(m, j, i)
        else:
            pieces = [(M.cell_coords(m)[j, i], [0, 1, 2, 3])]
        inside = CM.cell_inside(m.body, j, i)
        for verts, cmap in pieces:
            K, _ = CM.piece_stiffness(verts)
            r = K @ lin(np.asarray(verts))
            for a, ca in enumerate(cmap):
                # a surface point stands for an inside corner: not a FREE row
                is_point = inside[ca]
                if not is_point:
                    y[j + CM.CJ[ca], i + CM.CI[ca]] += r[a]
    free = m.kind == M.FREE
    interior = np.zeros_like(free)
    interior[1:-1, 1:-1] = True
    assert np.abs(y[free & interior]).max() <= 1e-12


def exact_cylinder_psi(x, y, a, U=1.0):
    r2 = np.maximum(x * x + y * y, 1e-300)
    return U * y * (1.0 - a * a / r2)


def test_closed_form_cylinder_converges_on_the_cut_mesh():
    """Dirichlet data from psi = U y (1 - a^2/rho^2): C = 0 by symmetry, the nodal error
    falls with order > 1.5 (second order expected)."""
    errs, hs = [], []
    for nx in (64, 128, 256):
        m = CM.build_cut_mesh((-4.0, 4.0, -2.0, 2.0, nx, nx // 2), np.array([[0.0, 0.0, 0.5]]), 3 * nx // 8,
                              sigma=0.25)
        g = exact_cylinder_psi(m.x, m.y, 0.5).ravel()
        sysm = S.assemble(m, g=g)
        u, psi = SV.solve_direct(sysm)
        assert abs(u[-1]) < 1e-11
        free = (m.kind == M.FREE).ravel()
        errs.append(np.abs(psi - exact_cylinder_psi(m.x, m.y, 0.5).ravel())[free].max())
        hs.append(8.0 / nx)
    order = np.log(errs[1] / errs[2]) / np.log(hs[1] / hs[2])
    assert order > 1.5, (errs, order)


def test_signed_surface_velocity_approaches_two_u_sin_theta():
    err = []
    for nx in (128, 256):
        m = CM.build_cut_mesh((-4.0, 4.0, -2.0, 2.0, nx, nx // 2), np.array([[0.0, 0.0, 0.5]]), 3 * nx // 8)
        g = exact_cylinder_psi(m.x, m.y, 0.5).ravel()
        sysm = S.assemble(m, g=g)
        u, psi = SV.solve_direct(sysm)
        th, ut = CM.surface_velocity(m, psi, u[sysm.n_free:], 0)
        assert th.size > 20 and np.all((th >= 0) & (th < 360))
        err.append(np.mean(np.abs(ut - 2.0 * np.sin(np.radians(th)))))
        up = (th > 60) & (th < 120)
        down = (th > 240) & (th < 300)
        assert np.all(ut[up] > 0) and np.all(ut[down] < 0)
    assert err[1] < 0.75 * err[0] and err[1] < 0.3, err


def test_redistribution_identity_circle_and_spacing():
    c = W.five_cylinder_case(0.25, 200, 100, 20)
    m0 = CM.build_cut_mesh(c.grid, c.bodies, c.sweeps, c.bc, sigma=0.0)
    mz = CM.build_cut_mesh(c.grid, c.bodies, c.sweeps, c.bc, sigma=0.0)
    np.testing.assert_array_equal(np.nan_to_num(m0.cut_points, nan=7.0), np.nan_to_num(mz.cut_points, nan=7.0))
    sigma = 0.4
    m1 = CM.build_cut_mesh(c.grid, c.bodies, c.sweeps, c.bc, sigma=sigma)
    hmin = min((c.grid[1] - c.grid[0]) / c.grid[4], (c.grid[3] - c.grid[2]) / c.grid[5])
    smin = sigma * hmin
    ok = ~np.isnan(m1.cut_points[..., 0])
    assert np.array_equal(ok, ~np.isnan(m0.cut_points[..., 0]))
    for d in range(4):
        js, is_ = np.nonzero(ok[d])
        for j, i in zip(js, is_):
            cx, cy, r = c.bodies[m1.body[j, i]]
            p = m1.cut_points[d, j, i]
            assert abs(np.hypot(p[0] - cx, p[1] - cy) - r) <= 4e-16 * r * 4
    L0 = np.array([np.hypot(*(B - A)) for (A, _, _), (B, _, _) in (CM.chord(m0, j, i) for j, i in CM.cut_cells(m0))])
    L1 = np.array([np.hypot(*(B - A)) for (A, _, _), (B, _, _) in (CM.chord(m1, j, i) for j, i in CM.cut_cells(m1))])
    short = (L0 > 0) & (L0 < smin)
    assert short.sum() > 5
    assert np.all(L1[short] > L0[short])
    assert np.all(L1[short] > 0.95 * smin)            # one pass brings an isolated short chord to ~s_min
    assert np.count_nonzero(m1.cut_points[ok[..., None].repeat(2, -1)] != m0.cut_points[ok[..., None].repeat(2, -1)]) > 0


def test_saddle_and_two_body_cells_are_refused():
    # two circles one cell apart on the diagonal: a cell with two diagonal inside corners
    with pytest.raises(M.MeshError, match="diagonal"):
        CM.build_cut_mesh((0.0, 12.0, 0.0, 12.0, 12, 12), np.array([[5.0, 5.0, 0.3], [6.0, 6.0, 0.3]]), 0)
    # side by side: a cell with inside corners of both
    with pytest.raises(M.MeshError, match="two bodies"):
        CM.build_cut_mesh((0.0, 12.0, 0.0, 12.0, 12, 12), np.array([[5.0, 5.0, 0.3], [6.0, 5.0, 0.3]]), 0)


def test_free_node_coordinates_follow_the_directional_smoothing_by_hand():
    """One sweep by hand on the single-inside-node layout: the east neighbour (5, 4) of the
    split node averages its four neighbours, the split node contributing its E point."""
    m1 = single_inside_node_mesh(S=1)
    m0 = single_inside_node_mesh(S=0)
    pE = m0.cut_points[0, 4, 4]
    dx = (((pE[0] - 4.0) + 0.0) + 0.0) + 0.0
    assert m1.x[4, 5] == 5.0 + dx / 4.0
    assert m1.y[4, 5] == 4.0                           # the E point lies on the row: no y move
    assert m1.x[4, 4] == 4.0 and m1.y[4, 4] == 4.0     # BODY nodes keep the background position


# ---------------------------------------------------------------- polygon bodies
from oracle import shapes as SH  # noqa: E402


def test_polygon_surface_points_by_hand():
    """The square [2.5, 5.5]^2 on a unit grid: inside nodes 3..5 both ways; every surface
    point lies on a side of the square, and the corner node (5, 5) splits into (5.5, 5)
    and (5, 5.5)."""
    sq = W.PolygonBody([(2.5, 2.5), (5.5, 2.5), (5.5, 5.5), (2.5, 5.5)], ref=(4.0, 4.0))
    m = CM.build_cut_mesh((0.0, 10.0, 0.0, 10.0, 10, 10), np.zeros((0, 3)), 0, polygons=[sq])
    assert sorted(zip(*np.nonzero(m.body >= 0))) == [(j, i) for j in (3, 4, 5) for i in (3, 4, 5)]
    np.testing.assert_array_equal(m.cut_points[0, 5, 5], (5.5, 5.0))
    np.testing.assert_array_equal(m.cut_points[1, 5, 5], (5.0, 5.5))
    np.testing.assert_array_equal(m.cut_points[2, 4, 3], (2.5, 4.0))
    np.testing.assert_array_equal(m.cut_points[3, 3, 4], (4.0, 2.5))
    assert np.isnan(m.cut_points[:, 4, 4]).all()             # (4, 4) has no outside neighbour
    assert len(CM.cut_polygon(m, 5, 5)) == 5                 # cell (5, 5): one inside corner


def _polygon_cut(kind, nx, sweeps, sigma):
    if kind == "ellipse":
        body = W.ellipse_body(0.8, 0.4, 720, angle=-np.radians(10.0))
        grid = (-4.0, 4.0, -2.0, 2.0, nx, nx // 2)
    else:
        body = W.joukowski_airfoil(0.5, 0.08, 400, alpha=np.radians(6.0))
        grid = (-3.0, 3.0, -1.5, 1.5, nx, nx // 2)
    return body, CM.build_cut_mesh(grid, np.zeros((0, 3)), sweeps, polygons=[body], sigma=sigma)


@pytest.mark.parametrize("kind", ["ellipse", "airfoil"])
def test_polygon_cut_mesh_tiles_and_points_on_the_boundary(kind):
    body, m = _polygon_cut(kind, 192, 40, 0.3)
    x0, x1, y0, y1 = m.xg[0, 0], m.xg[0, -1], m.yg[0, 0], m.yg[-1, 0]
    total = 0.0
    cut = set(CM.cut_cells(m))
    for j, i in zip(*np.nonzero(m.active)):
        if (j, i) in cut:
            for verts, _ in CM.cut_pieces(m, j, i):
                a = CM.signed_area(verts)
                assert a > 0
                total += a
        else:
            total += CM.signed_area(M.cell_coords(m)[j, i])
    hole = chord_polygon_area(m, 0)
    assert total == pytest.approx((x1 - x0) * (y1 - y0) + hole, rel=1e-12)
    assert -hole == pytest.approx(SH.signed_area(body.vertices), rel=0.01)
    ok = ~np.isnan(m.cut_points[..., 0])
    pts = m.cut_points[ok]
    qx, qy = SH.nearest_on_polygon(pts[:, 0], pts[:, 1], body.vertices)
    assert np.hypot(pts[:, 0] - qx, pts[:, 1] - qy).max() <= 1e-14
    if kind == "airfoil":
        n = m.wake_node[0]
        T, _, Wp = SH.kutta_points(body, 6.0 / 192)
        assert m.x.ravel()[n] == Wp[0] and m.y.ravel()[n] == Wp[1]


def test_ellipse_flow_converges_on_the_polygon_cut_mesh():
    a, b, alpha = 0.8, 0.4, np.radians(10.0)
    errs = []
    for nx in (96, 192):
        _, m = _polygon_cut("ellipse", nx, nx // 4, 0.25)
        g = SH.ellipse_psi(m.x.ravel(), m.y.ravel(), a, b, 1.0, alpha)
        u, psi = SV.solve_direct(S.assemble(m, g=g))
        errs.append(np.abs(psi - g)[(m.kind == M.FREE).ravel()].max())
        assert abs(u[-1]) < 1e-10
    assert errs[1] < 0.6 * errs[0], errs


def test_kutta_circulation_on_the_polygon_cut_mesh():
    """The Joukowski airfoil at 6 degrees with the exact Kutta data: the body value
    converges to the exact one (error halving per refinement, below 1e-3 at 512 x 256)."""
    errs = []
    for nx in (128, 256, 512):
        af, m = _polygon_cut("airfoil", nx, nx // 4, 0.25)
        g, psi_b = SH.joukowski_psi(m.x.ravel(), m.y.ravel(), af, 1.0, kutta=True)
        s = S.assemble(m, g=g)
        u, _ = SV.solve_kutta(s, m)
        errs.append(abs(u[s.n_free] - psi_b))
    assert errs[2] < 0.6 * errs[1] < 0.36 * errs[0] and errs[2] < 1e-3, errs


def exact_cylinder_velocity(x, y, a, U=1.0):
    """(u, v) = (dpsi/dy, -dpsi/dx) of psi = U y (1 - a^2 / rho^2)."""
    r2 = x * x + y * y
    u = U * (1.0 - a * a * (x * x - y * y) / (r2 * r2))
    v = -U * 2.0 * a * a * x * y / (r2 * r2)
    return u, v


def test_cut_cell_velocity_approaches_the_exact_flow():
    """Element velocity of the cut cells (area-weighted mean of the pieces' gradients) on the
    exact-data cylinder: the error against the exact velocity at the cell's vertex centroid
    falls under refinement (first order at the boundary), and a mix-up of the pieces'
    gradients (say the triangle's b and c exchanged) would not converge."""
    errs = []
    for nx in (128, 256):
        m = CM.build_cut_mesh((-4.0, 4.0, -2.0, 2.0, nx, nx // 2), np.array([[0.0, 0.0, 0.5]]), 3 * nx // 8,
                              sigma=0.25)
        g = exact_cylinder_psi(m.x, m.y, 0.5).ravel()
        sysm = S.assemble(m, g=g)
        _, psi = SV.solve_direct(sysm)
        uu, vv = CM.velocity_field(m, psi)
        pos = -np.ones((m.ny, m.nx), dtype=np.int64)
        pos[m.active] = np.arange(int(m.active.sum()))
        e = []
        for (j, i) in CM.cut_cells(m):
            V = np.array([p[0] for p in CM.cut_polygon(m, j, i)])
            ue, ve = exact_cylinder_velocity(V[:, 0].mean(), V[:, 1].mean(), 0.5)
            e.append(np.hypot(uu[pos[j, i]] - ue, vv[pos[j, i]] - ve))
        errs.append(np.mean(e))
    assert errs[1] < 0.75 * errs[0] and errs[1] < 0.2, errs


def test_three_solution_routes_agree_on_a_small_cut_mesh():
    """Dense Cholesky (which needs the cut-cell system to be symmetric positive definite),
    sparse LU and the element-by-element CG of Appendix A agree on a small mixed-cell mesh
    with two bodies, one of them a polygon."""
    sq = W.PolygonBody([(1.0, -0.6), (1.9, -0.6), (1.9, 0.5), (1.0, 0.5)], ref=(1.45, 0.0))
    m = CM.build_cut_mesh((-3.0, 3.0, -2.0, 2.0, 36, 24), np.array([[-1.0, 0.2, 0.7]]), 9, polygons=[sq],
                          sigma=0.3)
    sysm = S.assemble(m, 1.3)
    A = sysm.A.toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    u1, psi1 = SV.solve_direct(sysm, dense=True)
    u2, psi2 = SV.solve_direct(sysm)
    np.testing.assert_allclose(psi1, psi2, rtol=0, atol=1e-12)
    x, psik, it, _ = SV.cg_paper(sysm, m.kind.ravel(), m.body.ravel(), tol=1e-14, criterion="relative")
    assert it > 10
    np.testing.assert_allclose(x, psi2, rtol=0, atol=1e-10)
    np.testing.assert_allclose(psik, u2[sysm.n_free:], rtol=0, atol=1e-10)
