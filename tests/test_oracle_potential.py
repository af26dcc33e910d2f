"""Pins of the oracle's velocity potential phi and element velocities.

Closed forms (linear patch test, the uniform stream, potential flow past a cylinder with
second-order nodal convergence), invariants (antisymmetry of a centred cylinder, flux
balance between inlet and outlet), the flow net (velocities from phi and from psi agree,
and both converge to the exact flow) and a brute-force loop assembly on a tiny mesh."""
import numpy as np

from oracle import element as E, mesh as M, potential as PO, solve as SV, system as S
from paper_2512_12232_gb300 import workloads as W


def distorted_mesh_without_bodies(nx=20, ny=14, seed=0, amp=0.3):
    m = M.build_mesh((0.0, 2.0, -1.0, 0.4, nx, ny), np.zeros((0, 3)), 0)
    rng = np.random.default_rng(seed)
    hx, hy = 2.0 / nx, 1.4 / ny
    m.x[1:-1, 1:-1] += rng.uniform(-amp, amp, (ny - 1, nx - 1)) * hx
    m.y[1:-1, 1:-1] += rng.uniform(-amp, amp, (ny - 1, nx - 1)) * hy
    return m


def cylinder_mesh(nx, a=0.5):
    c = W.Case(-4.0, 4.0, -2.0, 2.0, nx, nx // 2, np.array([[0.0, 0.0, a]]), 3 * nx // 8)
    return M.build_mesh(c.grid, c.bodies, c.sweeps, c.bc)


def exact_phi(x, y, a, U=1.0):
    r2 = x * x + y * y
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(r2 > 0, U * x * (1.0 + a * a / r2), 0.0)   # r = 0 only at an inactive node


def exact_psi(x, y, a, U=1.0):
    r2 = x * x + y * y
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(r2 > 0, U * y * (1.0 - a * a / r2), 0.0)


def exact_velocity(x, y, a, U=1.0):
    r2 = x * x + y * y
    return U * (1.0 + a * a * (y * y - x * x) / r2 ** 2), -2.0 * U * a * a * x * y / r2 ** 2


def test_linear_patch_test_on_distorted_mesh():
    """Dirichlet data of a linear field on the outer ring: phi_h equals it everywhere."""
    m = distorted_mesh_without_bodies()
    g = (0.7 * m.x - 1.9 * m.y + 0.3).ravel()
    s = PO.assemble_phi(m, dirichlet=PO.ring_mask(m), g=g)
    phi = PO.solve_phi(s)
    np.testing.assert_allclose(phi, g, rtol=0, atol=1e-13)
    u, v = PO.velocity_from_phi(m, phi)
    np.testing.assert_allclose(u, 0.7, rtol=0, atol=1e-12)
    np.testing.assert_allclose(v, -1.9, rtol=0, atol=1e-12)


def test_uniform_stream_without_bodies():
    """phi = U x on inlet and outlet, no flux through the other sides: the exact solution
    is the uniform stream phi = U x (it has zero normal derivative on y = const)."""
    m = distorted_mesh_without_bodies(seed=3)
    U = 1.7
    phi = PO.solve_phi(PO.assemble_phi(m, U=U))
    np.testing.assert_allclose(phi, U * m.x.ravel(), rtol=0, atol=1e-12)
    u, v = PO.velocity_from_phi(m, phi)
    np.testing.assert_allclose(u, U, rtol=0, atol=1e-11)
    np.testing.assert_allclose(v, 0.0, rtol=0, atol=1e-11)


def test_brute_force_assembly_on_a_tiny_mesh():
    """The vectorised assembly against plain loops over cells and corners."""
    c = W.Case(-3.0, 3.0, -2.0, 2.0, 12, 8, np.array([[0.2, 0.1, 0.9]]), 5)
    m = M.build_mesh(c.grid, c.bodies, c.sweeps, c.bc)
    U = 1.3
    s = PO.assemble_phi(m, U=U)
    kind = m.kind.ravel()
    N = m.n_nodes
    xs, ys = m.x.ravel(), m.y.ravel()
    dirichlet = np.zeros(N, dtype=bool)
    for n in range(N):
        i = n % (m.nx + 1)
        dirichlet[n] = (i == 0 or i == m.nx) and kind[n] != M.INACTIVE
    idx, k = {}, 0
    for n in range(N):
        if kind[n] != M.INACTIVE and not dirichlet[n]:
            idx[n] = k
            k += 1
    A = np.zeros((k, k))
    b = np.zeros(k)
    for j in range(m.ny):
        for i in range(m.nx):
            if not m.active[j, i]:
                continue
            corners = [j * (m.nx + 1) + i, j * (m.nx + 1) + i + 1, (j + 1) * (m.nx + 1) + i + 1,
                       (j + 1) * (m.nx + 1) + i]
            xy = np.array([[xs[n], ys[n]] for n in corners])
            Ke, _ = E.q4_stiffness(xy)
            for a_, na in enumerate(corners):
                if na not in idx:
                    continue
                for b_, nb in enumerate(corners):
                    if nb in idx:
                        A[idx[na], idx[nb]] += Ke[a_, b_]
                    elif dirichlet[nb]:
                        b[idx[na]] -= Ke[a_, b_] * U * xs[nb]
    np.testing.assert_allclose(s.A.toarray(), A, rtol=0, atol=1e-13)
    np.testing.assert_allclose(s.b, b, rtol=0, atol=1e-13)
    assert (m.kind == M.BODY).any() and all(s.dof[n] >= 0 for n in np.flatnonzero(kind == M.BODY))


def test_closed_form_cylinder_second_order_convergence():
    """Dirichlet data from phi = U x (1 + a^2/r^2) on the outer ring and no flux through the
    cylinder (exact: d phi/dr = 0 at r = a): the nodal error falls with order ~2."""
    errs, hs = [], []
    for nx in (64, 128, 256):
        m = cylinder_mesh(nx)
        ex = exact_phi(m.x, m.y, 0.5).ravel()
        s = PO.assemble_phi(m, dirichlet=PO.ring_mask(m), g=ex)
        phi = PO.solve_phi(s)
        live = (m.kind != M.INACTIVE).ravel()
        errs.append(np.abs(phi - ex)[live].max())
        hs.append(8.0 / nx)
    order = np.log(errs[1] / errs[2]) / np.log(hs[1] / hs[2])
    assert order > 1.7, (errs, order)


def test_centred_cylinder_is_antisymmetric_in_x():
    """With phi = U x on x = +-L the solution is odd in x: phi(-x, y) = -phi(x, y)."""
    m = cylinder_mesh(64)
    phi = PO.solve_phi(PO.assemble_phi(m, U=1.0)).reshape(m.ny + 1, m.nx + 1)
    live = m.kind != M.INACTIVE
    assert np.array_equal(live, live[:, ::-1])
    scale = np.abs(phi).max()
    np.testing.assert_allclose(phi[live], -phi[:, ::-1][live], rtol=0, atol=1e-12 * scale)


def test_flux_balance_between_inlet_and_outlet():
    """Columns of K sum to zero and the unknowns' rows are solved, so the flux entering at
    the inlet leaves at the outlet; both are U times the channel height up to blockage."""
    c = W.five_cylinder_case(0.5, 160, 80, 20)
    m = M.build_mesh(c.grid, c.bodies, c.sweeps, c.bc)
    U = 1.0
    s = PO.assemble_phi(m, U=U)
    phi = PO.solve_phi(s)
    r = PO.nodal_residual(s, phi)
    i = np.arange(m.n_nodes) % (m.nx + 1)
    inlet = r[s.dirichlet & (i == 0)].sum()
    outlet = r[s.dirichlet & (i == m.nx)].sum()
    assert abs(np.abs(r[s.dof >= 0]).max()) < 1e-10
    assert abs(inlet + outlet) <= 1e-10 * abs(inlet)
    H = c.grid[3] - c.grid[2]
    assert 0.5 * U * H < abs(inlet) < 1.01 * U * H


def test_flow_net_velocities_agree_and_converge():
    """The velocity from phi (grad phi) and from psi ((dpsi/dy, -dpsi/dx)), both with
    closed-form Dirichlet data around a cylinder, approach the exact flow and each other."""
    d_pp, d_ex = [], []
    for nx in (64, 128):
        m = cylinder_mesh(nx)
        g_phi = exact_phi(m.x, m.y, 0.5).ravel()
        phi = PO.solve_phi(PO.assemble_phi(m, dirichlet=PO.ring_mask(m), g=g_phi))
        sp = S.assemble(m, g=exact_psi(m.x, m.y, 0.5).ravel())
        _, psi = SV.solve_direct(sp)
        uf, vf = PO.velocity_from_phi(m, phi)
        us, vs = PO.velocity_from_psi(m, psi)
        _, _, cx, cy = PO.element_gradient(m, phi)
        ue, ve = exact_velocity(cx, cy, 0.5)
        d_pp.append(np.sqrt(np.mean((uf - us) ** 2 + (vf - vs) ** 2)))
        d_ex.append(np.sqrt(np.mean((uf - ue) ** 2 + (vf - ve) ** 2)))
    assert d_pp[1] < 0.6 * d_pp[0] and d_pp[1] < 0.05, d_pp
    assert d_ex[1] < 0.6 * d_ex[0] and d_ex[1] < 0.05, d_ex
