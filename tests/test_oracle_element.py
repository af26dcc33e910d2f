"""Pins of the oracle's Q4 element stiffness (section "Weak formulation")."""
import numpy as np
import pytest

from oracle.element import (q4_stiffness, rectangle_closed_form, stiffness_shape_derivative)


def random_quads(n, seed=0, distort=0.25):
    """Unit-ish squares with corners jittered: convex, det J > 0."""
    rng = np.random.default_rng(seed)
    base = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=float)
    q = base[None] + rng.uniform(-distort, distort, size=(n, 4, 2))
    scale = rng.uniform(0.01, 10.0, size=(n, 1, 1))
    shift = rng.uniform(-50, 50, size=(n, 1, 2))
    return q * scale + shift


@pytest.mark.parametrize("hx,hy", [(1.0, 1.0), (2.0, 1.0), (0.15625, 0.15625), (0.3, 0.05)])
def test_rectangle_matches_textbook_closed_form(hx, hy):
    xy = np.array([[0, 0], [hx, 0], [hx, hy], [0, hy]], dtype=float) + np.array([3.7, -1.2])
    K, detmin = q4_stiffness(xy)
    np.testing.assert_allclose(K, rectangle_closed_form(hx, hy), rtol=0, atol=1e-14 * max(hx / hy, hy / hx))
    assert detmin == pytest.approx(hx * hy / 4)


def test_square_is_scale_invariant_textbook_matrix():
    K, _ = q4_stiffness(np.array([[0, 0], [7.0, 0], [7, 7], [0, 7]]))
    ref = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    np.testing.assert_allclose(K, ref, atol=1e-15)


def test_row_sums_zero_symmetric_psd_constant_nullspace():
    xy = random_quads(200)
    K, detmin = q4_stiffness(xy)
    assert np.all(detmin > 0)
    scale = np.abs(K).max(axis=(1, 2))
    assert np.abs(K.sum(axis=2)).max(axis=1).max() <= 1e-13 * scale.max()
    np.testing.assert_allclose(K, np.swapaxes(K, 1, 2), atol=1e-14 * scale.max())
    w = np.linalg.eigvalsh(K)
    assert np.all(np.abs(w[:, 0]) <= 1e-12 * w[:, -1])     # one zero eigenvalue (constants)
    assert np.all(w[:, 1] > 1e-6 * w[:, -1])               # the rest strictly positive


def test_rigid_motion_and_scale_invariance():
    xy = random_quads(50, seed=3)
    K, _ = q4_stiffness(xy)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    K2, _ = q4_stiffness(xy @ R.T + np.array([11.0, -4.0]))
    np.testing.assert_allclose(K2, K, atol=1e-12 * np.abs(K).max())
    K3, _ = q4_stiffness(xy * 13.0)
    np.testing.assert_allclose(K3, K, atol=1e-12 * np.abs(K).max())


def test_parallelogram_two_point_rule_is_exact():
    """On a parallelogram the integrand of K_e is polynomial in (xi, eta) of degree 2
    per variable; a 5x5 Gauss rule evaluated independently must agree."""
    xy = np.array([[0, 0], [2.0, 0.3], [2.5, 1.8], [0.5, 1.5]])
    K, _ = q4_stiffness(xy)
    pts, wts = np.polynomial.legendre.leggauss(5)
    xia = np.array([-1, 1, 1, -1.0])
    etaa = np.array([-1, -1, 1, 1.0])
    K5 = np.zeros((4, 4))
    for xi, wx in zip(pts, wts):
        for eta, wy in zip(pts, wts):
            dxi = xia * (1 + etaa * eta) / 4
            deta = etaa * (1 + xia * xi) / 4
            J = np.array([[dxi @ xy[:, 0], dxi @ xy[:, 1]], [deta @ xy[:, 0], deta @ xy[:, 1]]])
            G = np.linalg.solve(J, np.vstack([dxi, deta]))
            K5 += wx * wy * np.linalg.det(J) * G.T @ G
    np.testing.assert_allclose(K, K5, atol=1e-14)


def test_complex_step_derivative_matches_central_differences():
    xy = random_quads(5, seed=7)
    dK = stiffness_shape_derivative(xy)
    h = 1e-6
    for a in range(4):
        for c in range(2):
            p = xy.copy(); p[:, a, c] += h
            m = xy.copy(); m[:, a, c] -= h
            fd = (q4_stiffness(p)[0] - q4_stiffness(m)[0]) / (2 * h)
            np.testing.assert_allclose(dK[:, a, c], fd, atol=1e-7 * np.abs(fd).max() + 1e-9)
    # translation invariance: derivatives summed over corners vanish
    np.testing.assert_allclose(dK.sum(axis=1), 0.0, atol=1e-10 * np.abs(dK).max())
