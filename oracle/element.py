"""Oracle: bilinear quadrilateral (Q4) element stiffness.

Section "Weak formulation": K_e = int_{Omega_e} (grad N)^T (grad N) dOmega with the
element shape functions N.  The paper does not state the quadrature; this uses
the standard 2x2 Gauss rule (points +-1/sqrt(3), unit weights), which integrates
the bilinear element exactly on parallelograms.

Isoparametric map: N_a(xi, eta) = (1 + xi_a xi)(1 + eta_a eta)/4 with reference
corners (-1,-1), (1,-1), (1,1), (-1,1) matching the counter-clockwise cell corners
(i,j), (i+1,j), (i+1,j+1), (i,j+1).  J = d(x,y)/d(xi,eta), grad N = J^{-1} dN/d(xi,eta),
K_e = sum_g det J_g B_g^T B_g.

Written for any numpy dtype so that the same code evaluates complex-step
derivatives (coordinates perturbed by i*h).
"""
from __future__ import annotations

import numpy as np

XI_A = np.array([-1.0, 1.0, 1.0, -1.0])
ETA_A = np.array([-1.0, -1.0, 1.0, 1.0])
_G = 1.0 / np.sqrt(3.0)
GAUSS_2x2 = ((-_G, -_G), (_G, -_G), (_G, _G), (-_G, _G))


def shape_derivatives(xi, eta):
    """dN_a/dxi and dN_a/deta at (xi, eta) for the four corners."""
    dxi = XI_A * (1.0 + ETA_A * eta) / 4.0
    deta = ETA_A * (1.0 + XI_A * xi) / 4.0
    return dxi, deta


def q4_stiffness(xy):
    """K_e for corner coordinates xy[..., 4, 2]; returns (..., 4, 4) and the
    minimum det J over the Gauss points (..., )."""
    xy = np.asarray(xy)
    x = xy[..., 0]
    y = xy[..., 1]
    K = np.zeros(xy.shape[:-2] + (4, 4), dtype=xy.dtype)
    detmin = None
    for xi, eta in GAUSS_2x2:
        dxi, deta = shape_derivatives(xi, eta)
        j00 = x @ dxi      # dx/dxi
        j01 = y @ dxi      # dy/dxi
        j10 = x @ deta     # dx/deta
        j11 = y @ deta     # dy/deta
        det = j00 * j11 - j01 * j10
        # grad N = J^{-1} [dN/dxi; dN/deta], J = [[j00, j01], [j10, j11]]
        dndx = (j11[..., None] * dxi - j01[..., None] * deta) / det[..., None]
        dndy = (-j10[..., None] * dxi + j00[..., None] * deta) / det[..., None]
        K = K + det[..., None, None] * (dndx[..., :, None] * dndx[..., None, :]
                                        + dndy[..., :, None] * dndy[..., None, :])
        dr = np.real(det)
        detmin = dr if detmin is None else np.minimum(detmin, dr)
    return K, detmin


def rectangle_closed_form(hx, hy):
    """Textbook closed form of K_e for an axis-aligned hx-by-hy rectangle
    (used as an independent pin of `q4_stiffness`)."""
    b = hy / hx
    a = hx / hy
    Kx = np.array([[2, -2, -1, 1], [-2, 2, 1, -1], [-1, 1, 2, -2], [1, -1, -2, 2]], dtype=float)
    Ky = np.array([[2, 1, -1, -2], [1, 2, -2, -1], [-1, -2, 2, 1], [-2, -1, 1, 2]], dtype=float)
    return (b / 6.0) * Kx + (a / 6.0) * Ky


def stiffness_shape_derivative(xy, step=1e-30):
    """dK_e/dx_{a,c} for every corner a and component c by the complex step
    Im K(x + i*step*e_{a,c}) / step; returns (..., 4, 2, 4, 4)."""
    xy = np.asarray(xy, dtype=np.float64)
    out = np.zeros(xy.shape[:-2] + (4, 2, 4, 4))
    for a in range(4):
        for c in range(2):
            z = xy.astype(np.complex128)
            z[..., a, c] += 1j * step
            Kz, _ = q4_stiffness(z)
            out[..., a, c, :, :] = Kz.imag / step
    return out
