"""Oracle: surface tangential velocity, flow rate between bodies and CoPFI.

Section "Velocity Field and Surface Tangential Velocity": u_t ~ (psi_c - psi_b) / d_nc
with psi_b the body's stream-function value, psi_c the average psi of the adjacent
fluid element and d_nc the perpendicular distance from the element centroid to the
boundary edge.  Readings where the paper is silent: a boundary edge is an edge of an
active cell whose two end nodes are BODY nodes of the same body at distinct
positions; the centroid is the mean of the four corners; u_t keeps its sign;
theta is the polar angle of the edge midpoint about the body centre in degrees,
in [0, 360), counter-clockwise from +x.  Edges are listed in cell order (row j,
then column i) and, within a cell, by the edge's first corner 0..3.

Section "Effect of Gap Ratio": Q54 = psi_5 - psi_4 and CoPFI = Q54 / delta with
delta = h_c / h_d.  With total flow U*h_d this is Q / (U * h_c); the general form
used here is CoPFI = (C_hi - C_lo) / (U * (cy_hi - cy_lo)).
"""
from __future__ import annotations

import numpy as np

from .mesh import BODY, Mesh, cell_nodes


def boundary_edges(mesh: Mesh, k: int):
    """(cell j, cell i, edge a) of every boundary edge of body k, in output order."""
    nx, ny = mesh.nx, mesh.ny
    kind = mesh.kind.ravel()
    body = mesh.body.ravel()
    X = mesh.x.ravel()
    Y = mesh.y.ravel()
    cn = cell_nodes(nx, ny)
    out = []
    js, is_ = np.nonzero(mesh.active)
    wake = mesh.wake.ravel() if mesh.wake is not None else np.zeros(kind.shape, dtype=bool)
    for j, i in zip(js, is_):                      # row-major order
        nodes = cn[j, i]
        for a in range(4):
            na, nb_ = nodes[a], nodes[(a + 1) % 4]
            if (kind[na] == BODY and kind[nb_] == BODY and body[na] == k and body[nb_] == k
                    and not wake[na] and not wake[nb_]
                    and (X[na] != X[nb_] or Y[na] != Y[nb_])):
                out.append((j, i, a))
    return out


def surface_velocity(mesh: Mesh, psi: np.ndarray, C: np.ndarray, k: int):
    """Returns arrays theta_deg, u_t for body k in output order."""
    X = mesh.x.ravel()
    Y = mesh.y.ravel()
    cn = cell_nodes(mesh.nx, mesh.ny)
    cx, cy, _ = mesh.bodies[k]
    th, ut = [], []
    for (j, i, a) in boundary_edges(mesh, k):
        nodes = cn[j, i]
        psic = psi[nodes].mean()
        gx = X[nodes].mean()
        gy = Y[nodes].mean()
        na, nb_ = nodes[a], nodes[(a + 1) % 4]
        ex, ey = X[nb_] - X[na], Y[nb_] - Y[na]
        dnc = abs(ex * (gy - Y[na]) - ey * (gx - X[na])) / np.hypot(ex, ey)
        ut.append((psic - C[k]) / dnc)
        mx = 0.5 * (X[na] + X[nb_])
        my = 0.5 * (Y[na] + Y[nb_])
        t = np.degrees(np.arctan2(my - cy, mx - cx))
        th.append(t + 360.0 if t < 0 else t)
    return np.array(th), np.array(ut)


def copfi(C, bodies, lo, hi, U):
    """(CoPFI, Q) for the body pair (lo, hi)."""
    q = C[hi] - C[lo]
    return q / (U * (bodies[hi][1] - bodies[lo][1])), q
