"""torch.autograd bridge for the adjoint shape gradients of CoPFI / transverse-gap flow.

Two ways in, both ending in the library's adjoint solve and shape-derivative kernels
(pf_grad); the Python side only marshals tensors:

* `objective(centres, ...)`: J as a function of the body centres.  Forward builds the
  body-conforming mesh for the centres, solves for psi and returns J (CoPFI or
  C_hi - C_lo); backward returns dJ/dc through the mesh generator.
* `mesh_coords(centres, ...)` and `objective_at_coords(X, centres, ...)`: the same chain
  split at the node coordinates, so that X is a differentiable tensor of its own.
  `mesh_coords` returns the smoothed node coordinates X(c) (backward: the mesh
  generator's vector-Jacobian product, pf_coords_vjp); `objective_at_coords` solves on the
  given coordinates X (pf_mesh_set_coords, topology of the centres' mesh) and returns J
  (backward: dJ/dX from the adjoint, and the objective's own dependence on the centres,
  which CoPFI has through its normalisation U (cy_hi - cy_lo)).
  `objective_at_coords(mesh_coords(c), c)` has the same value and centre gradient as
  `objective(c)`, and X.grad holds dJ/dX; any differentiable map may sit between them.

Topology (which nodes are inside which body) is fixed by the centres, so gradients are
those of the discrete objective at fixed topology."""
from __future__ import annotations

import numpy as np
import torch

from . import api


def _bodies(centres, radii):
    c = centres.detach().cpu().numpy().astype(np.float64).reshape(-1, 2)
    r = np.asarray(radii, dtype=np.float64).reshape(-1, 1)
    return np.concatenate([c, r], axis=1)


class ObjectiveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, centres, radii, grid, sweeps, bc, U, lo, hi, objective, tol):
        with api.mesh_build(grid, _bodies(centres, radii), sweeps, bc) as mesh:
            api.psi_solve(mesh, U=U, tol=tol, precision=api.PF_MIXED)
            _, dJdc, J = api.grad(mesh, objective, lo, hi, U, tol, want_dX=False)
        ctx.save_for_backward(torch.from_numpy(dJdc).to(centres.dtype))
        return centres.new_tensor(float(J[0]))

    @staticmethod
    def backward(ctx, gJ):
        (dJdc,) = ctx.saved_tensors
        return (gJ.cpu() * dJdc).to(gJ.device) if gJ.is_cuda else gJ * dJdc, \
            None, None, None, None, None, None, None, None, None


class MeshCoordsFn(torch.autograd.Function):
    """centres -> X, the final (smoothed) node coordinates of the body-conforming mesh."""

    @staticmethod
    def forward(ctx, centres, radii, grid, sweeps, bc):
        mesh = api.mesh_build(grid, _bodies(centres, radii), sweeps, bc)
        ctx.mesh = mesh                          # the generator's transpose runs on this handle
        ctx.centres_meta = (centres.dtype, centres.device)
        return mesh.coords(0)

    @staticmethod
    def backward(ctx, gX):
        dtype, device = ctx.centres_meta
        gc = ctx.mesh.coords_vjp(gX.contiguous())
        return torch.from_numpy(gc).to(dtype=dtype, device=device), None, None, None, None


class ObjectiveAtCoordsFn(torch.autograd.Function):
    """(X, centres) -> J on the mesh whose topology the centres give and whose node
    coordinates are X."""

    @staticmethod
    def forward(ctx, X, centres, radii, grid, sweeps, bc, U, lo, hi, objective, tol):
        with api.mesh_build(grid, _bodies(centres, radii), sweeps, bc) as mesh:
            if mesh.set_coords(X.detach()) != 0:
                raise ValueError("the given node coordinates fold a cell (det J <= 0)")
            api.psi_solve(mesh, U=U, tol=tol, precision=api.PF_MIXED)
            dJdX, dJdc, J = api.grad(mesh, objective, lo, hi, U, tol, want_dX=True)
            # pf_grad's dJ/dc is the generator's transpose applied to dJ/dX plus the
            # objective's own dependence on the centres; keep the latter only
            explicit = dJdc - mesh.coords_vjp(dJdX)
        ctx.save_for_backward(dJdX.to(X.device, X.dtype), torch.from_numpy(explicit).to(centres.dtype))
        ctx.centres_device = centres.device
        return X.new_tensor(float(J[0]))

    @staticmethod
    def backward(ctx, gJ):
        dJdX, explicit = ctx.saved_tensors
        gX = gJ.to(dJdX.device) * dJdX
        gc = (gJ.detach().cpu() * explicit).to(ctx.centres_device)
        return gX, gc, None, None, None, None, None, None, None, None, None


def objective(centres: torch.Tensor, radii, grid, sweeps, bc=(0, 0, 0, 0), U=1.0, lo=3, hi=4,
              kind=api.PF_OBJ_COPFI, tol=1e-12) -> torch.Tensor:
    """J(centres) with autograd support; centres is an (n_bodies, 2) float64 tensor."""
    return ObjectiveFn.apply(centres, radii, grid, sweeps, bc, U, lo, hi, kind, tol)


def mesh_coords(centres: torch.Tensor, radii, grid, sweeps, bc=(0, 0, 0, 0)) -> torch.Tensor:
    """X(centres): the (nodes, 2) float64 CUDA tensor of final node coordinates, with
    autograd support back to the centres."""
    return MeshCoordsFn.apply(centres, radii, grid, sweeps, bc)


def objective_at_coords(X: torch.Tensor, centres: torch.Tensor, radii, grid, sweeps, bc=(0, 0, 0, 0), U=1.0,
                        lo=3, hi=4, kind=api.PF_OBJ_COPFI, tol=1e-12) -> torch.Tensor:
    """J on node coordinates X (topology from the centres' mesh), with autograd support to X
    (dJ/dX at fixed topology) and to the centres (the objective's explicit dependence)."""
    return ObjectiveAtCoordsFn.apply(X, centres, radii, grid, sweeps, bc, U, lo, hi, kind, tol)


def copfi(centres, radii, grid, sweeps, **kw):
    return objective(centres, radii, grid, sweeps, kind=api.PF_OBJ_COPFI, **kw)


def gap_flow(centres, radii, grid, sweeps, **kw):
    return objective(centres, radii, grid, sweeps, kind=api.PF_OBJ_GAP_FLOW, **kw)
