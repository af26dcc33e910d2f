"""torch.autograd bridge for the adjoint shape gradients of CoPFI / transverse-gap flow.

`objective(centres, ...)` builds the body-conforming mesh for the given body centres,
solves for psi and returns J (CoPFI or C_hi - C_lo); its backward pass returns dJ/dc
from the library's adjoint solve and shape-derivative kernels (pf_grad).  The mesh
topology is fixed for a given set of centres (which nodes are inside which body), so
gradients are those of the discrete objective at fixed topology."""
from __future__ import annotations

import numpy as np
import torch

from . import api


class ObjectiveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, centres, radii, grid, sweeps, bc, U, lo, hi, objective, tol):
        c = centres.detach().cpu().numpy().astype(np.float64).reshape(-1, 2)
        r = np.asarray(radii, dtype=np.float64).reshape(-1, 1)
        bodies = np.concatenate([c, r], axis=1)
        with api.mesh_build(grid, bodies, sweeps, bc) as mesh:
            api.psi_solve(mesh, U=U, tol=tol, precision=api.PF_MIXED)
            _, dJdc, J = api.grad(mesh, objective, lo, hi, U, tol, want_dX=False)
        ctx.save_for_backward(torch.from_numpy(dJdc).to(centres.dtype))
        return centres.new_tensor(float(J[0]))

    @staticmethod
    def backward(ctx, gJ):
        (dJdc,) = ctx.saved_tensors
        return (gJ.cpu() * dJdc).to(gJ.device) if gJ.is_cuda else gJ * dJdc, \
            None, None, None, None, None, None, None, None, None


def objective(centres: torch.Tensor, radii, grid, sweeps, bc=(0, 0, 0, 0), U=1.0, lo=3, hi=4,
              kind=api.PF_OBJ_COPFI, tol=1e-12) -> torch.Tensor:
    """J(centres) with autograd support; centres is an (n_bodies, 2) float64 tensor."""
    return ObjectiveFn.apply(centres, radii, grid, sweeps, bc, U, lo, hi, kind, tol)


def copfi(centres, radii, grid, sweeps, **kw):
    return objective(centres, radii, grid, sweeps, kind=api.PF_OBJ_COPFI, **kw)


def gap_flow(centres, radii, grid, sweeps, **kw):
    return objective(centres, radii, grid, sweeps, kind=api.PF_OBJ_GAP_FLOW, **kw)
