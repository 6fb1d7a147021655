"""Differentiable projection: torch.autograd.Function around the C ABI.

Forward runs the four projection steps on the GPU and checkpoints only beta
and the pressure p (not the multigrid history).  Backward runs the adjoint
(paris_project_adjoint: one more Poisson solve with the same operator, then
face-gradient products) and, when C needs a gradient, the adjoint of the face
coefficients (paris_face_coeffs_adjoint).  All arithmetic is in the CUDA
library; this module only wires tensors.
"""
from __future__ import annotations

import torch


class _Projection(torch.autograd.Function):
    @staticmethod
    def forward(fctx, C, us, vs, ws, pctx, rho1, rho2, dt, p0):
        u, v, w = us.detach().clone(), vs.detach().clone(), ws.detach().clone()
        p = p0.detach().clone() if p0 is not None else torch.zeros(
            pctx.grid.shape, dtype=torch.float64, device=us.device)
        bx, by, bz = pctx.face_coeffs(C.detach(), rho1, rho2)
        rhs, _ = pctx.divergence(u, v, w, dt, want_mean=False)
        fctx.stats = pctx.poisson_solve(bx, by, bz, rhs, p)
        pctx.project(bx, by, bz, p, dt, u, v, w)
        fctx.save_for_backward(bx, by, bz, p)
        fctx.pctx, fctx.rho1, fctx.rho2, fctx.dt = pctx, rho1, rho2, dt
        fctx.mark_non_differentiable(p)
        return u, v, w, p

    @staticmethod
    def backward(fctx, gu, gv, gw, gp):
        bx, by, bz, p = fctx.saved_tensors
        pctx = fctx.pctx
        grads = []
        for a, gx in enumerate((gu, gv, gw)):
            if gx is None:
                gx = torch.zeros(pctx.grid.face_shape(a), dtype=torch.float64, device=p.device)
            grads.append(gx.contiguous())
        (gus, gvs, gws), (gbx, gby, gbz), q, st = pctx.project_adjoint(bx, by, bz, p, fctx.dt, *grads)
        fctx.adjoint_stats = st
        gC = None
        if fctx.needs_input_grad[0]:
            gC = pctx.face_coeffs_adjoint(fctx.rho1, fctx.rho2, bx, by, bz, gbx, gby, gbz)
        return gC, gus, gvs, gws, None, None, None, None, None


def projection(C, us, vs, ws, pctx, rho1, rho2, dt, p0=None):
    """u, v, w, p = projection(C, u*, v*, w*, ...): differentiable in C and u*.

    C: cells, u*/v*/w*: face arrays (float64, on pctx's device).  p (mean-free
    pressure) is returned but not differentiable.  p0: initial guess."""
    return _Projection.apply(C, us, vs, ws, pctx, rho1, rho2, dt, p0)
