"""Differentiable AMG-DD solves of the 3D variable-coefficient diffusion
problem -div(kappa grad x) = b (7-point finite differences, harmonic-mean face
coefficients, Dirichlet boundary).

`diffusion_solve(kappa, b, ...)` returns x; its backward pass solves the
adjoint system A lam = dL/dx with the same AMG-DD handle (A is symmetric) and
returns dL/db = lam and dL/dkappa from the library's gradient kernel
(amgdd_kappa_grad_3d). The matrix A(kappa) is assembled on the host and set up
once per forward call; every solve and the gradient run on the GPU.
"""
from __future__ import annotations

import numpy as np
import torch

import amgdd_inputs as I

from . import capi
from .solver import Solver


class DiffusionSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, b, box, padding, n_fac, tol, max_iter):
        nz, ny, nx = kappa.shape
        rp, ci, v = I.diffusion3d(kappa.detach().cpu().numpy())
        part, nsub = I.box_partition((nx, ny, nz), box)
        s = Solver(rp, ci, v, part, nsub, padding, n_fac=n_fac)
        x = torch.zeros(nx * ny * nz, dtype=torch.float64, device=kappa.device)
        s.solve(b.detach().contiguous(), x, tol=tol, max_iter=max_iter)
        ctx.solver = s
        ctx.tol, ctx.max_iter = tol, max_iter
        ctx.save_for_backward(kappa, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        kappa, x = ctx.saved_tensors
        s = ctx.solver
        lam = torch.zeros_like(x)
        s.solve(gx.detach().contiguous(), lam, tol=ctx.tol, max_iter=ctx.max_iter)
        nz, ny, nx = kappa.shape
        gk = torch.empty_like(x)
        capi.amgdd_kappa_grad_3d((nx, ny, nz), kappa.detach().contiguous(), x, lam, gk)
        s.close()
        ctx.solver = None
        return gk.view(nz, ny, nx), lam, None, None, None, None, None


def diffusion_solve(kappa, b, box=(16, 16, 16), padding=2, n_fac=2, tol=1e-10, max_iter=200):
    """x = A(kappa)^{-1} b by AMG-DD, differentiable in kappa (nz, ny, nx) and b."""
    return DiffusionSolve.apply(kappa, b, tuple(box), padding, n_fac, tol, max_iter)
