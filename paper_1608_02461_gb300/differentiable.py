"""The FMM potential and the preconditioned Helmholtz solve as differentiable
torch operations.

phi = G~ q on the volume points of a tree (free-space sum with self terms, no
boundary correction), G~ the truncated FMM operator of Sec. 5.1.2 for the
tree's wavenumber k.  The backward pass is hand-written through the C ABI:

  dL/dq = G~^H (dL/dphi)                      (fmm_apply, HFMM_ADJ)
  dL/dk = Re sum conj(dL/dphi) * dG~/dk q     (fmm_grad_k: HFMM_DK apply and
                                               the sum, on the device)

following PyTorch's convention for complex tensors (the gradient of a real
loss is the conjugate Wirtinger derivative times two, so a linear map's
gradient is its conjugate transpose applied to the output gradient).
"""
from __future__ import annotations

import torch

from . import hfmm


class HelmholtzFMM(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, k, tree):
        if abs(float(k) - tree.k) > 1e-12 * max(1.0, abs(tree.k)):
            raise ValueError("k must equal the wavenumber the tree was built for")
        phi, _ = tree.apply(q.contiguous(), None, src=hfmm.SET_VOL, tgt=hfmm.SET_VOL)
        ctx.tree = tree
        ctx.save_for_backward(q)
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        (q,) = ctx.saved_tensors
        tree = ctx.tree
        g = grad_phi.contiguous()
        grad_q = grad_k = None
        if ctx.needs_input_grad[0]:
            grad_q, _ = tree.apply(g, None, src=hfmm.SET_VOL, tgt=hfmm.SET_VOL, mode=hfmm.ADJ)
        if ctx.needs_input_grad[1]:
            grad_k = tree.grad_k(q.contiguous(), g)
        return grad_q, grad_k, None


def fmm_potential(q, k, tree):
    """phi = G~ q, differentiable in q (complex128) and k (float64 scalar tensor)."""
    return HelmholtzFMM.apply(q, k, tree)


class HelmholtzSolve(torch.autograd.Function):
    """x = A(k)^-1 b for the 7-point operator of the tree's grid, solved by
    the FMM-preconditioned GMRES (gmres_solve).  For real k, A is real and
    symmetric, so the adjoint system A^H lam = dL/dx is the forward system and
    is solved the same way (the preconditioner changes the convergence, not
    the solution):

      dL/db = lam,    dL/dk = Re <lam, 2k x>     (dA/dk = -2k I; hfmm_solve_grad_k)

    with <u, v> = sum conj(u) v, in PyTorch's convention for complex tensors."""

    @staticmethod
    def forward(ctx, b, k, tree, kw):
        if abs(float(k) - tree.k) > 1e-12 * max(1.0, abs(tree.k)):
            raise ValueError("k must equal the wavenumber the tree was built for")
        x, info = tree.gmres(b.contiguous(), raise_on_nonconvergence=True, **kw)
        ctx.tree = tree
        ctx.kw = kw
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        lam, _ = ctx.tree.gmres(grad_x.contiguous(), raise_on_nonconvergence=True, **ctx.kw)
        grad_b = lam if ctx.needs_input_grad[0] else None
        grad_k = None
        if ctx.needs_input_grad[1]:
            grad_k = ctx.tree.solve_grad_k(lam, x)
        return grad_b, grad_k, None, None


def helmholtz_solve(b, k, tree, **gmres_kw):
    """x = A(k)^-1 b (FMM-preconditioned GMRES), differentiable in b
    (complex128) and k (float64 scalar tensor); gmres_kw go to Tree.gmres."""
    return HelmholtzSolve.apply(b, k, tree, gmres_kw)
