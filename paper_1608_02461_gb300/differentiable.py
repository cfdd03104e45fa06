"""The FMM potential as a differentiable torch operation.

phi = G~ q on the volume points of a tree (free-space sum with self terms, no
boundary correction), G~ the truncated FMM operator of Sec. 5.1.2 for the
tree's wavenumber k.  The backward pass is hand-written through the C ABI:

  dL/dq = G~^H (dL/dphi)                      (fmm_apply, HFMM_ADJ)
  dL/dk = Re sum conj(dL/dphi) * dG~/dk q     (fmm_apply, HFMM_DK)

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
            dphi, _ = tree.apply(q.contiguous(), None, src=hfmm.SET_VOL, tgt=hfmm.SET_VOL, mode=hfmm.DK)
            grad_k = (g.conj() * dphi).real.sum().to(torch.float64)
        return grad_q, grad_k, None


def fmm_potential(q, k, tree):
    """phi = G~ q, differentiable in q (complex128) and k (float64 scalar tensor)."""
    return HelmholtzFMM.apply(q, k, tree)
