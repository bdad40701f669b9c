"""Differentiable BLR least squares: x = argmin ||A~ x - B||_F as a
torch.autograd.Function (QR used for least squares, Section 1).

Forward: tiled Householder BLR-QR of A~ (FP64), x = R^{-1} (Q^T B)(1:n) and
refinement steps x += R^{-1} Q_1^T (B - A~ x), all through the C ABI.
Backward: blr_lstsq_backward, reusing the stored R: z = R^{-1} R^{-T} xbar,
dL/dB = A~ z, dL/dA~ = r z^T - (A~ z) x^T with r = B - A~ x, projected on
the tile storage (dense tiles: the block; low-rank tiles U V^T: dL/dU =
(dL/dA~)_ij V and dL/dV = (dL/dA~)_ij^T U).  This module only marshals
arguments: every product runs in the library's kernels.

A~ is given by its storage: ``tiles`` (a float64 CUDA tensor of p*q*b*b
elements in the library's tile layout) and the host ``ranks`` (-1 dense).
"""
from __future__ import annotations

import numpy as np
import torch

from . import blr


class _Handles:
    """Keeps the factor and the factored matrix alive until backward."""

    def __init__(self, fac: blr.Factor, a_orig: blr.Matrix):
        self.fac, self.a_orig = fac, a_orig

    def release(self):
        if self.fac is not None:
            self.fac.destroy()
            self.a_orig.destroy()
            self.fac = self.a_orig = None


class BLRLstsq(torch.autograd.Function):
    """x = BLRLstsq.apply(tiles, B, ranks, m, n, b, opts, refine_steps)."""

    @staticmethod
    def forward(ctx, tiles, bmat, ranks, m, n, b, opts, refine_steps=1):
        bf = blr.to_fortran(bmat.detach())
        a = blr.blr_matrix_import_device(m, n, b, np.asarray(ranks), tiles.detach().contiguous())
        keep = blr.blr_matrix_clone(a)
        fac = blr.blr_qr(a, opts)
        x = blr.blr_lstsq(fac, bf, a_orig=keep if refine_steps > 0 else None, refine_steps=refine_steps)
        ctx.handles = _Handles(fac, keep)
        ctx.save_for_backward(bf, x)
        return x.clone()

    @staticmethod
    def backward(ctx, xbar):
        bf, x = ctx.saved_tensors
        h = ctx.handles
        try:
            bbar, gtiles = blr.blr_lstsq_backward(h.fac, h.a_orig, bf, x, blr.to_fortran(xbar.detach()))
        finally:
            h.release()
        return gtiles, bbar, None, None, None, None, None, None


def blr_lstsq_autograd(tiles, bmat, ranks, m, n, b, opts, refine_steps=1):
    """Functional form of BLRLstsq."""
    return BLRLstsq.apply(tiles, bmat, ranks, m, n, b, opts, refine_steps)
