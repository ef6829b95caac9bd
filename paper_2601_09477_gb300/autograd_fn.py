"""torch.autograd wrapper of the differentiable (mean-over-d) estimator.

The median of Algorithm 1's Decompress has no useful gradient, so the
differentiable form averages the d repetitions: at pairs (I[q], J[q])
    est[q] = (1/d) sum_r s1_r(I_q) s2_r(J_q) R_r[h1_r(I_q) XOR h2_r(J_q)],
R the Compress sketch of A B.  Forward runs cmm_sketch + cmm_mean_pairs;
backward runs the hand-written adjoint kernel (cmm_backward), which sketches
the output gradient by bucket h1 XOR h2, transforms it and scatters back to
dA and dB.  Every step runs in libcmm.
"""
from __future__ import annotations

import torch

from . import cmm


class CompressedMeanAtPairs(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, I, J, hashes: cmm.Hashes, prec: str = "f32", transA: bool = False):
        R = cmm.sketch(A, B, hashes, prec=prec, transA=transA)
        out = cmm.mean_pairs(R, hashes, I, J)
        ctx.save_for_backward(A, B, I, J)
        ctx.hashes = hashes
        ctx.prec = prec
        ctx.transA = transA
        return out.to(A.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        A, B, I, J = ctx.saved_tensors
        if not (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]):
            return None, None, None, None, None, None, None
        dA, dB = cmm.backward(A, B, ctx.hashes, I, J, grad_out.to(torch.float64),
                              prec=ctx.prec, transA=ctx.transA)
        return (dA if ctx.needs_input_grad[0] else None,
                dB if ctx.needs_input_grad[1] else None, None, None, None, None, None)


def compressed_mean_at_pairs(A, B, I, J, hashes: cmm.Hashes, prec: str = "f32",
                             transA: bool = False):
    """Differentiable estimate of (A B)[I[q], J[q]] (mean over the d repetitions)."""
    return CompressedMeanAtPairs.apply(A, B, I, J, hashes, prec, transA)
