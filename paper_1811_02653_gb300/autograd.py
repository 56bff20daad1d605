"""OverSketch as a differentiable product (torch.autograd.Function).

Forward: C = (1/k) (X S_sel)(S_sel^T G) — the left and right sketch kernels
(kept blocks only) and the masked tensor-core GEMM.

Backward: C is bilinear in (X, G) and S enters linearly (Eq. 3), so

    dX = (1/k) (dC . B~_sel^T) . S_sel^T     dG = (1/k) S_sel . (A~_sel^T . dC)

computed by oversketch_matmul_backward: per side a tensor-core GEMM (the 1/k
in its epilogue) followed by an unsketch kernel (a signed gather through the
hash tables; every output written once, no atomics).  The sketched
operands A~ = X S and B~ = S^T G are either kept from the forward pass or, with
``recompute=True``, recomputed from X and G (two sketch launches instead of
holding m*z + l*z BF16 values).

Every step runs in the library's kernels; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import ops


class OverSketchMatmul(torch.autograd.Function):
    """C = (1/k) (X S_sel)(S_sel^T G) with a hand-written backward.

    Arguments: X (m x n), G (n x l) row-major FP32 or BF16 CUDA tensors; ``plan``
    an :class:`ops.Plan` of dimension n; ``mask`` the kept blocks; ``recompute``
    recomputes the sketches in backward instead of saving them.  The GEMMs run
    in BF16 with FP32 accumulation; gradients come back in the inputs' dtypes.
    """

    @staticmethod
    def forward(ctx, X, G, plan, mask: int, recompute: bool = False):
        At, _ = ops.sketch_left(plan, X, "bf16", block_mask=mask)
        BtT, _ = ops.sketch_right(plan, G, "bf16", block_mask=mask)
        C = ops.gemm_masked(plan, At, BtT, mask)
        ctx.plan, ctx.mask, ctx.recompute = plan, mask, recompute
        ctx.x_dtype, ctx.g_dtype = X.dtype, G.dtype
        if recompute:
            ctx.save_for_backward(X, G)
        else:
            ctx.save_for_backward(At, BtT)
        return C

    @staticmethod
    def backward(ctx, dC):
        plan, mask = ctx.plan, ctx.mask
        if ctx.recompute:
            X, G = ctx.saved_tensors
            At, _ = ops.sketch_left(plan, X, "bf16", block_mask=mask)
            BtT, _ = ops.sketch_right(plan, G, "bf16", block_mask=mask)
        else:
            At, BtT = ctx.saved_tensors
        if dC.stride(-1) != 1:
            dC = dC.contiguous()
        dX, dG = ops.matmul_backward(plan, At, BtT, dC.float(), mask, ctx.x_dtype, ctx.g_dtype,
                                     need_dx=ctx.needs_input_grad[0], need_dg=ctx.needs_input_grad[1])
        return dX, dG, None, None, None


def oversketch_matmul(X, G, plan, mask: int, recompute: bool = False):
    """Functional form of :class:`OverSketchMatmul`."""
    return OverSketchMatmul.apply(X, G, plan, mask, recompute)
