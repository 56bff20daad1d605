"""Interior-point LP whose Newton steps use the OverSketch Hessian (Sec. 5.2).

The LP  minimize c^T x  subject to  A x <= b  (A: n x m, n > m)  is solved by the
logarithmic barrier method: Newton's method on
    f(x) = tau c^T x - sum_i log(b_i - a_i x),
tau doubled every `every` iterations (10 in the paper, 100 iterations in all).
With slacks s = b - A x the gradient is tau c + A^T (1/s) and the Hessian is
A^T diag(1/s^2) A = (D^{1/2} A)^T (D^{1/2} A), D^{1/2} = diag(1/s).

The Hessian is the O(n m^2) step and runs on the OverSketch path:
  1. the right sketch of A (n x m, row-major, gathered in place) with row
     scale 1/s, BF16 output -- (S^T D^{1/2} A)^T, m x z, without forming
     D^{1/2} A;
  2. the masked block-sum GEMM with the termination rule of Alg. 3 applied to
     every bs x bs block of the Hessian: block (i, j) sums only the sketch blocks
     its bit mask keeps (the paper ignores e straggling workers per block of C),
     scaled by 1/k_ij.
The O(n m) vector work (slacks, gradient, line search) and the m x m Newton
solve are PyTorch (cuBLAS / cuSOLVER) around that.  A sketched Hessian whose
blocks keep different sketch blocks is neither symmetric nor, in general,
positive semidefinite (it is no longer a Gram matrix).  The Newton system uses
its symmetric part, Jacobi-equilibrated and factorised by Cholesky in FP32
with the smallest shift of 0, 1e-8, 1e-7, ..., 1e8 times the identity for which
the factorisation succeeds (a non-finite system, or one that no such shift
repairs, raises NewtonSystemError).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ops


MAX_SHIFT = 1e8
SHIFTS = (0.0,) + tuple(10.0 ** p for p in range(-8, 9))      # 0, 1e-8, ..., 1e8


class NewtonSystemError(ValueError):
    """The Newton system cannot be solved: a non-finite Hessian or gradient, or no
    shift up to MAX_SHIFT makes the equilibrated system positive definite."""


@dataclass
class LPHistory:
    objective: list = field(default_factory=list)      # c^T x after each iteration
    step: list = field(default_factory=list)            # accepted step size eta
    shifts: int = 0                                      # Newton systems that needed a shift
    hessian_ms: list = field(default_factory=list)      # sketch + masked GEMM, CUDA events
    iter_ms: list = field(default_factory=list)         # whole iteration, CUDA events


class SketchedBarrierLP:
    """Barrier-method LP solver with the sketched Hessian on the GPU.

    A (n x m), b (n), c (m): host or device tensors / arrays; A is held in FP32
    for the sketch and in FP64 for the vector work.  The sketch
    S has P = N + e blocks of width `blk` over the n constraints (seed `seed`);
    the Hessian's blocks are blk x blk, so `blk` must be a multiple of 256."""

    def __init__(self, A, b, c, *, blk: int, N: int, e: int, seed: int = 0, exact: bool = False,
                 device="cuda"):
        A = torch.as_tensor(np.asarray(A, dtype=np.float32)) if not torch.is_tensor(A) else A
        self.n, self.m = A.shape
        if blk % 256:
            raise ValueError("the Hessian block size must be a multiple of 256")
        self.device = torch.device(device)
        self.A = A.contiguous().to(self.device, torch.float32)
        self.A64 = self.A.double()
        self.At = None                                   # A^T in FP32, for the unsketched arm only
        self.b = torch.as_tensor(np.asarray(b, dtype=np.float64)).to(self.device)
        self.c = torch.as_tensor(np.asarray(c, dtype=np.float64)).to(self.device)
        self.blk, self.N, self.e, self.P = blk, N, e, N + e
        self.exact = exact
        self.nb = (self.m + blk - 1) // blk
        self.plan = ops.plan(self.n, blk, N, e, seed)
        self.H = torch.empty((self.m, self.m), dtype=torch.float32, device=self.device)
        self.Ask = None
        self.ws = torch.empty(ops.sketch_workspace(self.plan, self.m), dtype=torch.uint8, device=self.device)
        self.Ask = ops.sketch_right(self.plan, self.A, "bf16", workspace=self.ws)[0]

    # -- the sketched Hessian -------------------------------------------------
    def hessian(self, s: torch.Tensor, block_masks) -> torch.Tensor:
        """A^T diag(1/s^2) A through the sketch: (S^T D^{1/2} A)^T, then the
        masked-block products, block (i, j) keeping the sketch blocks of
        block_masks[i, j].  With `exact`, the unsketched BF16 product instead.
        When every block keeps the same set the product is a Gram matrix and the
        library computes its lower triangle only (one mask, the same operand twice)."""
        d = (1.0 / s).float()
        if self.exact:
            if self.At is None:
                self.At = self.A.t().contiguous()
            Xd = (self.At * d).to(torch.bfloat16)
            return ops.gemm_bf16(Xd, Xd, C=self.H)
        ops.sketch_right(self.plan, self.A, "bf16", out=self.Ask, workspace=self.ws, row_scale=d)
        bm = np.asarray(block_masks, dtype=np.int64)
        if bm.size and (bm == bm.flat[0]).all():
            return ops.gemm_masked(self.plan, self.Ask, self.Ask, int(bm.flat[0]), C=self.H)
        masks = torch.as_tensor(bm).to(self.device, non_blocking=True)
        return ops.gemm_masked_blocks(self.plan, self.Ask, self.Ask, masks, self.blk, self.blk, C=self.H)

    # -- the Newton system ----------------------------------------------------
    def newton_direction(self, H: torch.Tensor, g: torch.Tensor, hist: LPHistory) -> torch.Tensor:
        """-(H_sym + shift D)^{-1} g, D = diag(H_sym), with the smallest shift of
        0, 1e-8, 1e-7, ..., 1e8 for which the equilibrated system factorises
        (rows with a non-positive diagonal entry are left unscaled).  Raises
        NewtonSystemError for a non-finite H or g, or when no shift up to 1e8
        factorises, instead of searching forever."""
        if not (bool(torch.isfinite(H).all()) and bool(torch.isfinite(g).all())):
            raise NewtonSystemError("non-finite Hessian or gradient")
        Hs = 0.5 * (H + H.t())
        dH = Hs.diagonal()
        pos = dH > 0
        dg = torch.where(pos, torch.where(pos, dH, torch.ones_like(dH)).rsqrt(), torch.ones_like(dH))
        Heq = Hs * dg[:, None] * dg[None, :]
        rhs = (g.float() * dg)[:, None]
        for shift in SHIFTS:
            L, info = torch.linalg.cholesky_ex(Heq if shift == 0.0 else Heq + shift * self._eye())
            if int(info) == 0:
                hist.shifts += shift > 0.0
                y = torch.cholesky_solve(rhs, L)[:, 0]
                return -(y.double() * dg.double())
        raise NewtonSystemError("no shift up to 1e8 makes the Newton system positive definite")

    def _eye(self):
        if getattr(self, "_I", None) is None:
            self._I = torch.eye(self.m, dtype=torch.float32, device=self.device)
        return self._I

    def barrier(self, s: torch.Tensor, x: torch.Tensor, tau: float) -> float:
        if bool((s <= 0).any()):
            return math.inf
        return tau * float(self.c @ x) - float(torch.log(s).sum())

    # -- the method -----------------------------------------------------------
    def solve(self, x0=None, iters: int = 100, tau0: float = 1.0, every: int = 10, block_masks=None,
              timing: bool = False):
        """Newton iterations of the barrier method.  `block_masks(t)` gives the
        nb x nb int64 masks of iteration t (default: every block keeps all P).
        Returns (x, LPHistory)."""
        full = np.full((self.nb, self.nb), (1 << self.P) - 1 if self.P < 63 else -1, dtype=np.int64)
        x = torch.zeros(self.m, dtype=torch.float64, device=self.device) if x0 is None else \
            torch.as_tensor(np.asarray(x0, np.float64)).to(self.device)
        hist = LPHistory()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if timing else None
        for t in range(iters):
            tau = tau0 * 2.0 ** (t // every)
            if timing:
                ev[0].record()
            s = self.b - self.A64 @ x
            g = tau * self.c + self.A64.t() @ (1.0 / s)
            msk = block_masks(t) if block_masks is not None else full
            if timing:
                ev[1].record()
            H = self.hessian(s, msk)
            if timing:
                ev[2].record()
            dx = self.newton_direction(H, g, hist)
            Adx = self.A64 @ dx
            f0, slope = self.barrier(s, x, tau), float(g @ dx)
            eta = 1.0
            while eta > 1e-12:
                fn = self.barrier(s - eta * Adx, x + eta * dx, tau)
                if math.isfinite(fn) and fn <= f0 + 0.25 * eta * slope:
                    break
                eta *= 0.5
            if eta > 1e-12:
                x = x + eta * dx
            else:
                eta = 0.0
            if timing:
                ev[3].record()
                ev[3].synchronize()
                hist.hessian_ms.append(ev[1].elapsed_time(ev[2]))
                hist.iter_ms.append(ev[0].elapsed_time(ev[3]))
            hist.objective.append(float(self.c @ x))
            hist.step.append(eta)
        return x, hist
