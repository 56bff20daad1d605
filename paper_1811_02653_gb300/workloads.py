"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the method's arithmetic: it only draws matrices.
Both the CUDA path (via tests and bench.py) and the FP64 oracle take their
inputs from here, so both see the same bits.

Every row (or, for right operands, every column) is drawn from its own
numpy ``SeedSequence([seed, stream, index])``, so any single row or column can
be regenerated alone.  Low-rank terms use factors rounded to a 2^-20 grid so
that their inner products are exact in FP64 in any summation order; every
matrix is formed in FP64 and rounded once to FP32.

Workloads (sizes of the paper's experiments are context; these are the
synthetic stand-ins):

* ``small``   -- A 512x4096, B 4096x512, N(0,1); b=256, N=4, e=1; block 2
                 dropped (0-based); hash seed 0.
* ``square``  -- A 16384x65536, B 65536x16384, N(0,1) plus a shared rank-64
                 spike of scale 10; b=1024, N=8, e=2; blocks {1,6} dropped.
* ``hessian`` -- A 4096x1048576 with 1% nonzeros N(0,1) stored dense,
                 D log-uniform in [1e-6, 1e6] (the interior-point normal
                 matrix A D A^T of Sec. 5.2); b=4096, N=6, e=1; block 3 dropped.
* ``batched`` -- 256 uneven products, m,l ~ U[256,4096], n log-uniform in
                 [8192,131072] rounded to 2048, b=n/32, N=4, e=1.
* ``autograd``-- X 4096x65536, G 65536x4096, N(0, 0.02^2); b=2048, N=4, e=1;
                 block 2 dropped.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

# stream ids
_S_LEFT, _S_RIGHT, _S_U, _S_V, _S_W, _S_MASKPOS, _S_D, _S_DC, _S_SHAPES = range(9)


def _rng(seed: int, stream: int, index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream, index])))


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def _map_rows(fn, indices, ncols, out_dtype=np.float32):
    indices = list(indices)
    out = np.empty((len(indices), ncols), dtype=out_dtype)

    def work(t):
        out[t] = fn(indices[t])

    if len(indices) <= 4:
        for t in range(len(indices)):
            work(t)
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, range(len(indices))))
    return out


def normal_row(seed: int, stream: int, index: int, ncols: int, std: float = 1.0) -> np.ndarray:
    """One FP64 row of i.i.d. N(0, std^2)."""
    return _rng(seed, stream, index).standard_normal(ncols) * std


def dyadic_factor(seed: int, stream: int, nrows: int, rank: int) -> np.ndarray:
    """nrows x rank factor of N(0,1) entries rounded to multiples of 2^-20
    (|entries| < 8), so rank-64 inner products are exact in FP64."""
    g = _rng(seed, stream, 0).standard_normal((nrows, rank))
    g = np.clip(g, -7.999, 7.999)
    return np.round(g * 2.0 ** 20) / 2.0 ** 20


def gaussian_rows(seed: int, stream: int, rows, ncols: int, std: float = 1.0) -> np.ndarray:
    """FP32 rows of N(0, std^2), row r from its own stream."""
    return _map_rows(lambda r: normal_row(seed, stream, r, ncols, std), rows, ncols)


# --------------------------------------------------------------------------
# workload descriptions
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    m: int
    n: int
    l: int
    b: int
    N: int
    e: int
    mask: int
    hash_seed: int = 0
    data_seed: int = 1000
    spike_rank: int = 0
    spike_scale: float = 0.0
    std: float = 1.0
    density: float = 1.0
    extra: dict = field(default_factory=dict)

    @property
    def P(self) -> int:
        return self.N + self.e

    @property
    def z(self) -> int:
        return self.P * self.b

    @property
    def k(self) -> int:
        return bin(self.mask).count("1")

    # ---- left operand (m x n): row r from stream (data_seed, LEFT, r) ----
    def left_rows(self, rows) -> np.ndarray:
        rows = list(rows)
        if self.spike_rank:
            U = dyadic_factor(self.data_seed, _S_U, self.m, self.spike_rank)
            V = dyadic_factor(self.data_seed, _S_V, self.n, self.spike_rank)
            c = self.spike_scale / math.sqrt(self.spike_rank)

            def fn(r):
                return normal_row(self.data_seed, _S_LEFT, r, self.n, self.std) + c * (V @ U[r])
            return _map_rows(fn, rows, self.n)
        if self.density < 1.0:
            return _map_rows(lambda r: self._sparse_row(r), rows, self.n)
        return gaussian_rows(self.data_seed, _S_LEFT, rows, self.n, self.std)

    def _sparse_entries(self, r: int):
        """Row r of a sparse left operand as (sorted column indices, FP64
        values): i.i.d. Bernoulli(density) support (count ~ Binomial,
        positions a uniform subset) with N(0, std^2) values."""
        g = _rng(self.data_seed, _S_LEFT, r)
        cnt = int(g.binomial(self.n, self.density))
        idx = np.sort(g.choice(self.n, size=cnt, replace=False))
        return idx, g.standard_normal(cnt) * self.std

    def _sparse_row(self, r: int) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.float64)
        idx, val = self._sparse_entries(r)
        out[idx] = val
        return out

    def left_sparse(self, rows):
        """Rows of a sparse left operand in CSR form (offsets int64, column
        indices int64, values FP32 rounded once), the same entries as
        ``left_rows``: lets a caller scatter the dense matrix on a device
        without forming it on the host."""
        rows = list(rows)
        parts = [None] * len(rows)

        def work(t):
            parts[t] = self._sparse_entries(rows[t])

        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, range(len(rows))))
        offs = np.zeros(len(rows) + 1, dtype=np.int64)
        offs[1:] = np.cumsum([len(ix) for ix, _ in parts])
        idx = np.concatenate([ix for ix, _ in parts]).astype(np.int64)
        val = np.concatenate([v for _, v in parts]).astype(np.float32)
        return offs, idx, val

    # ---- right operand (n x l): column c from stream (data_seed, RIGHT, c) ----
    def right_cols(self, cols) -> np.ndarray:
        """Columns of B as rows of the returned (len(cols) x n) FP32 array."""
        cols = list(cols)
        if self.spike_rank:
            V = dyadic_factor(self.data_seed, _S_V, self.n, self.spike_rank)
            W = dyadic_factor(self.data_seed, _S_W, self.l, self.spike_rank)
            c = self.spike_scale / math.sqrt(self.spike_rank)

            def fn(q):
                return normal_row(self.data_seed, _S_RIGHT, q, self.n, self.std) + c * (V @ W[q])
            return _map_rows(fn, cols, self.n)
        return gaussian_rows(self.data_seed, _S_RIGHT, cols, self.n, self.std)

    def left(self) -> np.ndarray:
        return self.left_rows(range(self.m))

    def right(self) -> np.ndarray:
        """B (n x l) row-major FP32."""
        return np.ascontiguousarray(self.right_cols(range(self.l)).T)

    def col_scale(self) -> np.ndarray | None:
        """sqrt(D) for the interior-point Hessian, D log-uniform (FP32)."""
        lo, hi = self.extra.get("d_range", (None, None))
        if lo is None:
            return None
        g = _rng(self.data_seed, _S_D, 0)
        d = 10.0 ** g.uniform(math.log10(lo), math.log10(hi), size=self.n)
        return np.sqrt(d).astype(np.float32)

    def upstream_grad(self) -> np.ndarray:
        """dC (m x l) N(0,1) for the backward pass."""
        return gaussian_rows(self.data_seed, _S_DC, range(self.m), self.l, 1.0)


def mask_dropping(P: int, dropped) -> int:
    mask = (1 << P) - 1
    for j in dropped:
        mask &= ~(1 << j)
    return mask


SMALL = Workload("small 512x4096x512 fp32, b=256 N=4 e=1, block 2 dropped",
                 m=512, n=4096, l=512, b=256, N=4, e=1,
                 mask=mask_dropping(5, [2]), hash_seed=0, data_seed=1001)

SQUARE = Workload("square 16384x65536x16384 fp32 + rank-64 spike, b=1024 N=8 e=2, blocks {1,6} dropped",
                  m=16384, n=65536, l=16384, b=1024, N=8, e=2,
                  mask=mask_dropping(10, [1, 6]), hash_seed=0, data_seed=1002,
                  spike_rank=64, spike_scale=10.0)

HESSIAN = Workload("hessian A D A^T, A 4096x1048576 1% dense, b=4096 N=6 e=1, block 3 dropped",
                   m=4096, n=1048576, l=4096, b=4096, N=6, e=1,
                   mask=mask_dropping(7, [3]), hash_seed=0, data_seed=1003,
                   density=0.01, extra={"d_range": (1e-6, 1e6), "symmetric": True})

AUTOGRAD = Workload("autograd X 4096x65536 G 65536x4096 N(0,0.02^2), b=2048 N=4 e=1, block 2 dropped",
                    m=4096, n=65536, l=4096, b=2048, N=4, e=1,
                    mask=mask_dropping(5, [2]), hash_seed=0, data_seed=1005, std=0.02)

AUTOGRAD_FD = Workload("autograd finite-difference check 64x512x64, b=32 N=4 e=1, block 2 dropped",
                       m=64, n=512, l=64, b=32, N=4, e=1,
                       mask=mask_dropping(5, [2]), hash_seed=0, data_seed=1105, std=0.02)


def batched_shapes(count: int = 256, seed: int = 1004):
    """(m, n, l) of the uneven batch: m, l ~ U[256, 4096] integers, n
    log-uniform in [8192, 131072] rounded to a multiple of 2048 (b = n/32)."""
    g = _rng(seed, _S_SHAPES, 0)
    m = g.integers(256, 4097, size=count)
    l = g.integers(256, 4097, size=count)
    n = np.exp(g.uniform(math.log(8192), math.log(131072), size=count))
    n = np.clip(np.round(n / 2048) * 2048, 8192, 131072).astype(np.int64)
    return [(int(a), int(c), int(d)) for a, c, d in zip(m, n, l)]


def batched_device_inputs(shapes, p: int, device, seed: int = 1004, dtype=None):
    """Inputs of product p of the uneven batch drawn on a CUDA device:
    A_p (m x n) and B_p (n x l) row-major, i.i.d. N(0,1) FP32 from torch's
    seeded Philox generator (one generator per product, seed
    ``seed * 100003 + p``).  At the batch's full size (182 GB of inputs) the
    host cannot draw them; the oracle reads sampled rows and columns of these
    same tensors back from the device."""
    import torch
    m, n, l = shapes[p]
    g = torch.Generator(device=device)
    g.manual_seed(seed * 100003 + p)
    A = torch.randn((m, n), generator=g, device=device, dtype=torch.float32)
    B = torch.randn((n, l), generator=g, device=device, dtype=torch.float32)
    if dtype is not None:
        A, B = A.to(dtype), B.to(dtype)
    return A, B


def scaled(w: Workload, **kw) -> Workload:
    """Copy of a workload with some fields replaced (smaller parity cases)."""
    d = dict(w.__dict__)
    d.update(kw)
    return Workload(**d)


def lp_instance(n: int, m: int, seed: int = 1006, density: float = 0.05):
    """The LP  min c^T x  s.t.  A x <= b  of Sec. 5.2 (A: n x m, n > m), drawn so
    that it is strictly feasible and bounded: A ~ N(0, 1/m) rounded to FP32,
    b = 1 + |N(0,1)| (x = 0 is strictly feasible), and c = -A^T y for a
    nonnegative y with about `density` n nonzeros (then c^T x >= -y^T b on the
    feasible set).  Returns (A float32 n x m, b float64 n, c float64 m)."""
    A = gaussian_rows(seed, _S_LEFT, range(n), m, std=1.0 / math.sqrt(m))
    g = _rng(seed, _S_D, 0)
    b = 1.0 + np.abs(g.standard_normal(n))
    y = np.abs(g.standard_normal(n)) * (g.random(n) < density)
    c = -(A.astype(np.float64).T @ y)
    return A, b, c


def straggler_block_masks(P: int, e: int, rows: int, cols: int, seed: int, it: int,
                          shared: bool = False) -> np.ndarray:
    """rows x cols int64 bit masks over P sketch blocks, each with e bits cleared
    at positions drawn uniformly without replacement, independently per block of
    C and per iteration `it`: the e workers that straggle on that block.  With
    `shared` every block gets the first block's mask (one straggler set for the
    whole product)."""
    g = _rng(seed, _S_MASKPOS, it)
    full = (1 << P) - 1
    out = np.empty((rows, cols), dtype=np.int64)
    for i in range(rows):
        for j in range(cols):
            msk = full
            for pos in g.choice(P, size=e, replace=False):
                msk &= ~(1 << int(pos))
            out[i, j] = np.int64(msk - (1 << 64) if msk >= 1 << 63 else msk)
    if shared:
        out[:] = out[0, 0]
    return out


def sec51_factors(m: int, n: int):
    """Factors of Sec. 5.1's matrix A(x, y) = x + y (x = 1..m, y = 1..n):
    A = U V^T with U = [x, 1] (m x 2) and V = [1, y] (n x 2); B = A^T = V U^T."""
    x = np.arange(1, m + 1, dtype=np.float64)
    y = np.arange(1, n + 1, dtype=np.float64)
    return np.stack([x, np.ones(m)], 1), np.stack([np.ones(n), y], 1)


def sec51_device(m: int, n: int, device):
    """A(x, y) = x + y (m x n, FP32, exact below 2^24) and B = A^T (n x m), both
    row-major on a CUDA device, and the exact product A A^T rounded once to
    FP32 from FP64: (A A^T)[x, x'] = n x x' + (x + x') sum(y) + sum(y^2)."""
    import torch
    x = torch.arange(1, m + 1, dtype=torch.float64, device=device)
    y = torch.arange(1, n + 1, dtype=torch.float64, device=device)
    A = x.float()[:, None] + y.float()[None, :]          # integers below 2^24: exact in FP32
    B = A.t().contiguous()
    sy, syy = float(n * (n + 1) / 2), float(n * (n + 1) * (2 * n + 1) / 6)
    AB = (n * x[:, None] * x[None, :] + (x[:, None] + x[None, :]) * sy + syy).float()
    return A, B, AB
