"""OverSketch CPU oracle -- test infrastructure only.

Plain FP64 implementation of what the OverSketch hot path computes, written
from the paper (Gupta, Wang, Courtade, Ramchandran, "OverSketch: Approximate
Matrix Multiplication for the Cloud", arXiv 1811.02653).  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
it; the product path never does.  It shares no code with the CUDA library:
the loops live in ``oversketch_oracle.c`` (compiled here with gcc), the
dense contractions are numpy matmuls, and the quantisers below are written
from the IEEE-754 / OCP FP8 format definitions.

Every function cites the passage it follows:

* ``hash_tables``    -- Alg. 4 steps 1-2 (random sign, uniform bucket), one
                        independent Count-sketch per block of Eq. 3.
* ``sketch_matrix``  -- the explicit unscaled S = (S_1, ..., S_{N+e}) of Eq. 3.
* ``sketch_left`` / ``sketch_right`` -- A~ = A S and B~ = S^T B (Alg. 5,
                        Alg. 4 step 3), the implicit (hash-loop) form.
* ``masked_product`` -- Alg. 3 computation + termination + reduction phases:
                        sum over the kept blocks j of A~_j B~_j, scaled 1/k.
* ``masked_product_blocks`` -- the same with Alg. 3's termination rule applied
                        to every block of C on its own (its own kept set).
* ``gradients``      -- the adjoint of the bilinear map C(X, G) of Eq. 3.
* ``expected_sq_error`` -- Lemma "countEV" (appendix B) exact variance, summed
                        over the entries of C as in Lemma "lemma2";
                        ``expected_sq_error_factored`` the same closed form
                        for factored operands (Sec. 5.1's rank-2 matrix).
* ``oracle.lp``      -- the log-barrier interior-point LP of Sec. 5.2 with the
                        exact Hessian.

Where the paper is silent this module takes these readings: the hash family
is splitmix64 (seeded per block, then per index), buckets are 0-based, the
product is scaled by 1/k for k kept blocks, and the BF16/FP8 quantisers round
to nearest even (FP8 with a power-of-two scale per 128 sketched columns).  No
value here ever comes from the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oversketch_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oversketch_oracle.so")
_lib = None
_lock = threading.Lock()

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def build_oracle(force: bool = False) -> str:
    """Compile the C loops of the oracle with gcc (FP64, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, i32, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
            vp, dbl = ctypes.c_void_p, ctypes.c_double
            lib.osk_oracle_mix64.restype = u64
            lib.osk_oracle_mix64.argtypes = [u64]
            lib.osk_oracle_hash.restype = None
            lib.osk_oracle_hash.argtypes = [i64, i32, i32, u64, vp, vp]
            lib.osk_oracle_sketch_left.restype = None
            lib.osk_oracle_sketch_left.argtypes = [vp, i64, i64, i64, vp, vp, i32, i32, vp, vp]
            lib.osk_oracle_sketch_right.restype = None
            lib.osk_oracle_sketch_right.argtypes = [vp, i64, i64, i64, vp, vp, i32, i32, vp]
            lib.osk_oracle_unsketch_cols.restype = None
            lib.osk_oracle_unsketch_cols.argtypes = [vp, i64, i64, vp, vp, i64, i32, i32, u64, dbl, vp, i64]
            lib.osk_oracle_unsketch_rows.restype = None
            lib.osk_oracle_unsketch_rows.argtypes = [vp, i64, i64, vp, vp, i64, i32, i32, u64, dbl, vp, i64]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------
# Hash (Alg. 4 steps 1-2, one independent Count-sketch per block of Eq. 3)
# --------------------------------------------------------------------------

def mix64(z: int) -> int:
    """splitmix64 output finaliser (C implementation)."""
    return int(_load().osk_oracle_mix64(z & MASK64))


def splitmix64_stream(seed: int, count: int) -> list[int]:
    """First ``count`` outputs of splitmix64 seeded with ``seed``."""
    return [mix64((seed + (t + 1) * GAMMA) & MASK64) for t in range(count)]


def hash_tables(n: int, b: int, N: int, e: int, seed: int):
    """Buckets h (P x n, uint32, 0-based) and signs sigma (P x n, int8).

    Alg. 4 step 1 (sign flip with probability 1/2) and step 2 (uniform bucket
    in [1, b], stored 0-based) for each of the P = N + e independent blocks
    of Eq. 3.
    """
    P = N + e
    if not (n >= 1 and b >= 1 and N >= 1 and e >= 0 and P <= 64):
        raise ValueError("bad plan parameters")
    h = np.empty((P, n), dtype=np.uint32)
    s = np.empty((P, n), dtype=np.int8)
    _load().osk_oracle_hash(n, b, P, seed & MASK64, _ptr(h), _ptr(s))
    return h, s


def tables_from_sketch_matrix(Sc: np.ndarray):
    """Recover (h, sigma) of one Count-sketch block from an explicit n x b
    matrix with exactly one +-1 per row (e.g. Eq. 2, transposed)."""
    Sc = np.asarray(Sc)
    n, b = Sc.shape
    h = np.empty((1, n), dtype=np.uint32)
    s = np.empty((1, n), dtype=np.int8)
    for i in range(n):
        nz = np.nonzero(Sc[i])[0]
        if len(nz) != 1 or abs(Sc[i, nz[0]]) != 1:
            raise ValueError("row %d is not a Count-sketch row" % i)
        h[0, i] = nz[0]
        s[0, i] = int(Sc[i, nz[0]])
    return h, s


# --------------------------------------------------------------------------
# Explicit S (Eq. 3, unscaled)
# --------------------------------------------------------------------------

def sketch_matrix(h: np.ndarray, sigma: np.ndarray, b: int) -> np.ndarray:
    """S = (S_1, ..., S_P) of Eq. 3 without the 1/sqrt(N): n x (P b), FP64,
    S[i, j b + h_j(i)] = sigma_j(i)."""
    P, n = h.shape
    S = np.zeros((n, P * b), dtype=np.float64)
    rows = np.arange(n)
    for j in range(P):
        S[rows, j * b + h[j].astype(np.int64)] = sigma[j].astype(np.float64)
    return S


def selected_blocks(mask: int, P: int) -> list[int]:
    """Blocks kept by the mask (bit j keeps block j), ascending."""
    if mask <= 0 or mask >> P:
        raise ValueError("mask must select at least one block among the P blocks")
    return [j for j in range(P) if (mask >> j) & 1]


def selected_columns(mask: int, P: int, b: int) -> np.ndarray:
    return np.concatenate([np.arange(j * b, (j + 1) * b) for j in selected_blocks(mask, P)])


# --------------------------------------------------------------------------
# Sketches (Alg. 5 / Alg. 4 step 3), implicit form in C
# --------------------------------------------------------------------------

def sketch_left(A, h, sigma, b: int, col_scale=None) -> np.ndarray:
    """A~ = A diag(col_scale) S, m x (P b), FP64 (implicit hash loop)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    P = h.shape[0]
    assert h.shape == (P, n) and sigma.shape == (P, n)
    h = np.ascontiguousarray(h, dtype=np.uint32)
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    out = np.empty((m, P * b), dtype=np.float64)
    cs = None
    if col_scale is not None:
        cs = np.ascontiguousarray(col_scale, dtype=np.float64)
        assert cs.shape == (n,)
    _load().osk_oracle_sketch_left(_ptr(A), m, n, n, _ptr(h), _ptr(sigma), b, P,
                                   _ptr(cs) if cs is not None else None, _ptr(out))
    return out


def sketch_right(B, h, sigma, b: int) -> np.ndarray:
    """B~ = S^T B, (P b) x l, FP64 (implicit hash loop)."""
    B = np.ascontiguousarray(B, dtype=np.float64)
    n, l = B.shape
    P = h.shape[0]
    assert h.shape == (P, n) and sigma.shape == (P, n)
    h = np.ascontiguousarray(h, dtype=np.uint32)
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    out = np.empty((P * b, l), dtype=np.float64)
    _load().osk_oracle_sketch_right(_ptr(B), n, l, l, _ptr(h), _ptr(sigma), b, P, _ptr(out))
    return out


# --------------------------------------------------------------------------
# Masked block-sum product (Alg. 3 with Alg. 2's computation/reduction)
# --------------------------------------------------------------------------

def masked_product(At, Bt, b: int, mask: int) -> np.ndarray:
    """C = (1/k) sum_{j kept, ascending} A~[:, jb:(j+1)b] @ B~[jb:(j+1)b, :].

    Alg. 3: the computation phase multiplies b x b blocks, the termination
    rule keeps any k of the P blocks of the inner dimension, and the
    reduction phase adds the kept partial products.  The 1/N of Eq. 3 is
    applied once as 1/k (k = N when exactly N blocks are kept).
    """
    At = np.asarray(At, dtype=np.float64)
    Bt = np.asarray(Bt, dtype=np.float64)
    P = At.shape[1] // b
    assert At.shape[1] == P * b and Bt.shape[0] == P * b
    sel = selected_blocks(mask, P)
    C = np.zeros((At.shape[0], Bt.shape[1]), dtype=np.float64)
    for j in sel:
        C += At[:, j * b:(j + 1) * b] @ Bt[j * b:(j + 1) * b, :]
    return C / len(sel)


def masked_product_blocks(At, Bt, b: int, masks, bm: int, bn: int) -> np.ndarray:
    """Alg. 3's termination rule applied to every block of C separately: block
    (i, j) of C (rows i*bm .., columns j*bn ..) is the reduction of its own kept
    sketch blocks, C(i, j) = (1/k_ij) sum_{t in masks[i][j]} A~(i, t) B~(t, j);
    a block with no kept sketch block is zero.  masks[i][j] is a bit mask of the
    kept blocks t (ascending)."""
    At = np.asarray(At, dtype=np.float64)
    Bt = np.asarray(Bt, dtype=np.float64)
    P = At.shape[1] // b
    assert At.shape[1] == P * b and Bt.shape[0] == P * b
    m, l = At.shape[0], Bt.shape[1]
    C = np.zeros((m, l), dtype=np.float64)
    for i in range((m + bm - 1) // bm):
        for j in range((l + bn - 1) // bn):
            if int(masks[i][j]) == 0:
                continue
            sel = selected_blocks(int(masks[i][j]), P)
            rs, cs = slice(i * bm, min(m, (i + 1) * bm)), slice(j * bn, min(l, (j + 1) * bn))
            acc = np.zeros((rs.stop - rs.start, cs.stop - cs.start), dtype=np.float64)
            for t in sel:
                acc += At[rs, t * b:(t + 1) * b] @ Bt[t * b:(t + 1) * b, cs]
            C[rs, cs] = acc / len(sel)
    return C


def oversketch(A, B, h, sigma, b: int, mask: int, col_scale=None) -> np.ndarray:
    """The whole OverSketch product (A S)(S^T B) restricted to kept blocks."""
    return masked_product(sketch_left(A, h, sigma, b, col_scale),
                          sketch_right(B, h, sigma, b), b, mask)


def oversketch_explicit(A, B, S, b: int, mask: int) -> np.ndarray:
    """Same product from the explicit S: (A S_sel)(S_sel^T B) / k."""
    P = S.shape[1] // b
    cols = selected_columns(mask, P, b)
    Ssel = S[:, cols]
    k = len(cols) // b
    return (np.asarray(A, np.float64) @ Ssel) @ (Ssel.T @ np.asarray(B, np.float64)) / k


# --------------------------------------------------------------------------
# Gradients of C(X, G) = (1/k) sum_j X S_j S_j^T G
# --------------------------------------------------------------------------

def unsketch_cols(T, h, sigma, b: int, mask: int, scale: float) -> np.ndarray:
    """dX = scale * T S_sel^T, i.e. dX[r,i] = scale * sum_j sigma_j(i) T[r, jb+h_j(i)]."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    m = T.shape[0]
    P, n = h.shape
    out = np.empty((m, n), dtype=np.float64)
    _load().osk_oracle_unsketch_cols(_ptr(T), m, T.shape[1],
                                     _ptr(np.ascontiguousarray(h, np.uint32)),
                                     _ptr(np.ascontiguousarray(sigma, np.int8)),
                                     n, b, P, mask, float(scale), _ptr(out), n)
    return out


def unsketch_rows(U, h, sigma, b: int, mask: int, scale: float) -> np.ndarray:
    """dG = scale * S_sel U, i.e. dG[i,c] = scale * sum_j sigma_j(i) U[jb+h_j(i), c]."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    l = U.shape[1]
    P, n = h.shape
    out = np.empty((n, l), dtype=np.float64)
    _load().osk_oracle_unsketch_rows(_ptr(U), l, l,
                                     _ptr(np.ascontiguousarray(h, np.uint32)),
                                     _ptr(np.ascontiguousarray(sigma, np.int8)),
                                     n, b, P, mask, float(scale), _ptr(out), l)
    return out


def gradients(X, G, dC, h, sigma, b: int, mask: int):
    """Gradients of L = <dC, C(X, G)> for C = (1/k) sum_{j kept} X S_j S_j^T G.

    dX = (1/k) (dC B~_sel^T) S_sel^T and dG = (1/k) S_sel (A~_sel^T dC),
    with A~ = X S and B~ = S^T G: the adjoint of the linear map S of Eq. 3.
    """
    P = h.shape[0]
    k = len(selected_blocks(mask, P))
    At = sketch_left(X, h, sigma, b)
    Bt = sketch_right(G, h, sigma, b)
    dC = np.asarray(dC, np.float64)
    T = dC @ Bt.T            # m x (P b); only kept blocks are read below
    U = At.T @ dC            # (P b) x l
    return (unsketch_cols(T, h, sigma, b, mask, 1.0 / k),
            unsketch_rows(U, h, sigma, b, mask, 1.0 / k))


# --------------------------------------------------------------------------
# Statistics (appendix B)
# --------------------------------------------------------------------------

def expected_sq_error(A, B, k: int, b: int) -> float:
    """E ||AB - C||_F^2 for k kept, independent, fully random Count-sketch
    blocks of width b, scale 1/k.

    Lemma "countEV" gives, for one block, Var[x^T S_c S_c^T y] =
    (1/b) (sum_{p != q} x_p^2 y_q^2 + sum_{p != q} x_p y_p x_q y_q).
    Averaging k independent blocks divides it by k (Lemma
    "sketch_properties"), and summing over the entries (Lemma "lemma2")
    with x = row of A, y = column of B gives
    (1/(k b)) (||A||^2 ||B||^2 + ||AB||^2 - 2 sum_i ||A[:,i]||^2 ||B[i,:]||^2).
    """
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    a2 = (A * A).sum(axis=0)          # ||A[:, i]||^2
    b2 = (B * B).sum(axis=1)          # ||B[i, :]||^2
    AB = A @ B
    total = a2.sum() * b2.sum() + (AB * AB).sum() - 2.0 * (a2 * b2).sum()
    return total / (k * b)


def expected_sq_error_factored(U, V, Y, W, k: int, b: int) -> float:
    """expected_sq_error for factored operands A = U V^T (m x n) and B = Y W^T
    (n x l), without forming them: every term of the closed form is a trace of
    small Gram matrices, and the column norms ||A[:,i]||^2 = v_i^T (U^T U) v_i,
    row norms ||B[i,:]||^2 = y_i^T (W^T W) y_i (Sec. 5.1's rank-2 matrix
    A(x, y) = x + y at full size)."""
    U, V, Y, W = (np.asarray(t, np.float64) for t in (U, V, Y, W))
    Gu, Gv, Gy, Gw = U.T @ U, V.T @ V, Y.T @ Y, W.T @ W
    A2 = np.trace(Gu @ Gv)
    B2 = np.trace(Gy @ Gw)
    M = V.T @ Y                                    # AB = U M W^T
    AB2 = np.trace(M.T @ Gu @ M @ Gw)
    a2 = np.einsum("ij,jk,ik->i", V, Gu, V)
    b2 = np.einsum("ij,jk,ik->i", Y, Gw, Y)
    return (A2 * B2 + AB2 - 2.0 * (a2 * b2).sum()) / (k * b)


def rel_frob(x, ref) -> float:
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


# --------------------------------------------------------------------------
# Quantisers (format definitions; decisions taken on FP32 inputs, the
# precision the sketch kernels hold their sums in)
# --------------------------------------------------------------------------

def round_bf16(x) -> np.ndarray:
    """Round-to-nearest-even to bfloat16 (8 significant bits, exponent range
    of binary32, subnormal quantum 2^-133), returned as float64 values.
    Inputs are first rounded to binary32."""
    x = np.asarray(x, np.float32).astype(np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    _, E = np.frexp(x[nz])                 # |x| = m 2^E, m in [0.5, 1)
    q = np.ldexp(1.0, np.maximum(E - 1, -126) - 7)
    out[nz] = np.rint(x[nz] / q) * q       # np.rint rounds half to even
    big = np.abs(out) > 3.3895313892515355e38
    out[big] = np.sign(out[big]) * np.inf
    return out


FP8_E4M3_MAX = 448.0


def round_fp8_e4m3(x) -> np.ndarray:
    """Saturating round-to-nearest-even to OCP FP8 E4M3 (bias 7, 3 mantissa
    bits, no infinities, largest finite 448, subnormal quantum 2^-9),
    returned as float64 values."""
    x = np.asarray(x, np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    _, E = np.frexp(x[nz])
    q = np.ldexp(1.0, np.maximum(E - 1, -6) - 3)
    out[nz] = np.rint(x[nz] / q) * q
    return np.clip(out, -FP8_E4M3_MAX, FP8_E4M3_MAX)


def fp8_scale_exponent(amax) -> np.ndarray:
    """Smallest integer e with amax <= 448 * 2^e (0 where amax == 0), the
    power-of-two (UE8M0) block scale.  Exact integer decision."""
    amax = np.asarray(amax, np.float32).astype(np.float64)
    e = np.zeros(amax.shape, dtype=np.int64)
    nz = amax > 0
    m, E = np.frexp(amax[nz])              # amax = m 2^E, 448 = 0.875 2^9
    e[nz] = np.where(m <= 0.875, E - 9, E - 8)
    return np.clip(e, -127, 127)


def quantize_fp8_rows(X, block: int = 128):
    """Per-row, per-``block``-column-slice UE8M0 scaling then E4M3 rounding.

    Returns (q, e) with q the E4M3 values (float64) and e the int exponents
    (rows x ceil(cols/block)); the dequantised matrix is q * 2^e.
    Inputs are first rounded to binary32.
    """
    X = np.asarray(X, np.float32).astype(np.float64)
    r, c = X.shape
    nb = (c + block - 1) // block
    q = np.empty_like(X)
    e = np.empty((r, nb), dtype=np.int64)
    for t in range(nb):
        sl = X[:, t * block:(t + 1) * block]
        et = fp8_scale_exponent(np.abs(sl).max(axis=1))
        e[:, t] = et
        q[:, t * block:(t + 1) * block] = round_fp8_e4m3(sl / np.ldexp(1.0, et)[:, None])
    return q, e


def dequantize_fp8_rows(q, e, block: int = 128) -> np.ndarray:
    return q * np.repeat(np.ldexp(1.0, e), block, axis=1)[:, :q.shape[1]]
