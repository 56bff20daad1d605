"""Shared helpers of the parity tests: tolerances derived from the arithmetic.

All expected values come from the FP64 oracle; nothing here computes the
method itself.
"""
import numpy as np

import oracle

U32 = 2.0 ** -24          # unit roundoff of binary32


def gpu_lib():
    """Build (incrementally) and load the CUDA library."""
    from paper_1811_02653_gb300 import build, ops
    build.build()
    return ops


def max_bucket(h, b):
    return int(max(np.bincount(row.astype(np.int64), minlength=b).max() for row in h))


def fp32_sum_bound(abs_sum, cnt):
    """Bound on |fp32 sequential sum - exact sum| for cnt terms whose absolute
    values sum to abs_sum: every FMA of the chain rounds once, and every
    partial sum is bounded by abs_sum (Higham, Thm 3.1 with gamma_cnt)."""
    g = cnt * U32 / (1 - cnt * U32)
    return g * abs_sum + 1e-30


def sketch_bounds_left(A, h, s, b, col_scale=None):
    """(reference FP64 sketch, elementwise FP32 error bound) for the left sketch."""
    ref = oracle.sketch_left(A, h, s, b, col_scale)
    absA = np.abs(np.asarray(A, np.float64))
    if col_scale is not None:
        absA = absA * np.abs(np.asarray(col_scale, np.float64))
    abs_sum = oracle.sketch_left(absA, h, np.ones_like(s), b)
    cnt = max_bucket(h, b) + (1 if col_scale is not None else 0)
    return ref, fp32_sum_bound(abs_sum, cnt)


def sketch_bounds_right(B, h, s, b):
    ref = oracle.sketch_right(B, h, s, b)
    abs_sum = oracle.sketch_right(np.abs(np.asarray(B, np.float64)), h, np.ones_like(s), b)
    return ref, fp32_sum_bound(abs_sum, max_bucket(h, b))


def assert_fp32_within(gpu, ref, bound):
    gpu = np.asarray(gpu, np.float64)
    bad = np.abs(gpu - ref) > bound
    assert not bad.any(), f"{bad.sum()} elements outside the FP32 bound; worst {np.abs(gpu - ref).max()}"


def assert_bf16_within(gpu_bf16_as_f64, ref, bound):
    """The kernel's BF16 value is RNE(fp32 sum); the fp32 sum lies in
    [ref - bound, ref + bound] and RNE is monotone, so the BF16 value lies in
    [RNE(ref - bound), RNE(ref + bound)]."""
    lo = oracle.round_bf16(ref - bound)
    hi = oracle.round_bf16(ref + bound)
    g = np.asarray(gpu_bf16_as_f64, np.float64)
    bad = (g < lo) | (g > hi)
    assert not bad.any(), f"{bad.sum()} BF16 elements outside [RNE(ref-bound), RNE(ref+bound)]"


def assert_fp8_within(q_gpu, scales_gpu, ref, bound, block=128):
    """Per (row, 128-slice): the scale exponent is the one the FP32 amax
    (within amax_ref +- max bound) gives, and every code lies in
    [RNE8((ref - bound)/2^e), RNE8((ref + bound)/2^e)] at the kernel's e."""
    q_gpu = np.asarray(q_gpu, np.float64)
    rows, cols = ref.shape
    e_gpu = np.log2(np.asarray(scales_gpu, np.float64))
    assert np.array_equal(e_gpu, np.round(e_gpu)), "scales must be powers of two"
    nb = (cols + block - 1) // block
    for t in range(nb):
        sl = slice(t * block, min(cols, (t + 1) * block))
        r = ref[:, sl]
        bd = bound[:, sl]
        amax = np.abs(r).max(axis=1)
        bmax = bd.max(axis=1)
        # the exponent is monotone in the FP32 amax except at amax = 0, which takes
        # exponent 0 (an all-zero slice): allow it where the window reaches 0
        may_be_zero = amax - bmax <= 0
        e_lo = np.where(may_be_zero, -127, oracle.fp8_scale_exponent(np.maximum(amax - bmax, 0.0)))
        e_hi = oracle.fp8_scale_exponent(amax + bmax)
        et = e_gpu[:, t]
        ok = ((et >= e_lo) & (et <= e_hi)) | (may_be_zero & (et == 0))
        assert ok.all(), "FP8 scale exponent outside its FP32 window"
        sc = np.ldexp(1.0, et.astype(np.int64))[:, None]
        lo = oracle.round_fp8_e4m3((r - bd) / sc)
        hi = oracle.round_fp8_e4m3((r + bd) / sc)
        g = q_gpu[:, sl]
        bad = (g < lo) | (g > hi)
        assert not bad.any(), f"{bad.sum()} FP8 codes outside their window in slice {t}"
