"""GPU parity of the plan (bit-exact) and of the sketch kernels (within the
FP32 rounding bound of each output), through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import (assert_bf16_within, assert_fp32_within, assert_fp8_within, gpu_lib,
                     sketch_bounds_left, sketch_bounds_right)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


def _dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


PLAN_CASES = [
    (4096, 256, 4, 1, 0),          # small workload plan
    (65536, 1024, 8, 2, 0),        # square workload plan
    (5000, 1, 3, 1, 7),            # b = 1: every index in one bucket
    (37, 64, 2, 1, 3),             # b >= n
    (9999, 128, 60, 4, 11),        # N + e = 64, n not a multiple of the chunk
    (1, 16, 1, 0, 5),              # n = 1, e = 0
    (300_000, 4096, 6, 1, 0),      # wide buckets, many chunks
]


@pytest.mark.parametrize("n,b,N,e,seed", PLAN_CASES)
def test_plan_tables_bit_exact(ops, n, b, N, e, seed):
    p = ops.plan(n, b, N, e, seed)
    h, s, perm, offs = p.tables()
    h_ref, s_ref = oracle.hash_tables(n, b, N, e, seed)
    assert np.array_equal(h, h_ref)
    assert np.array_equal(s, s_ref)
    # bucket-CSR: stable counting sort of every block by bucket
    for j in range(N + e):
        order = np.argsort(h_ref[j], kind="stable")
        exp_perm = order.astype(np.uint32) | np.where(s_ref[j][order] < 0, np.uint32(1 << 31), np.uint32(0))
        assert np.array_equal(perm[j], exp_perm)
        cnt = np.bincount(h_ref[j].astype(np.int64), minlength=b)
        assert np.array_equal(offs[j], np.concatenate([[0], np.cumsum(cnt)]).astype(np.uint32))
    p.destroy()


def test_plan_from_tables_eq2(ops):
    ScT = np.array([[0, 0, 0, 1, -1, 0, -1, 0, 0], [1, -1, 0, 0, 0, 1, 0, 0, 0],
                    [0, 0, 1, 0, 0, 0, 0, -1, -1]], dtype=np.float64)
    h, s = oracle.tables_from_sketch_matrix(ScT.T)
    p = ops.plan_from_tables(h, s, 3, 1, 0)
    hh, ss, _, _ = p.tables()
    assert np.array_equal(hh, h) and np.array_equal(ss, s)
    A = np.random.default_rng(0).standard_normal((5, 9)).astype(np.float32)
    At, _ = ops.sketch_left(p, _dev(A), "f32")
    ref, bound = sketch_bounds_left(A, h, s, 3)
    assert_fp32_within(At.cpu().numpy(), ref, bound)
    # identity in: S_c out (exact)
    I = np.eye(9, dtype=np.float32)
    At, _ = ops.sketch_left(p, _dev(I), "f32")
    assert np.array_equal(At.cpu().numpy().astype(np.float64), ScT.T)


def test_plan_rejects_bad_tables(ops):
    with pytest.raises(ops.OverSketchError):
        ops.plan_from_tables(np.array([[5, 0]], np.uint32), np.array([[1, 1]], np.int8), 3, 1, 0)
    with pytest.raises(ops.OverSketchError):
        ops.plan(10, 4, 64, 1)


SKETCH_CASES = [
    # m, n, l, b, N, e
    (512, 4096, 512, 256, 4, 1),       # small workload
    (300, 2000, 130, 128, 3, 2),       # ragged tiles, free dims not multiples of 128
    (7, 513, 5, 32, 2, 1),             # tiny, odd sizes
    (129, 4096, 257, 1024, 2, 1),      # one bucket per CTA tile row
    (64, 3000, 300, 128, 3, 1),        # right sketch: 128-wide strips in place + packed remainder
    (32, 2048, 384, 256, 2, 1),        # right sketch: whole 128-wide strips only
    (130, 100_000, 70, 512, 3, 1),     # 4 windows of the sketched dimension, the last one ragged
    (64, 70_001, 200, 4096, 2, 1),     # 3 windows with few members per (window, bucket) list
    (64, 20_000, 1023, 512, 3, 1),     # right operand rows not 16-byte aligned: 124-wide strips in place
]


@pytest.mark.parametrize("m,n,l,b,N,e", SKETCH_CASES)
def test_sketch_fp32_parity(ops, m, n, l, b, N, e):
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    B = rng.standard_normal((n, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 0)
    h, s = oracle.hash_tables(n, b, N, e, 0)
    At, _ = ops.sketch_left(p, _dev(A), "f32")
    BtT, _ = ops.sketch_right(p, _dev(B), "f32")
    ref_l, bd_l = sketch_bounds_left(A, h, s, b)
    ref_r, bd_r = sketch_bounds_right(B, h, s, b)
    assert_fp32_within(At.cpu().numpy(), ref_l, bd_l)
    assert_fp32_within(BtT.cpu().numpy(), ref_r.T, bd_r.T)
    # bitwise reproducible (fixed order, no atomics)
    At2, _ = ops.sketch_left(p, _dev(A), "f32")
    assert torch.equal(At, At2)


@pytest.mark.parametrize("m,n,b,N,e,in_dtype,scaled,out", [
    (1000, 20_000, 256, 3, 1, None, False, "f32"),           # 8 strips, the last one ragged
    (1300, 9_000, 128, 4, 1, torch.bfloat16, False, "f32"),  # BF16 input: 256-row strips, 6 strips
    (777, 12_345, 512, 2, 2, None, True, "bf16"),            # column scale, BF16 output, ragged strip
    (2048, 4_096, 1024, 2, 1, None, False, "tf32x2"),        # 16 strips, hi/lo planes
])
def test_left_sketch_many_strips(ops, m, n, b, N, e, in_dtype, scaled, out):
    # many packed strips (128 rows of FP32, 256 of BF16), a ragged last strip, a
    # column scale and every output form: every kept element within the FP32
    # bound of the oracle
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    Ad = _dev(A, in_dtype)
    A64 = Ad.float().cpu().numpy()
    cs = rng.uniform(0.25, 4.0, n).astype(np.float32) if scaled else None
    p = ops.plan(n, b, N, e, 3)
    h, s = oracle.hash_tables(n, b, N, e, 3)
    mask = (1 << (N + e)) - 1 - 2            # block 1 dropped: only the other blocks are sketched
    At, _ = ops.sketch_left(p, Ad, out, col_scale=_dev(cs) if scaled else None, block_mask=mask)
    ref, bd = sketch_bounds_left(A64, h, s, b, cs)
    cols = oracle.selected_columns(mask, N + e, b)
    if out == "tf32x2":
        hi, lo = ops.tf32_planes(At)
        got = hi.cpu().numpy().astype(np.float64) + lo.cpu().numpy().astype(np.float64)
        assert_fp32_within(got[:, cols], ref[:, cols], bd[:, cols])
    elif out == "bf16":
        assert_bf16_within(At.float().cpu().numpy()[:, cols], ref[:, cols], bd[:, cols])
    else:
        assert_fp32_within(At.cpu().numpy()[:, cols], ref[:, cols], bd[:, cols])
    At2, _ = ops.sketch_left(p, Ad, out, col_scale=_dev(cs) if scaled else None, block_mask=mask)
    ct = torch.from_numpy(cols).cuda()
    assert torch.equal(At[:, ct], At2[:, ct])   # bitwise reproducible (dropped blocks are left unwritten)
    if out == "tf32x2":
        assert torch.equal(ops.tf32_planes(At)[1][:, ct], ops.tf32_planes(At2)[1][:, ct])


def test_sketch_col_scale(ops):
    m, n, b, N, e = 64, 3000, 256, 3, 1
    rng = np.random.default_rng(3)
    A = rng.standard_normal((m, n)).astype(np.float32)
    cs = np.sqrt(10.0 ** rng.uniform(-6, 6, n)).astype(np.float32)
    p = ops.plan(n, b, N, e, 1)
    h, s = oracle.hash_tables(n, b, N, e, 1)
    At, _ = ops.sketch_left(p, _dev(A), "f32", col_scale=_dev(cs))
    ref, bd = sketch_bounds_left(A, h, s, b, cs)
    assert_fp32_within(At.cpu().numpy(), ref, bd)


@pytest.mark.parametrize("l,in_dtype", [(384, None),                 # in-place strips
                                         (301, None),                 # in-place strips + packed remainder
                                         (70, torch.bfloat16)])       # packed BF16 operand
def test_sketch_right_row_scale(ops, l, in_dtype):
    # S^T diag(s) B: the right sketch with a scale per sketched index i equals the
    # left sketch of B^T with that column scale
    n, b, N, e = 3000, 256, 3, 1
    rng = np.random.default_rng(l)
    B = rng.standard_normal((n, l)).astype(np.float32)
    rs = np.sqrt(10.0 ** rng.uniform(-6, 6, n)).astype(np.float32)
    Bd = _dev(B, in_dtype)
    B64 = Bd.float().cpu().numpy()
    p = ops.plan(n, b, N, e, 2)
    h, s = oracle.hash_tables(n, b, N, e, 2)
    BtT, _ = ops.sketch_right(p, Bd, "f32", row_scale=_dev(rs))
    ref, bd = sketch_bounds_left(np.ascontiguousarray(B64.T), h, s, b, rs)
    assert_fp32_within(BtT.cpu().numpy(), ref, bd)
    Bb, _ = ops.sketch_right(p, Bd, "bf16", row_scale=_dev(rs))
    assert_bf16_within(Bb.float().cpu().numpy(), ref, bd)


@pytest.mark.parametrize("n,l,ldb,off,b,out,mask,N,e", [
    (3000, 1023, 1023, 0, 256, "f32", 0, 3, 1),        # rows 4 bytes apart mod 16: all four classes
    (5000, 500, 502, 0, 512, "f32", 0, 3, 1),          # two classes (row pitch 2 mod 4 elements)
    (4096, 376, 377, 1, 256, "bf16", 0b1011, 3, 1),    # three 124-wide strips + 4 packed columns, base 4 B past 16
    (2000, 128, 129, 3, 128, "f32", 0, 3, 1),          # one strip, base 12 bytes past 16
    (2000, 127, 127, 0, 128, "f32", 0, 3, 1),          # a strip would read past the row: packed
    (3000, 250, 251, 2, 256, "tf32x2", 0, 3, 1),       # two strips and a 2-column remainder, hi/lo planes
    (3000, 260, 261, 0, 256, "fp8", 0b1101, 3, 1),     # FP8 epilogue in clusters of four
    (3000, 1023, 1023, 0, 128, "f32", 0, 6, 2),        # 8 blocks gathered: packed instead
    (3000, 1023, 1023, 0, 128, "bf16", 0b00111111, 6, 2),   # 6 of 8 blocks: in place again
])
def test_sketch_right_misaligned_rows(ops, n, l, ldb, off, b, out, mask, N, e):
    # B rows that do not start on 16-byte boundaries are gathered in place (or
    # packed when more than 6 blocks are gathered): each lane reads the 16-byte
    # granule holding its first element and the sums are kept per misalignment
    # class, so every kept element stays within the FP32 bound of the oracle's
    # sketch and reruns are bitwise equal
    rng = np.random.default_rng(n + l + off)
    store = torch.from_numpy(rng.standard_normal((n + 1) * ldb).astype(np.float32)).cuda()
    Bd = torch.as_strided(store, (n, l), (ldb, 1), off)     # row pitch ldb, first element off floats in
    B64 = Bd.cpu().numpy().astype(np.float64)
    p = ops.plan(n, b, N, e, 4)
    h, s = oracle.hash_tables(n, b, N, e, 4)
    ref, bd = sketch_bounds_right(B64, h, s, b)
    ref, bd = ref.T, bd.T
    keep = mask or (1 << (N + e)) - 1
    cols = oracle.selected_columns(keep, N + e, b)
    Y, sc = ops.sketch_right(p, Bd, out, block_mask=mask)
    if out == "tf32x2":
        hi, lo = ops.tf32_planes(Y)
        got = hi.cpu().numpy().astype(np.float64) + lo.cpu().numpy().astype(np.float64)
        assert_fp32_within(got[:, cols], ref[:, cols], bd[:, cols])
    elif out == "bf16":
        assert_bf16_within(Y.float().cpu().numpy()[:, cols], ref[:, cols], bd[:, cols])
    elif out == "fp8":
        scale_rows = ops.fp8_scales_by_row(sc, l).cpu().numpy()
        slices = cols.reshape(-1, 128)[:, 0] // 128
        assert_fp8_within(Y.float().cpu().numpy()[:, cols], scale_rows[:, slices], ref[:, cols], bd[:, cols])
    else:
        assert_fp32_within(Y.cpu().numpy()[:, cols], ref[:, cols], bd[:, cols])
    Y2, _ = ops.sketch_right(p, Bd, out, block_mask=mask)
    ct = torch.from_numpy(cols).cuda()
    if out == "fp8":
        assert torch.equal(Y.view(torch.uint8)[:, ct], Y2.view(torch.uint8)[:, ct])
    else:
        assert torch.equal(Y[:, ct], Y2[:, ct])


@pytest.mark.parametrize("l,ldb,out,scaled", [
    (512, 512, "f32", False),      # two 256-wide BF16 strips in place
    (600, 600, "bf16", True),      # two strips in place + an 88-column packed remainder, row scale
    (300, 304, "fp8", False),      # one strip + 44 packed columns, padded rows
    (520, 521, "f32", False),      # rows not 16-byte aligned: packed
])
def test_sketch_right_bf16_in_place(ops, l, ldb, out, scaled):
    # a BF16 right operand with 16-byte aligned rows is gathered in place in
    # 256-wide strips (512-byte row pieces, as from a packed strip)
    n, b, N, e = 5000, 256, 3, 1
    rng = np.random.default_rng(l + ldb)
    store = torch.from_numpy(rng.standard_normal((n, ldb)).astype(np.float32)).to(torch.bfloat16).cuda()
    Bd = store[:, :l]
    B64 = Bd.float().cpu().numpy().astype(np.float64)
    rs = np.sqrt(10.0 ** rng.uniform(-3, 3, n)).astype(np.float32) if scaled else None
    p = ops.plan(n, b, N, e, 8)
    h, s = oracle.hash_tables(n, b, N, e, 8)
    Y, sc = ops.sketch_right(p, Bd, out, row_scale=_dev(rs) if scaled else None)
    ref, bd = sketch_bounds_left(np.ascontiguousarray(B64.T), h, s, b, rs)
    if out == "fp8":
        assert_fp8_within(Y.float().cpu().numpy(), ops.fp8_scales_by_row(sc, l).cpu().numpy(), ref, bd)
    elif out == "bf16":
        assert_bf16_within(Y.float().cpu().numpy(), ref, bd)
    else:
        assert_fp32_within(Y.cpu().numpy(), ref, bd)
    Y2, _ = ops.sketch_right(p, Bd, out, row_scale=_dev(rs) if scaled else None)
    assert torch.equal(Y.view(torch.uint8), Y2.view(torch.uint8))


@pytest.mark.parametrize("m,n,l,b,N,e", [(512, 4096, 512, 256, 4, 1), (200, 3000, 70, 128, 2, 1)])
def test_sketch_bf16_parity(ops, m, n, l, b, N, e):
    rng = np.random.default_rng(11)
    A = rng.standard_normal((m, n)).astype(np.float32)
    B = rng.standard_normal((n, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 0)
    h, s = oracle.hash_tables(n, b, N, e, 0)
    At, _ = ops.sketch_left(p, _dev(A), "bf16")
    BtT, _ = ops.sketch_right(p, _dev(B), "bf16")
    ref_l, bd_l = sketch_bounds_left(A, h, s, b)
    ref_r, bd_r = sketch_bounds_right(B, h, s, b)
    assert_bf16_within(At.float().cpu().numpy(), ref_l, bd_l)
    assert_bf16_within(BtT.float().cpu().numpy(), ref_r.T, bd_r.T)


def test_sketch_bf16_input(ops):
    # BF16 operands (the autograd workload's dtype) are read exactly
    m, n, l, b = 96, 4096, 80, 256
    rng = np.random.default_rng(12)
    A = (rng.standard_normal((m, n)) * 0.02).astype(np.float32)
    B = (rng.standard_normal((n, l)) * 0.02).astype(np.float32)
    Ab, Bb = _dev(A, torch.bfloat16), _dev(B, torch.bfloat16)
    A64 = Ab.float().cpu().numpy()
    B64 = Bb.float().cpu().numpy()
    p = ops.plan(n, b, 4, 1, 0)
    h, s = oracle.hash_tables(n, b, 4, 1, 0)
    At, _ = ops.sketch_left(p, Ab, "f32")
    BtT, _ = ops.sketch_right(p, Bb, "f32")
    ref_l, bd_l = sketch_bounds_left(A64, h, s, b)
    ref_r, bd_r = sketch_bounds_right(B64, h, s, b)
    assert_fp32_within(At.cpu().numpy(), ref_l, bd_l)
    assert_fp32_within(BtT.cpu().numpy(), ref_r.T, bd_r.T)


@pytest.mark.parametrize("m,n,l,b,N,e", [(256, 4096, 384, 256, 4, 1), (100, 5000, 33, 128, 3, 1),
                                         (130, 3000, 301, 128, 2, 1),    # in-place strips + packed remainder
                                         (96, 80_000, 260, 512, 2, 1)])  # several windows
def test_sketch_fp8_parity(ops, m, n, l, b, N, e):
    rng = np.random.default_rng(13)
    A = (rng.standard_normal((m, n)) * np.exp(rng.standard_normal((m, 1)) * 3)).astype(np.float32)
    B = rng.standard_normal((n, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 0)
    h, s = oracle.hash_tables(n, b, N, e, 0)
    At, sa = ops.sketch_left(p, _dev(A), "fp8")
    BtT, sb = ops.sketch_right(p, _dev(B), "fp8")
    ref_l, bd_l = sketch_bounds_left(A, h, s, b)
    ref_r, bd_r = sketch_bounds_right(B, h, s, b)
    assert sa.shape == ((N + e) * b // 128, (m + 3) // 4 * 4)      # slice-major scales
    assert_fp8_within(At.float().cpu().numpy(), ops.fp8_scales_by_row(sa, m).cpu().numpy(), ref_l, bd_l)
    assert_fp8_within(BtT.float().cpu().numpy(), ops.fp8_scales_by_row(sb, l).cpu().numpy(), ref_r.T, bd_r.T)


@pytest.mark.parametrize("m,n,l,b,N,e,mask", [(300, 4000, 260, 128, 3, 1, 0b1011),   # packed right remainder
                                               (130, 9000, 384, 256, 2, 2, 0)])        # right in place
def test_sketch_fp8_staged_equals_fused(ops, m, n, l, b, N, e, mask):
    # with room for F x z FP32 sums after the regular workspace the FP8 sketch stages
    # the sums and quantises them in a second pass; codes and scales are the fused
    # epilogue's bits, and within the oracle's FP8 windows
    rng = np.random.default_rng(m + l)
    A = (rng.standard_normal((m, n)) * np.exp(rng.standard_normal((m, 1)) * 3)).astype(np.float32)
    B = rng.standard_normal((n, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 5)
    h, s = oracle.hash_tables(n, b, N, e, 5)
    z = (N + e) * b
    for X, fn, rows in ((A, ops.sketch_left, m), (B, ops.sketch_right, l)):
        base = ops.sketch_workspace(p, rows)
        big = torch.empty((base + 255) // 256 * 256 + rows * z * 4 + 256, dtype=torch.uint8, device="cuda")
        fused, sf = fn(p, _dev(X), "fp8", block_mask=mask)
        staged, ss = fn(p, _dev(X), "fp8", block_mask=mask, workspace=big)
        cols = torch.from_numpy(oracle.selected_columns(mask or (1 << (N + e)) - 1, N + e, b)).cuda()
        sl = torch.from_numpy(np.unique(oracle.selected_columns(mask or (1 << (N + e)) - 1, N + e, b) // 128)).cuda()
        assert torch.equal(fused.view(torch.uint8)[:, cols], staged.view(torch.uint8)[:, cols])
        assert torch.equal(sf[sl, :rows], ss[sl, :rows])
        if fn is ops.sketch_left:
            ref, bd = sketch_bounds_left(A, h, s, b)
        else:
            ref, bd = sketch_bounds_right(B, h, s, b)
            ref, bd = ref.T, bd.T
        c = cols.cpu().numpy()
        scale_rows = ops.fp8_scales_by_row(ss, rows).cpu().numpy()
        slices = c.reshape(-1, 128)[:, 0] // 128
        assert_fp8_within(staged.float().cpu().numpy()[:, c], scale_rows[:, slices], ref[:, c], bd[:, c])


def test_sketch_argument_errors(ops):
    p = ops.plan(1000, 100, 2, 1, 0)          # b = 100: FP8 needs b % 128 == 0
    A = torch.zeros((4, 1000), device="cuda")
    with pytest.raises(ops.OverSketchError):
        ops.sketch_left(p, A, "fp8")
    with pytest.raises(ops.OverSketchError):
        ops.sketch_left(p, torch.zeros((4, 999), device="cuda"), "f32")   # lda < n
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ops.OverSketchError):
        ops.sketch_left(p, A, "f32", workspace=ws)                         # workspace too small


@pytest.mark.parametrize("l", [96, 99, 2100])   # 16-byte rows of U and dG (vector kernel), odd, several 1024-column slabs
def test_unsketch_parity(ops, l):
    m, n, b, N, e = 64, 3000, 128, 4, 1
    mask = 0b10111
    rng = np.random.default_rng(14)
    z = (N + e) * b
    T = rng.standard_normal((m, z)).astype(np.float32)
    U = rng.standard_normal((z, l)).astype(np.float32)
    cols = oracle.selected_columns(mask, N + e, b)
    # the kernels take the kept blocks only, compacted; the oracle reads them in place
    T_sel = np.ascontiguousarray(T[:, cols])
    U_sel = np.ascontiguousarray(U[cols])
    T[:, np.setdiff1d(np.arange(z), cols)] = np.nan     # dropped blocks must never be read
    U[np.setdiff1d(np.arange(z), cols)] = np.nan
    p = ops.plan(n, b, N, e, 2)
    h, s = oracle.hash_tables(n, b, N, e, 2)
    dX = ops.unsketch_cols(p, _dev(T_sel), mask, 0.25).cpu().numpy()
    dG = ops.unsketch_rows(p, _dev(U_sel), mask, 0.25).cpu().numpy()
    T = np.nan_to_num(T)
    U = np.nan_to_num(U)
    ref_x = oracle.unsketch_cols(T, h, s, b, mask, 0.25)
    ref_g = oracle.unsketch_rows(U, h, s, b, mask, 0.25)
    # 4 kept terms: FP32 bound with 5 roundings (4 adds + the scale)
    bx = 5 * 2.0 ** -24 * oracle.unsketch_cols(np.abs(T), h, np.ones_like(s), b, mask, 0.25) + 1e-30
    bg = 5 * 2.0 ** -24 * oracle.unsketch_rows(np.abs(U), h, np.ones_like(s), b, mask, 0.25) + 1e-30
    assert_fp32_within(dX, ref_x, bx)
    assert_fp32_within(dG, ref_g, bg)


@pytest.mark.parametrize("m,n,b,N,e,mask,out", [
    (66, 3000, 128, 4, 1, 0b10111, "f32"),      # rows of T staged 4 per CTA, last CTA partial
    (5, 20_000, 2048, 4, 1, 0b11011, "bf16"),   # 4 per CTA (the autograd workload's k b = 8192), last CTA 1
    (7, 6000, 4096, 4, 1, 0b10111, "bf16"),     # 2 per CTA (64 KB rows), last CTA 1
    (3, 9000, 8192, 4, 1, 0b01111, "f32"),      # one 128 KB row per CTA
    (2, 5000, 16384, 4, 0, 0b1111, "f32"),      # rows too long to stage: the unstaged kernel
])
def test_unsketch_cols_staging(ops, m, n, b, N, e, mask, out):
    rng = np.random.default_rng(m + b)
    P = N + e
    k = bin(mask).count("1")
    T_sel = rng.standard_normal((m, k * b)).astype(np.float32)
    cols = oracle.selected_columns(mask, P, b)
    T = np.zeros((m, P * b))
    T[:, cols] = T_sel
    p = ops.plan(n, b, N, e, 4)
    h, s = oracle.hash_tables(n, b, N, e, 4)
    dX = ops.unsketch_cols(p, _dev(T_sel), mask, 0.5, out_dtype=out).float().cpu().numpy()
    ref = oracle.unsketch_cols(T, h, s, b, mask, 0.5)
    bound = (k + 1) * 2.0 ** -24 * oracle.unsketch_cols(np.abs(T), h, np.ones_like(s), b, mask, 0.5) + 1e-30
    if out == "f32":
        assert_fp32_within(dX, ref, bound)
    else:
        assert_bf16_within(dX, ref, bound)


def test_frob_fp64(ops):
    rng = np.random.default_rng(15)
    X = rng.standard_normal((300, 500)).astype(np.float32)
    Y = rng.standard_normal((300, 500)).astype(np.float32)
    out = ops.frob(_dev(X), _dev(Y)).cpu().numpy()
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    ref = [((X64 - Y64) ** 2).sum(), (Y64 ** 2).sum(), (X64 * Y64).sum()]
    assert np.allclose(out, ref, rtol=1e-12, atol=0)
    out1 = ops.frob(_dev(X)).cpu().numpy()
    assert np.isclose(out1[0], (X64 ** 2).sum(), rtol=1e-12)
    assert np.array_equal(out, ops.frob(_dev(X), _dev(Y)).cpu().numpy())


def test_sketch_block_mask(ops):
    # only the listed blocks are computed; other columns are left untouched
    m, n, l, b, N, e = 96, 3000, 70, 128, 4, 1
    rng = np.random.default_rng(21)
    A = rng.standard_normal((m, n)).astype(np.float32)
    B = rng.standard_normal((n, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 4)
    h, s = oracle.hash_tables(n, b, N, e, 4)
    mask = 0b10110
    At = torch.full((m, p.z), 7.0, device="cuda")
    BtT = torch.full((l, p.z), 7.0, device="cuda")
    ops.sketch_left(p, _dev(A), "f32", out=At, block_mask=mask)
    ops.sketch_right(p, _dev(B), "f32", out=BtT, block_mask=mask)
    ref_l, bd_l = sketch_bounds_left(A, h, s, b)
    ref_r, bd_r = sketch_bounds_right(B, h, s, b)
    cols = oracle.selected_columns(mask, N + e, b)
    other = np.setdiff1d(np.arange(p.z), cols)
    At_h, Bt_h = At.cpu().numpy(), BtT.cpu().numpy()
    assert_fp32_within(At_h[:, cols], ref_l[:, cols], bd_l[:, cols])
    assert_fp32_within(Bt_h[:, cols], ref_r.T[:, cols], bd_r.T[:, cols])
    assert (At_h[:, other] == 7.0).all() and (Bt_h[:, other] == 7.0).all()
    with pytest.raises(ops.OverSketchError, match="MASK"):
        ops.sketch_left(p, _dev(A), "f32", block_mask=1 << 5)
