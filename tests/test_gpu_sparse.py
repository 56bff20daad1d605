"""GPU parity of the sparse-row left sketch (oversketch_sketch_left_sparse and
matmul's OS_OPT_SPARSE_A) against the FP64 oracle, through the C ABI: every
output within the FP32 rounding bound of its sum, at several densities
(including dense rows that overflow the entry buffer), output dtypes, input
dtypes, row alignments and block masks."""
import numpy as np
import pytest

import oracle
from helpers import assert_bf16_within, assert_fp32_within, assert_fp8_within, gpu_lib, sketch_bounds_left

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


def _sparse(rng, m, n, density, scale_rows=False):
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    if scale_rows:
        A = A * np.exp(rng.standard_normal((m, 1)) * 3)
    return A.astype(np.float32)


def _dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


SPARSE_CASES = [
    # m, n, b, N, e, density
    (37, 50_001, 512, 3, 1, 0.01),      # ragged n (not a multiple of 16), 1% nonzeros
    (64, 4096, 256, 4, 1, 0.10),        # small workload's plan, 10%
    (5, 20_000, 512, 3, 1, 1.0),        # dense rows: chunks larger than the entry buffer
    (3, 70_000, 4096, 6, 1, 0.01),      # the interior-point plan shape (k*b = 28672)
    (200, 3000, 32, 2, 1, 0.3),         # b <= 32: one bucket per range
]


@pytest.mark.parametrize("m,n,b,N,e,density", SPARSE_CASES)
def test_sparse_sketch_fp32_parity(ops, m, n, b, N, e, density):
    rng = np.random.default_rng(m * 13 + n)
    A = _sparse(rng, m, n, density)
    p = ops.plan(n, b, N, e, 2)
    h, s = oracle.hash_tables(n, b, N, e, 2)
    At, _ = ops.sketch_left_sparse(p, _dev(A), "f32")
    ref, bd = sketch_bounds_left(A, h, s, b)
    assert_fp32_within(At.cpu().numpy(), ref, bd)
    # bitwise reproducible (fixed order, no atomics)
    At2, _ = ops.sketch_left_sparse(p, _dev(A), "f32")
    assert torch.equal(At, At2)


@pytest.mark.parametrize("out", ["f32", "bf16", "fp8"])
def test_sparse_sketch_mixed_rows(ops, out):
    # rows whose nonzeros fit the one-pass regions beside rows that overflow them
    # (dense rows, and a row dense in one 32nd only) in one launch: every row
    # within the oracle's bound, reruns bitwise equal
    m, n, b, N, e = 24, 100_000, 1024, 5, 1
    rng = np.random.default_rng(77)
    A = _sparse(rng, m, n, 0.01, scale_rows=True)
    A[3] = rng.standard_normal(n)                          # dense
    A[10, 40_000:43_000] = rng.standard_normal(3000)       # one segment dense
    A[17] = 0.0                                            # empty
    A[18, ::5] = rng.standard_normal(len(range(0, n, 5)))  # 20 %: overflows, several flushes
    A = A.astype(np.float32)
    p = ops.plan(n, b, N, e, 6)
    h, s = oracle.hash_tables(n, b, N, e, 6)
    mask = 0b101111
    Y, sc = ops.sketch_left_sparse(p, _dev(A), out, block_mask=mask)
    ref, bd = sketch_bounds_left(A, h, s, b)
    cols = oracle.selected_columns(mask, N + e, b)
    if out == "fp8":
        scale_rows = ops.fp8_scales_by_row(sc, m).cpu().numpy()
        slices = cols.reshape(-1, 128)[:, 0] // 128
        assert_fp8_within(Y.float().cpu().numpy()[:, cols], scale_rows[:, slices], ref[:, cols], bd[:, cols])
    elif out == "bf16":
        assert_bf16_within(Y.float().cpu().numpy()[:, cols], ref[:, cols], bd[:, cols])
    else:
        assert_fp32_within(Y.cpu().numpy()[:, cols], ref[:, cols], bd[:, cols])
    Y2, _ = ops.sketch_left_sparse(p, _dev(A), out, block_mask=mask)
    ct = torch.from_numpy(cols).cuda()
    assert torch.equal(Y.view(torch.uint8)[:, ct] if out == "fp8" else Y[:, ct],
                       Y2.view(torch.uint8)[:, ct] if out == "fp8" else Y2[:, ct])


def test_sparse_sketch_special_rows(ops):
    # all-zero rows, one nonzero at the last index, one at index 0, n = 1
    n, b, N, e = 33_333, 128, 2, 1
    A = np.zeros((4, n), np.float32)
    A[1, n - 1] = 3.5
    A[2, 0] = -2.0
    A[3, ::97] = 1.0
    p = ops.plan(n, b, N, e, 0)
    h, s = oracle.hash_tables(n, b, N, e, 0)
    At, _ = ops.sketch_left_sparse(p, _dev(A), "f32")
    ref, bd = sketch_bounds_left(A, h, s, b)
    assert_fp32_within(At.cpu().numpy(), ref, bd)
    assert (At[0] == 0).all()
    p1 = ops.plan(1, 16, 2, 1, 0)
    A1 = np.array([[2.5], [0.0]], np.float32)
    h1, s1 = oracle.hash_tables(1, 16, 2, 1, 0)
    At1, _ = ops.sketch_left_sparse(p1, _dev(A1), "f32")
    assert np.array_equal(At1.cpu().numpy(), oracle.sketch_left(A1, h1, s1, 16))


def test_sparse_sketch_col_scale_and_unaligned_rows(ops):
    m, n, b, N, e = 50, 40_000, 256, 4, 1
    rng = np.random.default_rng(5)
    A = _sparse(rng, m, n, 0.02)
    cs = np.sqrt(10.0 ** rng.uniform(-6, 6, n)).astype(np.float32)
    p = ops.plan(n, b, N, e, 9)
    h, s = oracle.hash_tables(n, b, N, e, 9)
    ref, bd = sketch_bounds_left(A, h, s, b, cs)
    At, _ = ops.sketch_left_sparse(p, _dev(A), "f32", col_scale=_dev(cs))
    assert_fp32_within(At.cpu().numpy(), ref, bd)
    # rows 4 bytes apart from 16-byte alignment (lda = n + 1): scalar loads, no prefetch
    Ap = np.zeros((m, n + 1), np.float32)
    Ap[:, :n] = A
    Ad = _dev(Ap)[:, :n]
    At_u, _ = ops.sketch_left_sparse(p, Ad, "f32", col_scale=_dev(cs))
    assert torch.equal(At_u, At)


def test_sparse_sketch_bf16_input_and_outputs(ops):
    m, n, b, N, e = 40, 30_000, 256, 3, 1
    rng = np.random.default_rng(6)
    A = _sparse(rng, m, n, 0.05, scale_rows=True)
    A16 = torch.from_numpy(A).to(torch.bfloat16)
    A64 = A16.float().numpy().astype(np.float64)
    p = ops.plan(n, b, N, e, 3)
    h, s = oracle.hash_tables(n, b, N, e, 3)
    ref, bd = sketch_bounds_left(A64, h, s, b)
    Ab = A16.cuda()
    At32, _ = ops.sketch_left_sparse(p, Ab, "f32")
    assert_fp32_within(At32.cpu().numpy(), ref, bd)
    At16, _ = ops.sketch_left_sparse(p, Ab, "bf16")
    assert_bf16_within(At16.float().cpu().numpy(), ref, bd)
    At8, sc = ops.sketch_left_sparse(p, Ab, "fp8")
    assert_fp8_within(At8.float().cpu().numpy(), ops.fp8_scales_by_row(sc, m).cpu().numpy(), ref, bd)
    Att, _ = ops.sketch_left_sparse(p, Ab, "tf32x2")
    hi, lo = ops.tf32_planes(Att)
    assert torch.equal(hi.double() + lo.double(), At32.double())
    assert ((hi.view(torch.int32) & 0x1FFF) == 0).all()


def test_sparse_sketch_block_mask_and_limits(ops):
    m, n, b, N, e = 30, 20_000, 128, 4, 1
    rng = np.random.default_rng(8)
    A = _sparse(rng, m, n, 0.03)
    p = ops.plan(n, b, N, e, 4)
    h, s = oracle.hash_tables(n, b, N, e, 4)
    mask = 0b10110
    At = torch.full((m, p.z), 7.0, device="cuda")
    ops.sketch_left_sparse(p, _dev(A), "f32", out=At, block_mask=mask)
    ref, bd = sketch_bounds_left(A, h, s, b)
    cols = oracle.selected_columns(mask, N + e, b)
    other = np.setdiff1d(np.arange(p.z), cols)
    At_h = At.cpu().numpy()
    assert_fp32_within(At_h[:, cols], ref[:, cols], bd[:, cols])
    assert (At_h[:, other] == 7.0).all()
    with pytest.raises(ops.OverSketchError, match="MASK"):
        ops.sketch_left_sparse(p, _dev(A), "f32", block_mask=1 << 5)
    # k * b above the on-chip limit (5 * 8192 > 32768) is refused; three blocks fit
    pb = ops.plan(n, 8192, 4, 1, 0)
    with pytest.raises(ops.OverSketchError, match="UNSUPPORTED"):
        ops.sketch_left_sparse(pb, _dev(A), "f32")
    At3, _ = ops.sketch_left_sparse(pb, _dev(A), "f32", block_mask=0b00111)
    hb, sb = oracle.hash_tables(n, 8192, 4, 1, 0)
    ref3, bd3 = sketch_bounds_left(A, hb, sb, 8192)
    c3 = oracle.selected_columns(0b00111, 5, 8192)
    assert_fp32_within(At3.cpu().numpy()[:, c3], ref3[:, c3], bd3[:, c3])


def test_sparse_matmul_flag(ops):
    # the whole product with OS_OPT_SPARSE_A, general and symmetric with sqrt(D)
    m, n, l, b, N, e = 96, 60_000, 80, 512, 6, 1
    rng = np.random.default_rng(10)
    A = _sparse(rng, m, n, 0.01)
    B = rng.standard_normal((n, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 0)
    h, s = oracle.hash_tables(n, b, N, e, 0)
    mask = 0b1110111
    C = ops.matmul(p, _dev(A), _dev(B), mask, "bf16", sparse_a=True).cpu().numpy()
    Cref = oracle.masked_product(oracle.round_bf16(oracle.sketch_left(A, h, s, b)),
                                 oracle.round_bf16(oracle.sketch_right(B, h, s, b)), b, mask)
    assert oracle.rel_frob(C, Cref) <= 1e-4
    Cd = ops.matmul(p, _dev(A), _dev(B), mask, "bf16").cpu().numpy()
    assert oracle.rel_frob(C, Cd) <= 1e-4
    cs = np.sqrt(10.0 ** rng.uniform(-6, 6, n)).astype(np.float32)
    H = ops.matmul(p, _dev(A), None, mask, "bf16", col_scale=_dev(cs), symmetric=True, sparse_a=True).cpu().numpy()
    At_q = oracle.round_bf16(oracle.sketch_left(A, h, s, b, cs.astype(np.float64)))
    assert oracle.rel_frob(H, oracle.masked_product(At_q, At_q.T, b, mask)) <= 1e-4
    assert oracle.rel_frob(H, H.T) <= 1e-6


def test_sparse_sketch_table_plan_matches_hashed_plan(ops):
    # a plan built from explicit tables (the bucket codes are read from the table)
    # and the seeded plan with the same tables (codes recomputed from the seed)
    m, n, b, N, e = 20, 30_000, 256, 3, 1
    rng = np.random.default_rng(12)
    A = _sparse(rng, m, n, 0.02)
    h, s = oracle.hash_tables(n, b, N, e, 17)
    p_seed = ops.plan(n, b, N, e, 17)
    p_tab = ops.plan_from_tables(h, s, b, N, e)
    At_seed, _ = ops.sketch_left_sparse(p_seed, _dev(A), "f32")
    At_tab, _ = ops.sketch_left_sparse(p_tab, _dev(A), "f32")
    assert torch.equal(At_seed, At_tab)
    ref, bd = sketch_bounds_left(A, h, s, b)
    assert_fp32_within(At_tab.cpu().numpy(), ref, bd)
    # an injective table (h_j(i) = (i + j) mod b, b >= n) makes the product exact
    n2, b2 = 500, 512
    h2 = np.array([[(i + j) % b2 for i in range(n2)] for j in range(3)], np.uint32)
    s2 = np.where(rng.random((3, n2)) < 0.5, -1, 1).astype(np.int8)
    A2 = _sparse(rng, 8, n2, 0.2)
    p2 = ops.plan_from_tables(h2, s2, b2, 2, 1)
    At2, _ = ops.sketch_left_sparse(p2, _dev(A2), "f32")
    assert np.array_equal(At2.cpu().numpy(), oracle.sketch_left(A2, h2, s2, b2))
