"""GPU parity of the whole product (left sketch, right sketch, masked GEMM)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import gpu_lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1811_02653_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_small_workload_fp32(ops):
    # A 512x4096, B 4096x512, b=256, N=4, e=1, block 2 dropped, seed 0
    w = W.SMALL
    A, B = w.left(), w.right()
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    C = ops.matmul(p, _dev(A), _dev(B), w.mask, "f32").cpu().numpy()
    h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    C_ref = oracle.oversketch(A, B, h, s, w.b, w.mask)
    assert oracle.rel_frob(C, C_ref) <= 1e-5
    # the error of the sketched product itself against the exact A B matches
    # the closed-form expectation of appendix B (one draw; many entries)
    AB = A.astype(np.float64) @ B.astype(np.float64)
    sq = ((C - AB) ** 2).sum()
    expect = oracle.expected_sq_error(A, B, w.k, w.b)
    assert 0.8 < sq / expect < 1.25


@pytest.mark.parametrize("m,n,l,b,N,e,mask", [
    (300, 2000, 130, 128, 3, 2, 0b10110),      # ragged, non-contiguous kept blocks
    (64, 1024, 64, 64, 4, 1, 0b00011),         # k = 2 < N (graceful degradation)
    (1, 512, 1, 32, 2, 0, 0b11),               # single row and column
    (130, 4096, 129, 1024, 2, 1, 0b101),
])
def test_matmul_fp32_parity(ops, m, n, l, b, N, e, mask):
    rng = np.random.default_rng(m + n + l)
    A = rng.standard_normal((m, n)).astype(np.float32)
    B = rng.standard_normal((n, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 5)
    C = ops.matmul(p, _dev(A), _dev(B), mask, "f32").cpu().numpy()
    h, s = oracle.hash_tables(n, b, N, e, 5)
    assert oracle.rel_frob(C, oracle.oversketch(A, B, h, s, b, mask)) <= 1e-5


def test_injective_plan_is_exact(ops):
    # b >= n with an injective hash: S_j S_j^T = I and C = AB up to the FP32 path's
    # rounding (3xTF32 on the tensor cores: within the FP32 gate of 1e-5)
    n, b, N, e = 200, 256, 3, 1
    rng = np.random.default_rng(3)
    A = rng.standard_normal((96, n)).astype(np.float32)
    B = rng.standard_normal((n, 80)).astype(np.float32)
    h = np.array([[(i + 17 * j) % b for i in range(n)] for j in range(N + e)], np.uint32)
    s = np.where(rng.random((N + e, n)) < 0.5, -1, 1).astype(np.int8)
    p = ops.plan_from_tables(h, s, b, N, e)
    C = ops.matmul(p, _dev(A), _dev(B), 0b1011, "f32").cpu().numpy()
    assert oracle.rel_frob(C, A.astype(np.float64) @ B.astype(np.float64)) < 1e-5


def test_gemm_masked_beta_and_alpha(ops):
    n, b, N, e = 1024, 64, 3, 1
    rng = np.random.default_rng(4)
    z = (N + e) * b
    At = rng.standard_normal((70, z)).astype(np.float32)
    BtT = rng.standard_normal((90, z)).astype(np.float32)
    C0 = rng.standard_normal((70, 90)).astype(np.float32)
    p = ops.plan(n, b, N, e, 0)
    C = _dev(C0.copy())
    ops.gemm_masked(p, _dev(At), _dev(BtT), 0b1101, alpha=0.5, beta=2.0, C=C)
    ref = 0.5 * oracle.masked_product(At, BtT.T, b, 0b1101) + 2.0 * C0          # the library's 1/k, times alpha
    assert oracle.rel_frob(C.cpu().numpy(), ref) <= 1e-6


def test_matmul_mask_errors(ops):
    p = ops.plan(512, 32, 3, 1, 0)
    A = torch.zeros((8, 512), device="cuda")
    B = torch.zeros((512, 8), device="cuda")
    for bad in (0, 1 << 4, 1 << 10):
        with pytest.raises(ops.OverSketchError, match="MASK"):
            ops.matmul(p, A, B, bad, "f32")
    with pytest.raises(ops.OverSketchError):
        ops.matmul(p, torch.zeros((8, 500), device="cuda"), B, 0b111, "f32")   # n mismatch


@pytest.fixture(scope="module")
def square(ops):
    """The full-size square workload (16384 x 65536 x 16384, FP32 operands with
    the rank-64 spike) on the device, with sampled rows of A and columns of B
    that the oracle regenerates one by one, and their oracle sketches."""
    w = W.SQUARE
    A = torch.from_numpy(w.left()).cuda()
    Bt_host = w.right_cols(range(w.l))                       # l x n (columns of B)
    B = torch.from_numpy(Bt_host).cuda().t().contiguous()
    del Bt_host
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    rows = [0, 1, 777, 8191, 12288, 16383]
    cols = [0, 5, 4096, 12345, 16383]
    h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    At64 = oracle.sketch_left(w.left_rows(rows), h, s, w.b)          # FP64 sketches of the samples
    Bt64 = oracle.sketch_right(w.right_cols(cols).T, h, s, w.b)
    yield w, A, B, p, rows, cols, At64, Bt64
    del A, B


def test_square_workload_sampled_fp32(ops, square):
    # full-size square workload, FP32 path (3xTF32 GEMM), sampled rows and columns
    w, A, B, p, rows, cols, At64, Bt64 = square
    C = ops.matmul(p, A, B, w.mask, "f32")
    C_s = C[rows][:, cols].cpu().numpy()
    assert oracle.rel_frob(C_s, oracle.masked_product(At64, Bt64, w.b, w.mask)) <= 1e-5


def test_square_workload_sampled_bf16(ops, square):
    # the headline form: BF16 sketches (RNE of the FP32 sums) and the CTA-pair
    # tcgen05 GEMM; the oracle rounds its FP64 sketches to BF16 the same way
    w, A, B, p, rows, cols, At64, Bt64 = square
    C = ops.matmul(p, A, B, w.mask, "bf16")
    C_s = C[rows][:, cols].cpu().numpy()
    ref = oracle.masked_product(oracle.round_bf16(At64), oracle.round_bf16(Bt64), w.b, w.mask)
    assert oracle.rel_frob(C_s, ref) <= 1e-4
    assert ops.device_status() == 0


def test_square_workload_sampled_fp8(ops, square):
    # FP8 E4M3 sketches with per-(row, 128-column) UE8M0 scales and the
    # block-scaled tcgen05 GEMM; the oracle quantises its FP64 sketch rows with
    # the same scale rule
    w, A, B, p, rows, cols, At64, Bt64 = square
    C = ops.matmul(p, A, B, w.mask, "fp8")
    C_s = C[rows][:, cols].cpu().numpy()
    Aq = oracle.dequantize_fp8_rows(*oracle.quantize_fp8_rows(At64))
    Bq = oracle.dequantize_fp8_rows(*oracle.quantize_fp8_rows(Bt64.T))
    ref = oracle.masked_product(Aq, Bq.T, w.b, w.mask)
    assert oracle.rel_frob(C_s, ref) <= 1e-3
    assert ops.device_status() == 0


def test_empty_operands(ops):
    # an empty C (m = 0 or l = 0) is OS_OK with nothing launched, even where the
    # empty tensors carry no storage
    n, b, N, e = 512, 64, 4, 1
    p = ops.plan(n, b, N, e, 0)
    mask = 0b11011
    A0 = torch.empty((0, n), device="cuda")
    B = torch.randn((n, 96), device="cuda")
    A = torch.randn((64, n), device="cuda")
    B0 = torch.empty((n, 0), device="cuda")
    for gd in ("f32", "bf16"):
        assert ops.matmul(p, A0, B, mask, gd).shape == (0, 96)
        assert ops.matmul(p, A, B0, mask, gd).shape == (64, 0)
    assert ops.matmul(p, A0, None, mask, "bf16", symmetric=True).shape == (0, 0)
    At, _ = ops.sketch_left(p, A0, "bf16")
    BtT, _ = ops.sketch_right(p, B0, "bf16")
    assert At.shape == (0, p.z) and BtT.shape == (0, p.z)
    Bt1, _ = ops.sketch_right(p, B, "bf16")
    assert ops.gemm_masked(p, At, Bt1, mask).shape == (0, 96)
    masks = torch.full((1, 1), mask, dtype=torch.int64, device="cuda")
    assert ops.gemm_masked_blocks(p, At, Bt1, masks, 256, 256).shape == (0, 96)
    T0 = torch.empty((0, 4 * b), device="cuda")
    assert ops.unsketch_cols(p, T0, mask, 1.0).shape == (0, n)
    C = ops.matmul_host(p, torch.empty((0, n)), torch.randn((n, 96)), mask, "bf16")
    torch.cuda.synchronize()
    assert C.shape == (0, 96)
