"""GPU parity of the tensor-core (tcgen05) masked GEMM and of the BF16
OverSketch path, through the C ABI."""
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


def _bf16(x):
    """Host FP32 -> device BF16 and the exact FP64 values of those BF16 numbers."""
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).cuda()
    return t, t.float().cpu().numpy().astype(np.float64)


GEMM_CASES = [
    # m, l, b, N, e, mask
    (128, 256, 64, 2, 1, 0b011),           # one tile, one K block per sketch block
    (256, 512, 256, 4, 1, 0b11011),        # small workload's block shape
    (300, 700, 128, 3, 2, 0b10101),        # ragged m and l, non-contiguous kept blocks
    (1, 1, 64, 1, 0, 0b1),                 # single element
    (1000, 130, 1024, 2, 1, 0b110),        # K = 2048, l < tile width
    (640, 1536, 512, 8, 2, 0b1110111101),  # many tiles (persistent loop, both TMEM buffers)
    (2100, 3000, 256, 4, 1, 0b11101),      # more tile pairs than clusters, the last pair half empty
]


@pytest.mark.parametrize("m,l,b,N,e,mask", GEMM_CASES)
def test_gemm_bf16_parity(ops, m, l, b, N, e, mask):
    rng = np.random.default_rng(m * 31 + l)
    z = (N + e) * b
    At, At64 = _bf16(rng.standard_normal((m, z)))
    Bt, Bt64 = _bf16(rng.standard_normal((l, z)))
    p = ops.plan(max(z, 64), b, N, e, 0)
    C = ops.gemm_masked(p, At, Bt, mask).cpu().numpy()
    ref = oracle.masked_product(At64, Bt64.T, b, mask)
    k = bin(mask).count("1")
    K = k * b
    absref = oracle.masked_product(np.abs(At64), np.abs(Bt64).T, b, mask)
    bound = 2 * K * 2.0 ** -24 * absref + 1e-30
    assert (np.abs(C - ref) <= bound).all()
    assert oracle.rel_frob(C, ref) <= 1e-5


def test_gemm_bf16_alpha_beta(ops):
    rng = np.random.default_rng(7)
    b, N, e = 128, 3, 1
    z = (N + e) * b
    At, At64 = _bf16(rng.standard_normal((200, z)))
    Bt, Bt64 = _bf16(rng.standard_normal((300, z)))
    C0 = rng.standard_normal((200, 300)).astype(np.float32)
    C = torch.from_numpy(C0.copy()).cuda()
    p = ops.plan(1024, b, N, e, 0)
    ops.gemm_masked(p, At, Bt, 0b1011, alpha=0.25, beta=-1.5, C=C)
    ref = 0.25 * oracle.masked_product(At64, Bt64.T, b, 0b1011) - 1.5 * C0      # the library's 1/k, times alpha
    assert oracle.rel_frob(C.cpu().numpy(), ref) <= 1e-5


def test_gemm_bf16_reproducible(ops):
    rng = np.random.default_rng(8)
    b, N, e = 256, 4, 1
    z = (N + e) * b
    At, _ = _bf16(rng.standard_normal((512, z)))
    Bt, _ = _bf16(rng.standard_normal((768, z)))
    p = ops.plan(4096, b, N, e, 0)
    C1 = ops.gemm_masked(p, At, Bt, 0b10111)
    C2 = ops.gemm_masked(p, At, Bt, 0b10111)
    assert torch.equal(C1, C2)
    assert ops.device_status() == 0


def _bf16_oracle(A, B, w, h, s):
    At_q = oracle.round_bf16(oracle.sketch_left(A, h, s, w.b))
    Bt_q = oracle.round_bf16(oracle.sketch_right(B, h, s, w.b))
    return oracle.masked_product(At_q, Bt_q, w.b, w.mask)


def test_small_workload_bf16(ops):
    w = W.SMALL
    A, B = w.left(), w.right()
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    C = ops.matmul(p, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), w.mask, "bf16")
    h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    assert oracle.rel_frob(C.cpu().numpy(), _bf16_oracle(A, B, w, h, s)) <= 1e-4


@pytest.mark.parametrize("m,n,l,b,N,e,mask", [(300, 5000, 200, 128, 3, 1, 0b1101),
                                              (130, 4096, 1000, 1024, 2, 1, 0b011)])
def test_matmul_bf16_parity(ops, m, n, l, b, N, e, mask):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    B = rng.standard_normal((n, l)).astype(np.float32)
    w = W.Workload("t", m, n, l, b, N, e, mask)
    p = ops.plan(n, b, N, e, 3)
    C = ops.matmul(p, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), mask, "bf16")
    h, s = oracle.hash_tables(n, b, N, e, 3)
    assert oracle.rel_frob(C.cpu().numpy(), _bf16_oracle(A, B, w, h, s)) <= 1e-4


def test_symmetric_product(ops):
    # H = (1/k) A~_sel A~_sel^T with the column scale sqrt(D) (Sec. 5.2's Hessian form)
    m, n, b, N, e, mask = 256, 8192, 256, 6, 1, 0b1110111
    rng = np.random.default_rng(9)
    A = (rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.05)).astype(np.float32)
    cs = np.sqrt(10.0 ** rng.uniform(-6, 6, n)).astype(np.float32)
    p = ops.plan(n, b, N, e, 0)
    H = ops.matmul(p, torch.from_numpy(A).cuda(), None, mask, "bf16",
                   col_scale=torch.from_numpy(cs).cuda(), symmetric=True).cpu().numpy()
    h, s = oracle.hash_tables(n, b, N, e, 0)
    At_q = oracle.round_bf16(oracle.sketch_left(A, h, s, b, cs))
    ref = oracle.masked_product(At_q, At_q.T, b, mask)
    assert oracle.rel_frob(H, ref) <= 1e-4
    assert oracle.rel_frob(H, H.T) <= 1e-6


@pytest.mark.parametrize("m,b,N,e,mask,beta", [
    (300, 128, 3, 2, 0b10101, 0.0),       # two tile pairs per side, the last pair half empty
    (1000, 256, 4, 1, 0b11011, 0.0),      # 4 x 4 pairs: 10 computed, 6 mirrored
    (4096, 512, 3, 1, 0b1011, 0.5),       # 16 x 16 pairs (more than the clusters), beta C added
    (1, 64, 1, 0, 0b1, 0.0),              # a single element
])
def test_gemm_bf16_symmetric_lower_triangle(ops, m, b, N, e, mask, beta):
    # At At^T with the same operand twice computes the tile pairs on and below the
    # diagonal and stores each off-diagonal one transposed as well: the same bits
    # as the general kernel in the lower triangle, an exactly symmetric C, and
    # within the FP32 accumulation bound of the oracle everywhere
    rng = np.random.default_rng(m + b)
    z = (N + e) * b
    At, At64 = _bf16(rng.standard_normal((m, z)))
    p = ops.plan(max(z, 64), b, N, e, 0)
    C0 = torch.from_numpy(rng.standard_normal((m, m)).astype(np.float32)).cuda()
    C_sym = ops.gemm_masked(p, At, At, mask, beta=beta, C=C0.clone())
    C_gen = ops.gemm_masked(p, At, At.clone(), mask, beta=beta, C=C0.clone())
    low = torch.tril(torch.ones((m, m), dtype=torch.bool, device="cuda"))
    pair = torch.arange(m, device="cuda") // 256
    low |= pair[:, None] == pair[None, :]            # whole diagonal pairs come from the kernel
    assert torch.equal(C_sym[low], C_gen[low])
    assert torch.equal(C_sym, C_sym.T) or beta != 0.0
    ref = oracle.masked_product(At64, At64.T, b, mask) + beta * C0.cpu().numpy().astype(np.float64)
    K = bin(mask).count("1") * b
    absref = oracle.masked_product(np.abs(At64), np.abs(At64).T, b, mask) + abs(beta) * np.abs(C0.cpu().numpy())
    bound = 2 * (K + 1) * 2.0 ** -24 * absref + 1e-30
    assert (np.abs(C_sym.cpu().numpy() - ref) <= bound).all()


def _split_tf32(x):
    """hi = x with the low 13 mantissa bits cleared (exact in TF32), lo = x - hi."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    hi = (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    return hi, (x - hi).astype(np.float32)


@pytest.mark.parametrize("m,l,b,N,e,mask", [(128, 128, 32, 2, 1, 0b011), (300, 700, 128, 3, 2, 0b10101),
                                            (1000, 130, 1024, 2, 1, 0b110), (1, 1, 64, 1, 0, 0b1),
                                            (2100, 1000, 128, 3, 1, 0b1011)])
def test_gemm_tf32x3_parity(ops, m, l, b, N, e, mask):
    # FP32 operands as hi/lo TF32 planes: three tensor-core products give FP32 accuracy
    rng = np.random.default_rng(m + 7 * l)
    z = (N + e) * b
    A = rng.standard_normal((m, z)).astype(np.float32)
    B = rng.standard_normal((l, z)).astype(np.float32)
    Ah, Al = _split_tf32(A)
    Bh, Bl = _split_tf32(B)
    Abuf = torch.from_numpy(np.stack([Ah, Al])).cuda()
    Bbuf = torch.from_numpy(np.stack([Bh, Bl])).cuda()
    p = ops.plan(max(z, 64), b, N, e, 0)
    C = ops.gemm_masked(p, Abuf[0], Bbuf[0], mask, dtype="tf32x2").cpu().numpy()
    ref = oracle.masked_product(A.astype(np.float64), B.astype(np.float64).T, b, mask)
    assert oracle.rel_frob(C, ref) <= 1e-5


def test_sketch_tf32x2_planes(ops):
    m, n, l, b, N, e = 200, 3000, 300, 128, 3, 1
    rng = np.random.default_rng(17)
    A = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
    B = torch.from_numpy(rng.standard_normal((n, l)).astype(np.float32)).cuda()
    p = ops.plan(n, b, N, e, 0)
    for X, fn in ((A, ops.sketch_left), (B, ops.sketch_right)):
        ref, _ = fn(p, X, "f32")
        out, _ = fn(p, X, "tf32x2")
        hi, lo = ops.tf32_planes(out)
        hi_u = hi.contiguous().view(torch.int32).cpu().numpy()
        assert (hi_u & 0x1FFF == 0).all()                     # hi is exact in TF32
        assert torch.equal(hi + lo, ref)                      # hi + lo is the FP32 sum


def test_small_workload_fp32_tensor_path(ops):
    # matmul with FP32 GEMM dtype runs 3xTF32 on the tensor cores (b % 32 == 0)
    w = W.SMALL
    A, B = w.left(), w.right()
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    C = ops.matmul(p, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), w.mask, "f32")
    h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    assert oracle.rel_frob(C.cpu().numpy(), oracle.oversketch(A, B, h, s, w.b, w.mask)) <= 1e-5


def _fp8_operand(rng, rows, z, emin=-8, emax=8):
    """Random E4M3 codes (no NaN codes) and slice-major power-of-two scales;
    returns device codes, device scales and the exact FP64 dequantised matrix."""
    codes = rng.integers(0, 256, size=(rows, z), dtype=np.uint8)
    codes[(codes & 0x7F) == 0x7F] = 0x38                       # NaN codes -> 1.0
    q = torch.from_numpy(codes).cuda().view(torch.float8_e4m3fn)
    vals = q.float().cpu().numpy().astype(np.float64)
    nsl, ld = z // 128, (rows + 3) // 4 * 4
    e = rng.integers(emin, emax + 1, size=(nsl, ld))
    sc = np.ldexp(1.0, e).astype(np.float32)
    sc[:, rows:] = np.nan                                      # padding rows must never be read
    deq = vals * np.repeat(np.ldexp(1.0, e[:, :rows]).T, 128, axis=1)
    return q, torch.from_numpy(sc).cuda(), deq


FP8_CASES = [
    # m, l, b, N, e, mask
    (128, 224, 128, 2, 1, 0b011),          # one tile
    (300, 700, 256, 3, 2, 0b10101),        # ragged m and l, non-contiguous kept blocks
    (1, 1, 128, 1, 0, 0b1),                # single element
    (1000, 130, 1024, 2, 1, 0b110),        # K = 2048, l < tile width
    (129, 449, 128, 4, 1, 0b11110),        # l just past two tile widths
    (640, 1536, 512, 8, 2, 0b1110111101),  # many tiles (persistent loop, both accumulators)
    (2100, 3000, 256, 4, 1, 0b11101),      # more tile pairs than clusters, the last pair half empty
]


@pytest.mark.parametrize("m,l,b,N,e,mask", FP8_CASES)
def test_gemm_fp8_parity(ops, m, l, b, N, e, mask):
    # block-scaled E4M3 x E4M3 products are exact in FP32; only the accumulation rounds
    rng = np.random.default_rng(m * 17 + l)
    z = (N + e) * b
    At, sa, A64 = _fp8_operand(rng, m, z)
    Bt, sb, B64 = _fp8_operand(rng, l, z)
    p = ops.plan(max(z, 64), b, N, e, 0)
    C = ops.gemm_masked(p, At, Bt, mask, a_scales=sa, b_scales=sb).cpu().numpy()
    ref = oracle.masked_product(A64, B64.T, b, mask)
    K = bin(mask).count("1") * b
    absref = oracle.masked_product(np.abs(A64), np.abs(B64).T, b, mask)
    bound = 2 * K * 2.0 ** -24 * absref + 1e-30
    assert np.isfinite(C).all()
    assert (np.abs(C - ref) <= bound).all()


def test_gemm_fp8_extreme_scales(ops):
    # wide scale range, and the smallest UE8M0 scale 2^-127 (a subnormal FP32 value)
    rng = np.random.default_rng(21)
    m, l, b, N, e, mask = 256, 224, 128, 2, 0, 0b11
    z = (N + e) * b
    At, sa, A64 = _fp8_operand(rng, m, z, -60, 40)
    Bt, sb, B64 = _fp8_operand(rng, l, z, -40, 40)
    sa[0, :m] = 2.0 ** -127
    A64[:, :128] = At.float().cpu().numpy()[:, :128].astype(np.float64) * 2.0 ** -127
    p = ops.plan(z, b, N, e, 0)
    C = ops.gemm_masked(p, At, Bt, mask, alpha=1.0, a_scales=sa, b_scales=sb).cpu().numpy()
    ref = oracle.masked_product(A64, B64.T, b, mask)          # the library applies 1/k, as the oracle does
    absref = oracle.masked_product(np.abs(A64), np.abs(B64).T, b, mask)
    assert np.isfinite(C).all()
    assert (np.abs(C - ref) <= 2 * z * 2.0 ** -24 * absref + 1e-37).all()


def _fp8_oracle(A, B, w, h, s, cs=None):
    At_q = oracle.dequantize_fp8_rows(*oracle.quantize_fp8_rows(oracle.sketch_left(A, h, s, w.b, cs)))
    Bt_q = oracle.dequantize_fp8_rows(*oracle.quantize_fp8_rows(oracle.sketch_right(B, h, s, w.b)))
    return oracle.masked_product(At_q, Bt_q, w.b, w.mask)


def test_small_workload_fp8(ops):
    w = W.SMALL
    A, B = w.left(), w.right()
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    C = ops.matmul(p, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), w.mask, "fp8")
    h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    assert oracle.rel_frob(C.cpu().numpy(), _fp8_oracle(A, B, w, h, s)) <= 1e-3


@pytest.mark.parametrize("m,n,l,b,N,e,mask", [(300, 5000, 200, 128, 3, 1, 0b1101),
                                              (130, 4096, 1000, 1024, 2, 1, 0b011)])
def test_matmul_fp8_parity(ops, m, n, l, b, N, e, mask):
    rng = np.random.default_rng(n + 1)
    A = (rng.standard_normal((m, n)) * np.exp(rng.standard_normal((m, 1)) * 2)).astype(np.float32)
    B = rng.standard_normal((n, l)).astype(np.float32)
    w = W.Workload("t", m, n, l, b, N, e, mask)
    p = ops.plan(n, b, N, e, 5)
    C = ops.matmul(p, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), mask, "fp8")
    h, s = oracle.hash_tables(n, b, N, e, 5)
    assert oracle.rel_frob(C.cpu().numpy(), _fp8_oracle(A, B, w, h, s)) <= 1e-3


def test_symmetric_product_fp8(ops):
    m, n, b, N, e, mask = 200, 6000, 256, 4, 1, 0b11101
    rng = np.random.default_rng(23)
    A = rng.standard_normal((m, n)).astype(np.float32)
    p = ops.plan(n, b, N, e, 0)
    H = ops.matmul(p, torch.from_numpy(A).cuda(), None, mask, "fp8", symmetric=True).cpu().numpy()
    h, s = oracle.hash_tables(n, b, N, e, 0)
    At_q = oracle.dequantize_fp8_rows(*oracle.quantize_fp8_rows(oracle.sketch_left(A, h, s, b)))
    assert oracle.rel_frob(H, oracle.masked_product(At_q, At_q.T, b, mask)) <= 1e-3
    assert oracle.rel_frob(H, H.T) <= 1e-6
