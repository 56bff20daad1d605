"""oversketch_matmul_host: the whole product from and to host memory with the
transfers overlapped, against the device entry point on the same inputs (the
same kernels run on the same operands, chunked by rows of A and panels of C:
identical results) and against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from helpers import gpu_lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


@pytest.mark.parametrize("m,n,l,b,N,e,dtype", [
    (1000, 8192, 777, 256, 4, 1, "bf16"),      # ragged m and l; A in 8 chunks, C in 4 panels
    (300, 4096, 1030, 128, 3, 2, "bf16"),
    (257, 4096, 300, 256, 4, 1, "f32"),        # 3xTF32: one chunk, one panel
    (384, 4096, 256, 256, 4, 1, "fp8"),
])
def test_host_matches_device(ops, m, n, l, b, N, e, dtype):
    rng = np.random.default_rng(m + l)
    A = rng.standard_normal((m, n)).astype(np.float32)
    B = rng.standard_normal((n, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 5)
    mask = ((1 << (N + e)) - 1) & ~(1 << 1)
    A_h = torch.from_numpy(A).pin_memory()
    B_h = torch.from_numpy(B).pin_memory()
    C_h = ops.matmul_host(p, A_h, B_h, mask, dtype)
    torch.cuda.synchronize()
    C_d = ops.matmul(p, A_h.cuda(), B_h.cuda(), mask, dtype).cpu()
    assert torch.equal(C_h, C_d)
    h, s = oracle.hash_tables(n, b, N, e, 5)
    if dtype == "bf16":
        ref = oracle.masked_product(oracle.round_bf16(oracle.sketch_left(A, h, s, b)),
                                    oracle.round_bf16(oracle.sketch_right(B, h, s, b)), b, mask)
        assert oracle.rel_frob(C_h.numpy(), ref) <= 1e-4
    elif dtype == "f32":
        assert oracle.rel_frob(C_h.numpy(), oracle.oversketch(A, B, h, s, b, mask)) <= 1e-5


@pytest.mark.parametrize("l", [777, 512])
def test_host_bf16_operands_match_device(ops, l):
    # BF16 operands: B's device copy gets 16-byte rows and is gathered in place,
    # the device entry point on B.cuda() packs it when l is not a multiple of 8;
    # the sums are the same in the same order, so C is bitwise equal
    m, n, b, N, e = 600, 8192, 256, 4, 1
    rng = np.random.default_rng(l)
    A = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).to(torch.bfloat16)
    B = torch.from_numpy(rng.standard_normal((n, l)).astype(np.float32)).to(torch.bfloat16)
    p = ops.plan(n, b, N, e, 3)
    mask = 0b11101
    C_h = ops.matmul_host(p, A.pin_memory(), B.pin_memory(), mask, "bf16")
    torch.cuda.synchronize()
    C_d = ops.matmul(p, A.cuda(), B.cuda(), mask, "bf16").cpu()
    assert torch.equal(C_h, C_d)
    h, s = oracle.hash_tables(n, b, N, e, 3)
    A64 = A.float().numpy().astype(np.float64)
    B64 = B.float().numpy().astype(np.float64)
    ref = oracle.masked_product(oracle.round_bf16(oracle.sketch_left(A64, h, s, b)),
                                oracle.round_bf16(oracle.sketch_right(B64, h, s, b)), b, mask)
    assert oracle.rel_frob(C_h.numpy(), ref) <= 1e-4


def test_host_symmetric_sparse_unpinned_and_strided(ops):
    m, n, b, N, e = 700, 20_000, 512, 6, 1
    rng = np.random.default_rng(3)
    A = (rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.02)).astype(np.float32)
    cs = np.sqrt(10.0 ** rng.uniform(-6, 6, n)).astype(np.float32)
    p = ops.plan(n, b, N, e, 0)
    mask = 0b1110111
    csd = torch.from_numpy(cs).cuda()
    H = ops.matmul_host(p, torch.from_numpy(A), None, mask, "bf16", col_scale=csd, symmetric=True,
                        sparse_a=True)                                   # pageable host memory
    torch.cuda.synchronize()
    Hd = ops.matmul(p, torch.from_numpy(A).cuda(), None, mask, "bf16", col_scale=csd, symmetric=True,
                    sparse_a=True).cpu()
    assert torch.equal(H, Hd)
    # host rows with padding (lda > n) and an output with ldc > l
    l = 200
    B = rng.standard_normal((n, l)).astype(np.float32)
    Ap = np.zeros((m, n + 5), np.float32)
    Ap[:, :n] = A
    Cp = torch.full((m, l + 3), -1.0).pin_memory()
    ops.matmul_host(p, torch.from_numpy(Ap)[:, :n], torch.from_numpy(B), mask, "bf16", C=Cp[:, :l])
    torch.cuda.synchronize()
    Cd = ops.matmul(p, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), mask, "bf16").cpu()
    assert torch.equal(Cp[:, :l], Cd)
    assert (Cp[:, l:] == -1.0).all()
