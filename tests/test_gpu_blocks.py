"""Alg. 3's termination rule per block of C (oversketch_gemm_masked_blocks):
every block of C keeps its own sketch blocks, against the FP64 oracle
(masked_product_blocks) within the FP32 accumulation bound, through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import gpu_lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


def _bf16(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).cuda()
    return t, t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("m,l,b,N,e,bm,bn", [(1000, 700, 256, 4, 1, 256, 256),
                                             (600, 1100, 128, 3, 2, 512, 256),
                                             (2100, 3000, 256, 4, 1, 1024, 1024)])
def test_blocks_parity(ops, m, l, b, N, e, bm, bn):
    rng = np.random.default_rng(m + l)
    P = N + e
    z = P * b
    At, A64 = _bf16(rng.standard_normal((m, z)))
    Bt, B64 = _bf16(rng.standard_normal((l, z)))
    nbr, nbc = (m + bm - 1) // bm, (l + bn - 1) // bn
    masks = np.zeros((nbr, nbc), dtype=np.int64)
    for i in range(nbr):
        for j in range(nbc):
            drop = rng.choice(P, size=e, replace=False)        # e stragglers of this block of C
            masks[i, j] = sum(1 << t for t in range(P) if t not in drop)
    masks[0, 0] = 0b11                                          # fewer blocks returned (graceful degradation)
    if nbr > 1 and nbc > 1:
        masks[1, 1] = 0                                         # nothing returned: a zero block
    p = ops.plan(max(z, 64), b, N, e, 0)
    C = ops.gemm_masked_blocks(p, At, Bt, torch.from_numpy(masks).cuda(), bm, bn).cpu().numpy()
    ref = oracle.masked_product_blocks(A64, B64.T, b, masks.tolist(), bm, bn)
    absref = oracle.masked_product_blocks(np.abs(A64), np.abs(B64).T, b,
                                          [[m_ if m_ else 0 for m_ in row] for row in masks.tolist()], bm, bn)
    bound = 2 * P * b * 2.0 ** -24 * absref + 1e-30
    assert (np.abs(C - ref) <= bound).all()
    if nbr > 1 and nbc > 1:
        assert (C[bm:2 * bm, bn:2 * bn] == 0).all()


def test_blocks_with_one_mask_equal_the_masked_gemm(ops):
    rng = np.random.default_rng(5)
    m, l, b, N, e = 800, 900, 256, 4, 1
    z = (N + e) * b
    At, _ = _bf16(rng.standard_normal((m, z)))
    Bt, _ = _bf16(rng.standard_normal((l, z)))
    p = ops.plan(z, b, N, e, 0)
    mask = 0b11011
    masks = torch.full(((m + 255) // 256, (l + 255) // 256), mask, dtype=torch.int64, device="cuda")
    C1 = ops.gemm_masked_blocks(p, At, Bt, masks, 256, 256)
    C0 = ops.gemm_masked(p, At, Bt, mask)
    assert torch.equal(C0, C1)
    with pytest.raises(ops.OverSketchError, match="UNSUPPORTED"):
        ops.gemm_masked_blocks(p, At, Bt, masks, 128, 256)
