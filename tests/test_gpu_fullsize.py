"""GPU parity at the full sizes of the interior-point and batched workloads,
on sampled outputs that the FP64 oracle computes one by one.

* Interior-point normal matrix H = A D A^T (Sec. 5.2): A 4096 x 1048576 with
  1% nonzeros stored dense, D log-uniform in [1e-6, 1e6]; b=4096, N=6, e=1,
  block 3 dropped; BF16 symmetric product with sqrt(D) folded into the sketch.
* Uneven batch: 256 products, m, l ~ U[256, 4096], n log-uniform in
  [8192, 131072] (182 GB of FP32 inputs on the device), b = n/32, N=4, e=1,
  product p drops block p mod 5; one CUDA graph, BF16 grouped GEMM.
"""
import numpy as np
import pytest

import oracle
from helpers import gpu_lib

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


def _free_cache():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_hessian_workload_sampled(ops):
    from paper_1811_02653_gb300 import workloads as W
    w = W.HESSIAN
    _free_cache()
    offs, idx, val = w.left_sparse(range(w.m))
    A = torch.zeros((w.m, w.n), dtype=torch.float32, device="cuda")
    rows_of = torch.repeat_interleave(torch.arange(w.m, device="cuda"),
                                      torch.from_numpy(np.diff(offs)).cuda())
    A[rows_of, torch.from_numpy(idx).cuda()] = torch.from_numpy(val).cuda()
    del rows_of
    cs = w.col_scale()
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    csd = torch.from_numpy(cs).cuda()
    # the sparse-row sketch (what the bench times) and the dense gather path
    H = ops.matmul(p, A, None, w.mask, "bf16", col_scale=csd, symmetric=True, sparse_a=True)
    H_dense = ops.matmul(p, A, None, w.mask, "bf16", col_scale=csd, symmetric=True)
    torch.cuda.synchronize()
    assert ops.device_status() == 0
    rows = [0, 1, 777, 2048, 3333, 4095]
    A_r = A[rows].cpu().numpy().astype(np.float64)
    del A
    _free_cache()
    # the sampled rows are those the generator draws
    ref_rows = w.left_rows(rows).astype(np.float64)
    assert np.array_equal(A_r, ref_rows)
    h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    At = oracle.round_bf16(oracle.sketch_left(A_r, h, s, w.b, cs.astype(np.float64)))
    H_ref = oracle.masked_product(At, At.T, w.b, w.mask)
    H_gpu = H[rows][:, rows].cpu().numpy().astype(np.float64)
    assert oracle.rel_frob(H_gpu, H_ref) <= 1e-4
    assert oracle.rel_frob(H_dense[rows][:, rows].cpu().numpy().astype(np.float64), H_ref) <= 1e-4
    # symmetric by construction (B~ = A~)
    assert np.array_equal(H_gpu, H_gpu.T)
    # the sketched H against the exact A D A^T on the sample (reported by the bench, loose here)
    H_exact = (A_r * (cs.astype(np.float64) ** 2)) @ A_r.T
    assert oracle.rel_frob(H_gpu, H_exact) < 0.5


def test_batched_workload_sampled(ops):
    from paper_1811_02653_gb300 import workloads as W
    shapes = W.batched_shapes()
    _free_cache()
    dev = []
    for q, (m, n, l) in enumerate(shapes):
        A, B = W.batched_device_inputs(shapes, q, "cuda")
        C = torch.full((m, l), float("nan"), dtype=torch.float32, device="cuda")
        b = n // 32
        mask = 0b11111 & ~(1 << (q % 5))
        dev.append((A, B, C, ops.plan(n, b, 4, 1, 0), mask))
    batch = ops.Batch(dev)
    info = batch.info()
    assert info["count"] == 256
    batch.run()
    torch.cuda.synchronize()
    assert ops.device_status() == 0
    order = sorted(range(256), key=lambda q: shapes[q][1])
    sample = sorted({0, 1, 100, 255, order[0], order[-1], max(range(256), key=lambda q: shapes[q][0])})
    for q in sample:
        A, B, C, p, mask = dev[q]
        m, n, l = shapes[q]
        rows = sorted({0, m // 2, m - 1})
        cols = sorted({0, l // 3, l - 1})
        A_r = A[rows].cpu().numpy().astype(np.float64)
        B_c = B[:, cols].cpu().numpy().astype(np.float64)
        h, s = oracle.hash_tables(n, n // 32, 4, 1, 0)
        At = oracle.round_bf16(oracle.sketch_left(A_r, h, s, n // 32))
        Bt = oracle.round_bf16(oracle.sketch_right(B_c, h, s, n // 32))
        ref = oracle.masked_product(At, Bt, n // 32, mask)
        got = C[rows][:, cols].cpu().numpy().astype(np.float64)
        assert oracle.rel_frob(got, ref) <= 1e-4, q
    # every output was written (no NaN left from the fill)
    assert all(not torch.isnan(C).any().item() for (_, _, C, _, _) in dev)
    batch.close()
    del dev
    _free_cache()
