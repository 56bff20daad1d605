"""The left sketch without allocation, checked against the regular entry point.

oversketch_sketch_left_noalloc serves callers that cannot allocate device
memory where they sketch (inside a CUDA graph capture, under another
allocator's budget, in loops that must not call cudaMalloc): its packing
workspace is the library's fixed 32 MiB scratch array.  This file is
collected last so that a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import assert_fp32_within, gpu_lib, sketch_bounds_left

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


def test_noalloc_matches_sketch_left_two_calls(ops):
    m, n, b, N, e = 200, 5000, 128, 3, 1          # packed operand: 256 x 5000 x 4 B = 5.1 MB
    rng = np.random.default_rng(31)
    p = ops.plan(n, b, N, e, 9)
    h, s = oracle.hash_tables(n, b, N, e, 9)
    for call in range(2):                          # two calls in a row share the scratch array
        A = rng.standard_normal((m, n)).astype(np.float32)
        Ad = torch.from_numpy(A).cuda()
        ref, _ = ops.sketch_left(p, Ad, "f32")
        out = torch.full_like(ref, float("nan"))
        ops.sketch_left_noalloc(p, Ad, out, "f32")
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # same kernels, same order: equal to the regular entry point, and both
        # within the FP32 rounding bound of the oracle
        assert_fp32_within(got, ref.cpu().numpy().astype(np.float64), np.zeros(got.shape))
        r64, bound = sketch_bounds_left(A, h, s, b)
        assert_fp32_within(got, r64, bound)


def test_noalloc_bf16_output_and_block_mask(ops):
    m, n, b, N, e = 96, 3000, 256, 4, 1
    rng = np.random.default_rng(32)
    p = ops.plan(n, b, N, e, 2)
    Ad = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
    ref, _ = ops.sketch_left(p, Ad, "bf16", block_mask=0b10110)
    out = torch.zeros_like(ref)
    ops.sketch_left_noalloc(p, Ad, out, "bf16", block_mask=0b10110)
    cols = oracle.selected_columns(0b10110, N + e, b)
    assert torch.equal(out[:, cols], ref[:, cols])


def test_noalloc_rejects_operands_beyond_the_scratch(ops):
    n, b = 65536, 1024
    p = ops.plan(n, b, 2, 1, 0)
    m = 256                                        # 256 x 65536 x 4 B = 64 MiB > 32 MiB
    A = torch.zeros((m, n), device="cuda")
    out = torch.empty((m, p.z), device="cuda")
    with pytest.raises(ops.OverSketchError, match="WORKSPACE"):
        ops.sketch_left_noalloc(p, A, out, "f32")
    # through the raw C ABI as well: the status comes back before any launch
    L = ops.load_library()
    st = L.oversketch_sketch_left_noalloc(p.handle, ctypes.c_void_p(A.data_ptr()), 0, m, n,
                                          ctypes.c_void_p(out.data_ptr()), 0, p.z, None, None, 0,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 8


def test_noalloc_bf16_input_with_col_scale(ops):
    # BF16 operand and a column scale (A diag(s) S) through the scratch array,
    # within the FP32 bound of the oracle and equal to the regular entry point
    m, n, b, N, e = 72, 2500, 128, 3, 1
    rng = np.random.default_rng(33)
    p = ops.plan(n, b, N, e, 4)
    h, s = oracle.hash_tables(n, b, N, e, 4)
    Ab = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).to(torch.bfloat16).cuda()
    cs = rng.uniform(0.5, 2.0, n).astype(np.float32)
    csd = torch.from_numpy(cs).cuda()
    ref, _ = ops.sketch_left(p, Ab, "f32", col_scale=csd)
    out = torch.full_like(ref, float("nan"))
    ops.sketch_left_noalloc(p, Ab, out, "f32", col_scale=csd)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    r64, bound = sketch_bounds_left(Ab.float().cpu().numpy(), h, s, b, col_scale=cs)
    assert_fp32_within(out.cpu().numpy(), r64, bound)


def test_noalloc_inside_a_captured_graph(ops):
    # the reason for the entry point: it can be recorded into a CUDA graph, where
    # the caller could not allocate a workspace.  One warm call first (it looks up
    # the scratch array's address), then capture, then replay on new contents of A.
    m, n, b, N, e = 128, 4096, 256, 4, 1
    rng = np.random.default_rng(34)
    p = ops.plan(n, b, N, e, 6)
    Ad = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
    out = torch.empty((m, p.z), device="cuda", dtype=torch.bfloat16)
    ops.sketch_left_noalloc(p, Ad, out, "bf16")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ops.sketch_left_noalloc(p, Ad, out, "bf16")
    for seed in (35, 36):
        Ad.copy_(torch.from_numpy(np.random.default_rng(seed).standard_normal((m, n)).astype(np.float32)))
        out.zero_()
        g.replay()
        ref, _ = ops.sketch_left(p, Ad, "bf16")
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_empty_output_and_argument_errors(ops):
    # an empty output is OS_OK with NULL pointers; argument errors come back as
    # from oversketch_sketch_left, before the operand size is considered
    n, b = 65536, 1024
    p = ops.plan(n, b, 2, 1, 0)
    L = ops.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.oversketch_sketch_left_noalloc(p.handle, None, 0, 0, n, None, 0, p.z, None, None, 0, stream) == 0
    A = torch.zeros((256, n), device="cuda")
    out = torch.empty((256, p.z), device="cuda")
    a, o = ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(out.data_ptr())
    # lda < n, an unsupported dtype and a mask beyond N+e: the regular entry point's codes
    assert L.oversketch_sketch_left_noalloc(p.handle, a, 0, 256, n - 1, o, 0, p.z, None, None, 0, stream) == 1
    assert L.oversketch_sketch_left_noalloc(p.handle, a, 2, 256, n, o, 0, p.z, None, None, 0, stream) == 3
    assert L.oversketch_sketch_left_noalloc(p.handle, a, 0, 256, n, o, 0, p.z, None, None, 1 << 5, stream) == 2
    assert L.oversketch_sketch_left_noalloc(p.handle, a, 0, 256, n, None, 0, p.z, None, None, 0, stream) == 1
