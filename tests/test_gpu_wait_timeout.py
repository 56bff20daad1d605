"""A bounded device wait that runs out, on purpose, and the launch after it.

Every wait of the tensor-core kernels on an mbarrier gives up after a limit,
records OS_ERR_TIMEOUT in the device status word, waits for the copies it did
issue, frees its tensor memory and returns (the straggler that never reports
back becomes an error the host reads, not a hung GPU).  The test hook leaves
one K step of the first tile unloaded with a 20 microsecond limit on that CTA;
nothing faults and the context stays usable, so the next launch on the same
stream must be correct."""
import numpy as np
import pytest

import oracle
from helpers import gpu_lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


def _split_tf32(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    hi = (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    return hi, (x - hi).astype(np.float32)


@pytest.mark.parametrize("skip_kb", [0, 1])
def test_wait_runs_out_then_next_launch_is_correct(ops, skip_kb):
    # one 128 x 128 tile of the 3xTF32 product (one CTA), three kept blocks of 32:
    # K steps 0, 1, 2.  skip 0: no MMA was issued when the wait runs out; skip 1:
    # the MMAs of step 0 are in flight and are drained before TMEM is freed
    m = l = 128
    b, N, e, mask = 32, 3, 1, 0b1011
    z = (N + e) * b
    rng = np.random.default_rng(40 + skip_kb)
    A = rng.standard_normal((m, z)).astype(np.float32)
    B = rng.standard_normal((l, z)).astype(np.float32)
    Abuf = torch.from_numpy(np.stack(_split_tf32(A))).cuda()
    Bbuf = torch.from_numpy(np.stack(_split_tf32(B))).cuda()
    p = ops.plan(z, b, N, e, 0)
    ref = oracle.masked_product(A.astype(np.float64), B.astype(np.float64).T, b, mask)
    assert ops.device_status(reset=True) == 0
    ops.test_wait_timeout(20_000, skip_kb)
    ops.gemm_masked(p, Abuf[0], Bbuf[0], mask, dtype="tf32x2")
    assert ops.device_status(reset=True) == 6           # OS_ERR_TIMEOUT, read on the host
    # the hook was consumed: the next launch on the same stream is whole and correct
    C = ops.gemm_masked(p, Abuf[0], Bbuf[0], mask, dtype="tf32x2").cpu().numpy()
    assert ops.device_status(reset=True) == 0
    assert oracle.rel_frob(C, ref) <= 1e-5


def test_wait_hook_arguments(ops):
    L = ops.load_library()
    assert L.oversketch_test_wait_timeout(0, 0) == 1     # a skip needs a positive limit
    assert L.oversketch_test_wait_timeout(0, -1) == 0    # withdraw (nothing pending)
