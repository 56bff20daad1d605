"""Sec. 5.1's accuracy experiment on the GPU path: A(x, y) = x + y, B = A^T,
n = 60b, m = l = 10b, sketch dimension z = 30b, e sketch blocks ignored per b x b
block of C (Alg. 3 per block).  Over ten sketch seeds the mean squared error
||AB - C||_F^2 matches the oracle's exact expectation (Appendix B's closed form,
factored for this rank-2 matrix), and sampled entries of C match the oracle's
per-block product of the same sketches."""
import numpy as np
import pytest

import oracle
from helpers import gpu_lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

B_W, P = 256, 30
M_, N_ = 10 * B_W, 60 * B_W


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


@pytest.fixture(scope="module")
def operands():
    from paper_1811_02653_gb300 import workloads
    return workloads.sec51_device(M_, N_, "cuda")


def _product(ops, A, B, seed, e):
    from paper_1811_02653_gb300 import workloads
    p = ops.plan(N_, B_W, P - 4, 4, seed)
    At, _ = ops.sketch_left(p, A, "bf16")
    BtT, _ = ops.sketch_right(p, B, "bf16")
    nb = M_ // B_W
    masks = workloads.straggler_block_masks(P, e, nb, nb, seed, 0)
    C = ops.gemm_masked_blocks(p, At, BtT, torch.from_numpy(masks).cuda(), B_W, B_W)
    return C, masks


@pytest.mark.parametrize("e", [0, 4])
def test_sec51_mean_error_matches_the_expectation(ops, operands, e):
    from paper_1811_02653_gb300 import workloads
    A, B, AB = operands
    U, V = workloads.sec51_factors(M_, N_)
    expect = oracle.expected_sq_error_factored(U, V, V, U, P - e, B_W)
    sq = []
    for seed in range(10):
        C, _ = _product(ops, A, B, seed, e)
        sq.append(float(ops.frob(C, AB)[0]))
    ratio = np.mean(sq) / expect
    assert 0.35 < ratio < 2.0, ratio


def test_sec51_sampled_entries_match_the_oracle(ops, operands):
    A, B, _ = operands
    C, masks = _product(ops, A, B, 3, 4)
    rows, cols = [0, 1000, M_ - 1], [0, 777, M_ - 1]
    h, s = oracle.hash_tables(N_, B_W, P - 4, 4, 3)
    At_r = oracle.round_bf16(oracle.sketch_left(A[rows].cpu().numpy().astype(np.float64), h, s, B_W))
    Bt_c = oracle.round_bf16(oracle.sketch_right(B[:, cols].cpu().numpy().astype(np.float64), h, s, B_W))
    ref = np.empty((3, 3))
    for a, r in enumerate(rows):
        for c_, c in enumerate(cols):
            mk = int(masks[r // B_W, c // B_W])
            ref[a, c_] = oracle.masked_product(At_r[a:a + 1], Bt_c[:, c_:c_ + 1], B_W, mk)[0, 0]
    got = C[rows][:, cols].cpu().numpy().astype(np.float64)
    assert oracle.rel_frob(got, ref) <= 1e-4
