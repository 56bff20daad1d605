"""Sec. 5.2's interior-point LP with the OverSketch Hessian on the GPU
(paper_1811_02653_gb300.lp): the sketched Hessian at an iterate against the FP64
oracle's sketch and per-block product, and the whole barrier method against the
oracle's exact-Hessian barrier method (oracle/lp.py) on the same LP."""
import numpy as np
import pytest

import oracle
from oracle import lp as olp
from helpers import gpu_lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the paper's proportions (n = 8 m, sketch dimension z = n / 2) at a size the
# oracle finishes in seconds: n = 4096 constraints, m = 512 variables, P = 8
# sketch blocks of width 256, Hessian blocks of 256 x 256 (2 x 2 of them)
NC, MV, BLK, P = 4096, 512, 256, 8


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


@pytest.fixture(scope="module")
def problem():
    from paper_1811_02653_gb300 import workloads
    return workloads.lp_instance(NC, MV, 7)


@pytest.fixture(scope="module")
def exact_run(problem):
    A, b, c = problem
    return olp.barrier_lp(A.astype(np.float64), b, c, np.zeros(MV))


def test_lp_hessian_parity(ops, problem, exact_run):
    from paper_1811_02653_gb300 import lp, workloads
    A, b, c = problem
    A64 = A.astype(np.float64)
    x = exact_run[0]                                      # slacks spanning orders of magnitude
    solver = lp.SketchedBarrierLP(A, b, c, blk=BLK, N=P - 1, e=1, seed=0)
    s = torch.from_numpy(b - A64 @ x).cuda()
    masks = workloads.straggler_block_masks(P, 1, 2, 2, 11, 0)
    masks[0, 1] = 0b1                                     # one block returned
    H = solver.hessian(s, masks).cpu().numpy().astype(np.float64)
    # the sketch: A^T diag(1/s) S with the scale the kernel reads (FP32), BF16 output
    d = (1.0 / s).float().cpu().numpy().astype(np.float64)
    h, sg = oracle.hash_tables(NC, BLK, P - 1, 1, 0)
    ref = oracle.sketch_left(A64.T, h, sg, BLK, col_scale=d)
    absref = oracle.sketch_left(np.abs(A64.T), h, np.ones_like(sg), BLK, col_scale=d)
    Ask = solver.Ask.float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Ask - ref) <= 2.0 ** -8 * np.abs(ref) + 64 * 2.0 ** -24 * absref + 1e-30)
    # the per-block product of that sketch, FP32 accumulation bound
    refH = oracle.masked_product_blocks(Ask, Ask.T, BLK, masks.tolist(), 256, 256)
    absH = oracle.masked_product_blocks(np.abs(Ask), np.abs(Ask).T, BLK, masks.tolist(), 256, 256)
    assert np.all(np.abs(H - refH) <= 2 * P * BLK * 2.0 ** -24 * absH + 1e-30)
    # and the whole sketched Hessian against the exact one: the sketch's own error
    exact = (A64.T * (1.0 / (b - A64 @ x)) ** 2) @ A64
    assert oracle.rel_frob(0.5 * (H + H.T), exact) < 0.5


def _gap(f, f_ref):
    return abs(f - f_ref) / abs(f_ref)


def test_lp_sketched_newton_matches_exact_newton(ops, problem, exact_run):
    """All P sketch blocks kept, and one straggler set shared by the whole Hessian:
    the sketched Hessian keeps its Gram form and the barrier path ends where the
    exact-Hessian path of the oracle does."""
    from paper_1811_02653_gb300 import lp, workloads
    A, b, c = problem
    f_exact = exact_run[1][-1]
    solver = lp.SketchedBarrierLP(A, b, c, blk=BLK, N=P - 1, e=1, seed=0)
    x0, h0 = solver.solve()
    x1, h1 = solver.solve(block_masks=lambda t: workloads.straggler_block_masks(P, 1, 2, 2, 11, t, shared=True))
    for x, h in ((x0, h0), (x1, h1)):
        xs = x.cpu().numpy()
        assert np.all(b - A.astype(np.float64) @ xs > 0)
        assert _gap(h.objective[-1], f_exact) <= 2e-3
        assert h.shifts <= 3                              # FP32 factorisation near the end


def test_lp_per_block_stragglers(ops, problem, exact_run):
    """e = 1 straggler per block of the Hessian, independent per block: the
    shifted Newton system keeps the iterates strictly feasible and improving."""
    from paper_1811_02653_gb300 import lp, workloads
    A, b, c = problem
    solver = lp.SketchedBarrierLP(A, b, c, blk=BLK, N=P - 1, e=1, seed=0)
    x, h = solver.solve(block_masks=lambda t: workloads.straggler_block_masks(P, 1, 2, 2, 11, t))
    assert np.all(b - A.astype(np.float64) @ x.cpu().numpy() > 0)
    ends = [h.objective[k] for k in range(9, 100, 10)]
    assert ends[-1] < ends[0] and ends[-1] < ends[4]
    assert _gap(h.objective[-1], exact_run[1][-1]) < 0.3


def test_lp_exact_bf16_hessian(ops, problem, exact_run):
    """The unsketched BF16 Hessian (the comparison arm of the LP benchmark)."""
    from paper_1811_02653_gb300 import lp
    A, b, c = problem
    solver = lp.SketchedBarrierLP(A, b, c, blk=BLK, N=P - 1, e=1, seed=0, exact=True)
    _, h = solver.solve()
    assert _gap(h.objective[-1], exact_run[1][-1]) <= 2e-3
