"""GPU parity of the differentiable product: layout utilities, the plain
tensor-core GEMM, and OverSketchMatmul's forward and backward against the FP64
oracle's gradient (whose formula is pinned by finite differences in
test_oracle.py)."""
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


@pytest.fixture(scope="module")
def ag(ops):
    from paper_1811_02653_gb300 import autograd
    return autograd


def test_select_transpose_and_cast(ops):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((70, 5 * 64)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Y = ops.select_transpose(Xd, "f32", block_mask=0b10110, b=64).cpu().numpy()
    cols = oracle.selected_columns(0b10110, 5, 64)
    assert np.array_equal(Y, X[:, cols].T)
    Yt = ops.select_transpose(Xd).cpu().numpy()
    assert np.array_equal(Yt, X.T)
    Yb = ops.cast(Xd, "bf16").float().cpu().numpy()
    assert np.array_equal(Yb, oracle.round_bf16(X))
    Ybt = ops.select_transpose(Xd, "bf16").float().cpu().numpy()
    assert np.array_equal(Ybt, oracle.round_bf16(X).T)


@pytest.mark.parametrize("m,n,K", [(64, 64, 64), (300, 200, 512), (1000, 130, 4096), (70, 90, 96)])
def test_gemm_bf16_plain(ops, m, n, K):
    rng = np.random.default_rng(m + K)
    A = torch.from_numpy(rng.standard_normal((m, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    B = torch.from_numpy(rng.standard_normal((n, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    C = ops.gemm_bf16(A, B, alpha=0.5).cpu().numpy()
    A64, B64 = A.float().cpu().numpy().astype(np.float64), B.float().cpu().numpy().astype(np.float64)
    assert oracle.rel_frob(C, 0.5 * A64 @ B64.T) <= 1e-5


def _emulated_gradients(X, G, dC, h, s, b, mask):
    """The oracle's gradient with the GPU path's BF16 operand roundings applied:
    A~ and B~ rounded to BF16 (the forward's sketch outputs) and dC rounded to BF16."""
    P = h.shape[0]
    z = P * b
    k = len(oracle.selected_blocks(mask, P))
    cols = oracle.selected_columns(mask, P, b)
    At = oracle.round_bf16(oracle.sketch_left(X, h, s, b))
    Bt = oracle.round_bf16(oracle.sketch_right(G, h, s, b))
    dCq = oracle.round_bf16(dC)
    T = np.zeros((X.shape[0], z))
    T[:, cols] = dCq @ Bt[cols].T / k
    U = np.zeros((z, G.shape[1]))
    U[cols] = At[:, cols].T @ dCq / k
    return oracle.unsketch_cols(T, h, s, b, mask, 1.0), oracle.unsketch_rows(U, h, s, b, mask, 1.0)


@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_small_parity(ops, ag, recompute):
    m, n, l, b, N, e, mask = 64, 512, 64, 64, 4, 1, 0b11011
    rng = np.random.default_rng(5)
    X = (rng.standard_normal((m, n)) * 0.02).astype(np.float32)
    G = (rng.standard_normal((n, l)) * 0.02).astype(np.float32)
    dC = rng.standard_normal((m, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 0)
    h, s = oracle.hash_tables(n, b, N, e, 0)
    Xd = torch.from_numpy(X).cuda().requires_grad_(True)
    Gd = torch.from_numpy(G).cuda().requires_grad_(True)
    C = ag.oversketch_matmul(Xd, Gd, p, mask, recompute)
    C.backward(torch.from_numpy(dC).cuda())
    dX_ref, dG_ref = _emulated_gradients(X, G, dC, h, s, b, mask)
    assert oracle.rel_frob(Xd.grad.cpu().numpy(), dX_ref) <= 1e-4
    assert oracle.rel_frob(Gd.grad.cpu().numpy(), dG_ref) <= 1e-4
    # against the exact (unrounded) gradient: BF16 operand rounding only
    dX_ex, dG_ex = oracle.gradients(X, G, dC, h, s, b, mask)
    assert oracle.rel_frob(Xd.grad.cpu().numpy(), dX_ex) <= 2e-2
    assert oracle.rel_frob(Gd.grad.cpu().numpy(), dG_ex) <= 2e-2


@pytest.mark.parametrize("m,n,l,b,N,e,mask,sides", [
    (296, 3000, 200, 128, 4, 1, 0b10111, "both"),   # MN-major: ragged tile pairs, dC rows padded to 64
    (520, 4096, 328, 256, 3, 2, 0b10101, "both"),   # MN-major: blocks of two tile columns, two dropped
    (264, 4096, 304, 256, 4, 1, 0b01111, "dg"),     # MN-major dG alone (dC cast for it only)
    (8, 640, 8, 128, 2, 1, 0b010, "both"),          # MN-major, tiny: one kept block of 128, tiles mostly past the extents
    (300, 3000, 200, 128, 4, 1, 0b10111, "both"),   # m not a multiple of 8: K-major copies
    (129, 2000, 77, 64, 3, 2, 0b10101, "both"),     # b = 64: K-major copies
    (64, 512, 64, 32, 4, 1, 0b11011, "both"),       # b = 32: K-major copies
])
def test_matmul_backward_parity(ops, m, n, l, b, N, e, mask, sides):
    # oversketch_matmul_backward from the forward's BF16 sketches: with b a multiple
    # of 128 and m, l multiples of 8 the tensor cores read B~^T, A~ and dC MN-major
    # as stored; against the oracle's gradients with the same BF16 roundings
    rng = np.random.default_rng(m + l + b)
    X = (rng.standard_normal((m, n)) * 0.02).astype(np.float32)
    G = (rng.standard_normal((n, l)) * 0.02).astype(np.float32)
    dC = rng.standard_normal((m, l)).astype(np.float32)
    p = ops.plan(n, b, N, e, 2)
    h, s = oracle.hash_tables(n, b, N, e, 2)
    At, _ = ops.sketch_left(p, torch.from_numpy(X).cuda(), "bf16", block_mask=mask)
    BtT, _ = ops.sketch_right(p, torch.from_numpy(G).cuda(), "bf16", block_mask=mask)
    dX, dG = ops.matmul_backward(p, At, BtT, torch.from_numpy(dC).cuda(), mask,
                                 need_dx=sides == "both", need_dg=True)
    dX_ref, dG_ref = _emulated_gradients(X, G, dC, h, s, b, mask)
    if sides == "both":
        assert oracle.rel_frob(dX.cpu().numpy(), dX_ref) <= 1e-4
    assert oracle.rel_frob(dG.cpu().numpy(), dG_ref) <= 1e-4


def test_autograd_recompute_is_bitwise_equal(ops, ag):
    m, n, l, b, N, e, mask = 128, 4096, 96, 256, 4, 1, 0b10111
    rng = np.random.default_rng(6)
    X = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
    G = torch.from_numpy(rng.standard_normal((n, l)).astype(np.float32)).cuda()
    dC = torch.from_numpy(rng.standard_normal((m, l)).astype(np.float32)).cuda()
    p = ops.plan(n, b, N, e, 1)
    grads = []
    for rc in (False, True):
        Xd, Gd = X.clone().requires_grad_(True), G.clone().requires_grad_(True)
        ag.oversketch_matmul(Xd, Gd, p, mask, rc).backward(dC)
        grads.append((Xd.grad, Gd.grad))
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])


def test_autograd_workload_sampled(ops, ag):
    # X 4096 x 65536 and G 65536 x 4096 in BF16 with N(0, 0.02^2) entries; b=2048,
    # N=4, e=1, block 2 dropped.  Checked on sampled rows of dX, columns of dG and
    # entries of C, which the oracle computes one by one.
    w = W.AUTOGRAD
    X = torch.from_numpy(w.left()).to(torch.bfloat16).cuda().requires_grad_(True)
    Gt = torch.from_numpy(w.right_cols(range(w.l))).to(torch.bfloat16).cuda()
    G = Gt.t().contiguous().requires_grad_(True)
    del Gt
    dC = torch.from_numpy(w.upstream_grad()).cuda()
    p = ops.plan(w.n, w.b, w.N, w.e, w.hash_seed)
    C = ag.oversketch_matmul(X, G, p, w.mask)
    C.backward(dC)
    torch.cuda.synchronize()
    h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    X64 = X.detach().float().cpu().numpy().astype(np.float64)
    G64 = G.detach().float().cpu().numpy().astype(np.float64)
    dC64 = dC.cpu().numpy().astype(np.float64)
    cols = oracle.selected_columns(w.mask, w.P, w.b)
    k = w.k
    At = oracle.round_bf16(oracle.sketch_left(X64, h, s, w.b))
    Bt = oracle.round_bf16(oracle.sketch_right(G64, h, s, w.b))
    dCq = oracle.round_bf16(dC64)
    rows = [0, 17, 2048, 4095]
    ccols = [0, 33, 1024, 4095]
    # forward entries
    C_ref = oracle.masked_product(At[rows], Bt[:, ccols], w.b, w.mask)
    assert oracle.rel_frob(C.detach()[rows][:, ccols].cpu().numpy(), C_ref) <= 1e-4
    # dX rows
    T = np.zeros((len(rows), w.z))
    T[:, cols] = dCq[rows] @ Bt[cols].T / k
    dX_ref = oracle.unsketch_cols(T, h, s, w.b, w.mask, 1.0)
    dX_gpu = X.grad[rows].float().cpu().numpy()
    assert oracle.rel_frob(dX_gpu, dX_ref) <= 5e-3          # BF16 gradient output
    # dG columns
    U = np.zeros((w.z, len(ccols)))
    U[cols] = At[:, cols].T @ dCq[:, ccols] / k
    dG_ref = oracle.unsketch_rows(U, h, s, w.b, w.mask, 1.0)
    dG_gpu = G.grad[:, ccols].float().cpu().numpy()
    assert oracle.rel_frob(dG_gpu, dG_ref) <= 5e-3
