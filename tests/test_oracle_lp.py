"""The CPU reference of Sec. 5.2's interior-point LP (oracle/lp.py), pinned to an
independent LP solver: after 100 barrier iterations (tau doubling every 10) the
objective is within the barrier's duality gap n / tau of the LP optimum."""
import numpy as np
import pytest

from oracle import lp
from paper_1811_02653_gb300 import workloads


def test_barrier_reaches_the_lp_optimum():
    opt = pytest.importorskip("scipy.optimize")
    n, m = 400, 20
    A, b, c = workloads.lp_instance(n, m, 3)
    x, hist = lp.barrier_lp(A, b, c, np.zeros(m), iters=100, tau0=1.0, every=10)
    res = opt.linprog(c, A_ub=A, b_ub=b, bounds=[(None, None)] * m, method="highs")
    assert res.status == 0
    tau_last = 2.0 ** 9
    assert np.all(b - A @ x > 0)                          # strictly feasible throughout
    assert hist[-1] - res.fun >= -1e-9                     # never below the optimum
    assert hist[-1] - res.fun <= n / tau_last + 1e-6      # duality gap of the barrier


def test_barrier_objective_decreases_per_centring_stage():
    n, m = 300, 15
    A, b, c = workloads.lp_instance(n, m, 4)
    _, hist = lp.barrier_lp(A, b, c, np.zeros(m), iters=60, every=10)
    ends = [hist[k] for k in range(9, 60, 10)]
    assert all(ends[i + 1] <= ends[i] + 1e-9 for i in range(len(ends) - 1))


def _sketched_hessian(A, blk, P, masks_of, cb):
    import oracle
    n = A.shape[0]
    h, sg = oracle.hash_tables(n, blk, P - 1, 1, 0)

    def hess(x, s, t):
        Ask = oracle.sketch_left(A.T, h, sg, blk, col_scale=1.0 / s)
        return oracle.masked_product_blocks(Ask, Ask.T, blk, masks_of(t).tolist(), cb, cb)
    return hess


def test_gram_form_sketched_hessian_tracks_the_exact_newton_path():
    """With one kept set for the whole Hessian the sketched Hessian is the Gram
    matrix (S D^{1/2} A)^T (S D^{1/2} A) / k: positive semidefinite, and with the
    sketch dimension n/2 of Sec. 5.2 the barrier path ends where the exact one does."""
    n, m, blk, P = 2048, 512, 128, 8
    A, b, c = workloads.lp_instance(n, m, 5)
    A = A.astype(np.float64)
    _, exact = lp.barrier_lp(A, b, c, np.zeros(m))
    masks = lambda t: workloads.straggler_block_masks(P, 1, 2, 2, 11, t, shared=True)
    _, sk = lp.barrier_lp(A, b, c, np.zeros(m), hessian=_sketched_hessian(A, blk, P, masks, 256))
    assert abs(sk[-1] - exact[-1]) <= 2e-3 * abs(exact[-1])


def test_per_block_stragglers_break_the_gram_form_and_the_shift_keeps_descent():
    """Independent kept sets per block of the Hessian (Alg. 3 applied per block)
    give a symmetric part that is indefinite at most iterations; the shifted
    Newton system still yields descent steps, so the iterates stay strictly
    feasible and the objective improves from stage to stage."""
    n, m, blk, P = 2048, 512, 128, 8
    A, b, c = workloads.lp_instance(n, m, 5)
    A = A.astype(np.float64)
    masks = lambda t: workloads.straggler_block_masks(P, 1, 2, 2, 11, t)
    hess = _sketched_hessian(A, blk, P, masks, 256)
    t = next(t for t in range(100) if masks(t)[0, 1] != masks(t)[1, 0])
    H = hess(np.zeros(m), b.copy(), t)
    assert np.abs(H - H.T).max() > 1e-3 * np.abs(H).max()
    x, hist = lp.barrier_lp(A, b, c, np.zeros(m), hessian=hess)
    assert np.all(b - A @ x > 0)
    ends = [hist[k] for k in range(9, 100, 10)]
    assert ends[-1] < ends[0] and ends[-1] < ends[4]


def test_straggler_masks():
    m = workloads.straggler_block_masks(20, 1, 5, 5, 3, 0)
    assert m.shape == (5, 5) and all(bin(int(v)).count("1") == 19 for v in m.ravel())
    assert len(set(m.ravel().tolist())) > 1
    s = workloads.straggler_block_masks(20, 2, 5, 5, 3, 0, shared=True)
    assert len(set(s.ravel().tolist())) == 1 and bin(int(s[0, 0])).count("1") == 18
    assert (workloads.straggler_block_masks(20, 1, 5, 5, 3, 0) == m).all()


def test_barrier_follows_the_central_path_of_a_box():
    # min x s.t. 0 <= x <= 1: the barrier tau x - log x - log(1 - x) is minimised at the
    # root of tau x^2 - (tau + 2) x + 1 = 0 in (0, 1); ten Newton steps per tau land on it
    A = np.array([[-1.0], [1.0]])
    b = np.array([0.0, 1.0])
    c = np.array([1.0])
    for stages in (1, 3, 6):
        x, _ = lp.barrier_lp(A, b, c, np.array([0.5]), iters=10 * stages, tau0=1.0, every=10)
        tau = 2.0 ** (stages - 1)
        centre = ((tau + 2) - np.sqrt((tau + 2) ** 2 - 4 * tau)) / (2 * tau)
        assert abs(x[0] - centre) < 1e-9


def test_gpu_solver_newton_system_matches_the_oracle_rule():
    # the GPU solver's Newton system (FP32 Cholesky with the shift search) chooses the
    # same shift as the oracle's FP64 rule and gives the same direction, on the host
    torch = pytest.importorskip("torch")
    from paper_1811_02653_gb300 import lp as glp
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    for lam_min in (0.3, -0.5):                     # positive definite, then indefinite
        H = Q @ np.diag([lam_min, 1.0, 2.0, 3.0, 5.0, 8.0]) @ Q.T
        H = H + 0.01 * rng.standard_normal((6, 6))   # the sketched Hessian is not symmetric
        g = rng.standard_normal(6)
        solver = object.__new__(glp.SketchedBarrierLP)
        solver.m, solver.device, solver._I = 6, torch.device("cpu"), None
        hist = glp.LPHistory()
        d_gpu = solver.newton_direction(torch.tensor(H, dtype=torch.float32), torch.tensor(g), hist).numpy()
        d_ref = lp.newton_direction(H, g)
        assert np.allclose(d_gpu, d_ref, rtol=1e-4, atol=1e-5)
        assert hist.shifts == (1 if lam_min < 0 else 0)


@pytest.mark.parametrize("case", ["nan", "inf", "negative_diagonal", "hopeless"])
def test_newton_system_errors_instead_of_looping(case):
    # both solvers refuse a Newton system they cannot solve, instead of widening the
    # shift forever: a NaN or Inf Hessian, and one no shift up to 1e8 repairs
    # (a diagonal entry of -1e12 stays negative after equilibration-free scaling);
    # a negative diagonal entry alone is left unscaled and repaired by a shift
    torch = pytest.importorskip("torch")
    from paper_1811_02653_gb300 import lp as glp
    rng = np.random.default_rng(3)
    M = rng.standard_normal((5, 5))
    H = M @ M.T + 5 * np.eye(5)
    g = rng.standard_normal(5)
    if case == "nan":
        H[1, 2] = np.nan
    elif case == "inf":
        H[0, 0] = np.inf
    elif case == "negative_diagonal":
        H[3, 3] = -0.5
    else:
        H[2, 2] = -1e12
    solver = object.__new__(glp.SketchedBarrierLP)
    solver.m, solver.device, solver._I = 5, torch.device("cpu"), None
    if case == "negative_diagonal":
        d_ref = lp.newton_direction(H, g)
        assert np.all(np.isfinite(d_ref))
        hist = glp.LPHistory()
        d_gpu = solver.newton_direction(torch.tensor(H, dtype=torch.float32), torch.tensor(g), hist).numpy()
        assert np.all(np.isfinite(d_gpu)) and hist.shifts == 1
        assert np.allclose(d_gpu, d_ref, rtol=1e-3, atol=1e-5)
        return
    with pytest.raises(lp.NewtonSystemError):
        lp.newton_direction(H, g)
    with pytest.raises(glp.NewtonSystemError):
        solver.newton_direction(torch.tensor(H, dtype=torch.float32), torch.tensor(g), glp.LPHistory())
