"""The CPU reference of Sec. 5.2's interior-point LP (oracle/lp.py), pinned to an
independent LP solver: after 100 barrier iterations (tau doubling every 10) the
objective is within the barrier's duality gap n / tau of the LP optimum."""
import numpy as np
import pytest

from oracle import lp


def test_barrier_reaches_the_lp_optimum():
    opt = pytest.importorskip("scipy.optimize")
    n, m = 400, 20
    A, b, c = lp.synthetic_lp(n, m, 3)
    x, hist = lp.barrier_lp(A, b, c, np.zeros(m), iters=100, tau0=1.0, every=10)
    res = opt.linprog(c, A_ub=A, b_ub=b, bounds=[(None, None)] * m, method="highs")
    assert res.status == 0
    tau_last = 2.0 ** 9
    assert np.all(b - A @ x > 0)                          # strictly feasible throughout
    assert hist[-1] - res.fun >= -1e-9                     # never below the optimum
    assert hist[-1] - res.fun <= n / tau_last + 1e-6      # duality gap of the barrier


def test_barrier_objective_decreases_per_centring_stage():
    n, m = 300, 15
    A, b, c = lp.synthetic_lp(n, m, 4)
    _, hist = lp.barrier_lp(A, b, c, np.zeros(m), iters=60, every=10)
    ends = [hist[k] for k in range(9, 60, 10)]
    assert all(ends[i + 1] <= ends[i] + 1e-9 for i in range(len(ends) - 1))
