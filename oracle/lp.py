"""CPU reference of the interior-point LP of Sec. 5.2 -- test infrastructure only.

The LP   minimize c^T x  subject to  A x <= b   (A: n x m, n > m)
is solved by the logarithmic barrier method of Sec. 5.2: Newton's method on
f(x) = tau c^T x - sum_i log(b_i - a_i x), with tau doubled every `every`
iterations, using the exact Hessian A^T diag(1/(b - A x)^2) A and the gradient
tau c + sum_i a_i^T / (b_i - a_i x).  The Newton system uses the symmetric
part of the Hessian, Jacobi-equilibrated; when that is not positive definite (a
sketched Hessian whose blocks keep different sketch blocks need not be) the
smallest shift in 0, 1e-8, 1e-7, ... times the identity that makes it so is
added -- the paper does not say how an indefinite system is treated, this is
the reading both solvers share; a non-finite system, or one that no shift up
to 1e8 repairs, raises NewtonSystemError instead of looping.  The step size eta
comes from a backtracking line search that keeps every slack positive (Armijo condition with parameter
1/4, halving).  Plain FP64 numpy; shares no code with the GPU solver.  The
pinned fact: after the last centring step at barrier weight tau the objective
is within n / tau of the LP optimum (the barrier's duality gap).
"""
from __future__ import annotations

import numpy as np


def barrier_objective(A, b, c, x, tau):
    s = b - A @ x
    if np.any(s <= 0):
        return np.inf
    return tau * float(c @ x) - float(np.sum(np.log(s)))


class NewtonSystemError(ValueError):
    """The Newton system cannot be solved: a non-finite Hessian or gradient, or no
    shift up to MAX_SHIFT makes the equilibrated system positive definite."""


MAX_SHIFT = 1e8
SHIFTS = (0.0,) + tuple(10.0 ** p for p in range(-8, 9))      # 0, 1e-8, ..., 1e8


def newton_direction(H, g):
    """-(H_sym + shift D)^{-1} g with D = diag(H_sym) and the smallest shift of
    0, 1e-8, 1e-7, ..., 1e8 for which the equilibrated system is positive
    definite.  A row whose diagonal entry is not positive is left unscaled (a
    Hessian of Sec. 5.2, sketched or not, has a non-negative diagonal: each
    diagonal entry is a sum of squares).  Raises NewtonSystemError for a
    non-finite H or g, or when no shift up to 1e8 factorises."""
    H = np.asarray(H, np.float64)
    g = np.asarray(g, np.float64)
    if not (np.all(np.isfinite(H)) and np.all(np.isfinite(g))):
        raise NewtonSystemError("non-finite Hessian or gradient")
    Hs = 0.5 * (H + H.T)
    dH = np.diag(Hs)
    d = np.where(dH > 0.0, 1.0 / np.sqrt(np.where(dH > 0.0, dH, 1.0)), 1.0)
    He = Hs * d[:, None] * d[None, :]
    for shift in SHIFTS:
        try:
            L = np.linalg.cholesky(He + shift * np.eye(len(d)))
            break
        except np.linalg.LinAlgError:
            continue
    else:
        raise NewtonSystemError("no shift up to 1e8 makes the Newton system positive definite")
    y = np.linalg.solve(L.T, np.linalg.solve(L, g * d))
    return -(y * d)


def barrier_lp(A, b, c, x0, iters=100, tau0=1.0, every=10, hessian=None):
    """Newton iterations of the barrier method; returns (x, objective c^T x per
    iteration).  `hessian(x, s, t)` may replace the exact Hessian (iteration t,
    slacks s); the default is A^T diag(1/s^2) A."""
    A = np.asarray(A, np.float64)
    b = np.asarray(b, np.float64)
    c = np.asarray(c, np.float64)
    x = np.asarray(x0, np.float64).copy()
    hist = []
    for t in range(iters):
        tau = tau0 * 2.0 ** (t // every)
        s = b - A @ x
        g = tau * c + A.T @ (1.0 / s)
        H = hessian(x, s, t) if hessian is not None else (A.T * (1.0 / s ** 2)) @ A
        dx = newton_direction(H, g)
        f0 = barrier_objective(A, b, c, x, tau)
        eta, slope = 1.0, float(g @ dx)
        while eta > 1e-12:
            xn = x + eta * dx
            fn = barrier_objective(A, b, c, xn, tau)
            if np.isfinite(fn) and fn <= f0 + 0.25 * eta * slope:
                break
            eta *= 0.5
        if eta > 1e-12:
            x = x + eta * dx
        hist.append(float(c @ x))
    return x, hist

