"""oversketch_sketch_size (host-only, no GPU): the number of blocks for an
(eps, theta)-accurate product (Thm. 4.1: d = 2/(eps*theta)) and the extra
blocks for a straggler fraction, checked against the definitions and against
the oracle's exact expected error of the sketched product."""
import math

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def ops():
    from paper_1811_02653_gb300 import build, ops
    build.build()
    return ops


@pytest.mark.parametrize("eps,theta,b,p,r", [(0.01, 0.1, 256, 0.2, 1), (0.05, 0.5, 64, 0.0, 1),
                                             (0.02, 0.25, 128, 0.05, 2), (0.5, 0.9, 1, 0.3, 1)])
def test_size_is_the_smallest_that_meets_the_theorem(ops, eps, theta, b, p, r):
    N, e = ops.sketch_size(eps, theta, b, p, r)
    d = 2.0 / (eps * theta)
    assert N * b >= r * d - 1e-6 and (N - 1) * b < r * d        # enough columns, and no more blocks than needed
    assert e >= p * (N + e) - 1e-9                                 # dropping a fraction p leaves N blocks
    assert e == 0 or (e - 1) < p * (N + e - 1)                     # the smallest such e


def test_size_meets_the_bound_on_the_exact_expected_error(ops):
    # Markov's step of Thm. 4.1: E||AB - C||^2 <= eps*theta ||A||^2 ||B||^2 gives the
    # (eps, theta) guarantee; the oracle's closed form of E||AB - C||^2 (Lemma countEV)
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 300))
    B = rng.standard_normal((300, 30))
    for eps, theta, b in [(0.2, 0.5, 8), (0.1, 0.5, 16), (0.05, 0.8, 10)]:
        N, e = ops.sketch_size(eps, theta, b, 0.1, 1)
        expected = oracle.expected_sq_error(A, B, N, b)             # N kept blocks of width b
        bound = eps * theta * np.sum(A * A) * np.sum(B * B)
        assert expected <= bound


def test_size_rejects_bad_arguments(ops):
    for args in [(0.0, 0.1, 8, 0.0, 1), (0.1, 1.0, 8, 0.0, 1), (0.1, 0.1, 0, 0.0, 1),
                 (0.1, 0.1, 8, 1.0, 1), (0.1, 0.1, 8, 0.0, 0)]:
        with pytest.raises(ops.OverSketchError, match="INVALID_ARG"):
            ops.sketch_size(*args)
    with pytest.raises(ops.OverSketchError, match="UNSUPPORTED"):
        ops.sketch_size(1e-4, 0.01, 16, 0.0, 1)                   # 2/(eps theta) / b blocks > 64
