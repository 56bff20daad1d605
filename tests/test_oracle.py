"""Pins for the FP64 oracle (CPU only).

Each test ties the oracle to something other than itself: a worked example
printed in the paper, a published test vector of the hash, a closed form
from the paper's appendix, an exact special case, an invariant, or brute
force on tiny inputs.  A plausible mistake in the oracle (a dropped block, a
1/N instead of 1/k scale, a wrong sign or bucket, a transposed operand)
fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- hash ----

def test_splitmix64_published_vector():
    # First four outputs of splitmix64 seeded with 0, as produced by the
    # public-domain reference splitmix64.c (Vigna); the hash of every block
    # key and every index is an output of this generator.
    assert oracle.splitmix64_stream(0, 4) == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_hash_is_splitmix_stream():
    # key_j is output j+1 of splitmix64(seed); w(j, i) is output i+1 of
    # splitmix64(key_j); bucket = multiply-shift of w's high half, sign = w's low bit.
    n, b, N, e, seed = 37, 13, 3, 2, 12345
    h, s = oracle.hash_tables(n, b, N, e, seed)
    keys = oracle.splitmix64_stream(seed, N + e)
    for j in range(N + e):
        ws = oracle.splitmix64_stream(keys[j], n)
        for i in range(n):
            assert h[j, i] == ((ws[i] >> 32) * b) >> 32
            assert s[j, i] == (-1 if ws[i] & 1 else 1)


def test_hash_uniform_buckets_and_balanced_signs():
    # Alg. 4 steps 1-2: sign -1 w.p. 1/2, bucket uniform on b values.
    n, b, N, e = 200_000, 64, 3, 1
    h, s = oracle.hash_tables(n, b, N, e, 7)
    for j in range(N + e):
        cnt = np.bincount(h[j], minlength=b).astype(np.float64)
        exp = n / b
        chi2 = ((cnt - exp) ** 2 / exp).sum()
        # chi-square with 63 dof: mean 63, sd ~11.2; 6 sd bound
        assert chi2 < 63 + 6 * 11.3
        frac_neg = (s[j] < 0).mean()
        assert abs(frac_neg - 0.5) < 6 * 0.5 / np.sqrt(n)
    # blocks are independent: bucket collisions across blocks at rate 1/b,
    # sign agreement at rate 1/2
    for j in range(1, N + e):
        same = (h[0] == h[j]).mean()
        assert abs(same - 1 / b) < 6 * np.sqrt((1 / b) * (1 - 1 / b) / n)
        agree = (s[0] == s[j]).mean()
        assert abs(agree - 0.5) < 6 * 0.5 / np.sqrt(n)


def test_hash_rejects_bad_plans():
    with pytest.raises(ValueError):
        oracle.hash_tables(10, 4, 60, 5, 0)      # N + e > 64
    with pytest.raises(ValueError):
        oracle.hash_tables(0, 4, 2, 1, 0)


# ----------------------------------------------------- Eq. 2 example ----

def _eq2():
    rows = [list(map(float, ln.split())) for ln in open(os.path.join(GOLDEN, "eq2_count_sketch.txt"))
            if ln.strip() and not ln.startswith("#")]
    return np.array(rows)          # S_c^T, 3 x 9


def test_eq2_tables_and_sketch_of_identity():
    ScT = _eq2()
    h, s = oracle.tables_from_sketch_matrix(ScT.T)
    # text after Eq. 2 (1-based): columns 4,5,7 -> 1; 1,2,6 -> 2; 3,8,9 -> 3
    assert [int(x) + 1 for x in h[0]] == [2, 2, 3, 1, 1, 2, 1, 3, 3]
    assert np.array_equal(oracle.sketch_matrix(h, s, 3), ScT.T)
    # sketching the identity returns S_c itself
    At = oracle.sketch_left(np.eye(9), h, s, 3)
    assert np.array_equal(At, ScT.T)


def test_eq2_column_sums():
    # "columns with the same mapped value are summed (after possibly
    # multiplying with -1)": bucket sums read off the printed matrix.
    ScT = _eq2()
    h, s = oracle.tables_from_sketch_matrix(ScT.T)
    A = _rng(1).standard_normal((4, 9))
    At = oracle.sketch_left(A, h, s, 3)
    c = A.T  # c[k] = column k+1 of A (1-based as in the paper)
    assert np.allclose(At[:, 0], c[3] - c[4] - c[6], rtol=0, atol=1e-15)
    assert np.allclose(At[:, 1], c[0] - c[1] + c[5], rtol=0, atol=1e-15)
    assert np.allclose(At[:, 2], c[2] - c[7] - c[8], rtol=0, atol=1e-15)
    # right sketch of A^T is the transpose
    Bt = oracle.sketch_right(A.T, h, s, 3)
    assert np.allclose(Bt, At.T, rtol=0, atol=1e-15)


# ------------------------------------------------- implicit vs explicit ----

@pytest.mark.parametrize("m,n,l,b,N,e,seed", [(7, 50, 5, 8, 3, 1, 3), (16, 300, 9, 32, 4, 2, 11),
                                             (3, 64, 4, 1, 2, 0, 5), (5, 20, 6, 64, 2, 1, 9)])
def test_implicit_equals_explicit(m, n, l, b, N, e, seed):
    rng = _rng(seed)
    A = rng.standard_normal((m, n))
    B = rng.standard_normal((n, l))
    h, s = oracle.hash_tables(n, b, N, e, seed)
    S = oracle.sketch_matrix(h, s, b)
    assert np.allclose(oracle.sketch_left(A, h, s, b), A @ S, rtol=1e-13, atol=1e-13)
    assert np.allclose(oracle.sketch_right(B, h, s, b), S.T @ B, rtol=1e-13, atol=1e-13)
    cs = np.exp(rng.standard_normal(n))
    assert np.allclose(oracle.sketch_left(A, h, s, b, cs), (A * cs) @ S, rtol=1e-13, atol=1e-13)
    mask = (1 << (N + e)) - 1 - (1 << (N + e - 1))
    C1 = oracle.oversketch(A, B, h, s, b, mask)
    C2 = oracle.oversketch_explicit(A, B, S, b, mask)
    assert oracle.rel_frob(C1, C2) < 1e-13


def test_brute_force_nxn():
    # A (S_sel S_sel^T / k) B from the n x n matrix, tiny n
    rng = _rng(2)
    n, b, N, e = 48, 8, 3, 2
    A = rng.standard_normal((6, n))
    B = rng.standard_normal((n, 5))
    h, s = oracle.hash_tables(n, b, N, e, 99)
    mask = 0b10110
    M = np.zeros((n, n))
    for j in (1, 2, 4):
        for p in range(n):
            for q in range(n):
                if h[j, p] == h[j, q]:
                    M[p, q] += s[j, p] * s[j, q]
    C_bf = A @ (M / 3.0) @ B
    assert oracle.rel_frob(oracle.oversketch(A, B, h, s, b, mask), C_bf) < 1e-13


# ----------------------------------------------------- special cases ----

def test_injective_hash_is_exact():
    # b >= n with an injective bucket map: S_j S_j^T = I, so C = AB exactly.
    rng = _rng(4)
    n, b, N, e = 40, 64, 3, 1
    A = rng.standard_normal((9, n))
    B = rng.standard_normal((n, 7))
    h = np.array([[(i + 5 * j) % b for i in range(n)] for j in range(N + e)], dtype=np.uint32)
    s = np.where(rng.random((N + e, n)) < 0.5, -1, 1).astype(np.int8)
    for mask in (0b1111, 0b0111, 0b1010, 0b0001):
        C = oracle.oversketch(A, B, h, s, b, mask)
        assert oracle.rel_frob(C, A @ B) < 1e-14


def test_n_equals_one_is_exact():
    rng = _rng(5)
    A = rng.standard_normal((4, 1))
    B = rng.standard_normal((1, 3))
    h, s = oracle.hash_tables(1, 16, 4, 1, 3)
    assert oracle.rel_frob(oracle.oversketch(A, B, h, s, 16, 0b10111), A @ B) < 1e-15


def test_b_equals_one_rank_k():
    # b = 1: every index in bucket 0, C = (1/k) sum_j (A sigma_j)(sigma_j^T B)
    rng = _rng(6)
    n = 30
    A = rng.standard_normal((5, n))
    B = rng.standard_normal((n, 4))
    h, s = oracle.hash_tables(n, 1, 3, 1, 8)
    assert (h == 0).all()
    mask = 0b1011
    ref = sum(np.outer(A @ s[j], s[j] @ B) for j in (0, 1, 3)) / 3.0
    assert oracle.rel_frob(oracle.oversketch(A, B, h, s, 1, mask), ref) < 1e-14


def test_diagonal_of_sketch_gram_is_one():
    # every row of every Count-sketch block has exactly one +-1
    for seed in range(20):
        h, s = oracle.hash_tables(100, 16, 4, 2, seed)
        S = oracle.sketch_matrix(h, s, 16)
        cols = oracle.selected_columns(0b110111, 6, 16)
        G = S[:, cols] @ S[:, cols].T / 5.0
        assert np.array_equal(np.diag(G), np.ones(100))


def test_linearity_and_sign_flip():
    rng = _rng(7)
    n, b = 64, 8
    A1, A2 = rng.standard_normal((2, 5, n))
    B = rng.standard_normal((n, 6))
    h, s = oracle.hash_tables(n, b, 3, 1, 1)
    mask = 0b1101
    f = lambda X: oracle.oversketch(X, B, h, s, b, mask)
    assert oracle.rel_frob(f(2.0 * A1 - 3.0 * A2), 2.0 * f(A1) - 3.0 * f(A2)) < 1e-13
    # flipping every sign of a block leaves S_j S_j^T unchanged
    assert oracle.rel_frob(oracle.oversketch(A1, B, h, -s, b, mask), f(A1)) < 1e-14


def test_mask_uses_only_kept_blocks():
    rng = _rng(8)
    n, b, N, e = 80, 8, 3, 2
    A = rng.standard_normal((4, n))
    B = rng.standard_normal((n, 4))
    h, s = oracle.hash_tables(n, b, N, e, 21)
    mask = 0b11010
    C = oracle.oversketch(A, B, h, s, b, mask)
    for j in range(N + e):
        # relabelling the buckets of a block leaves S_j S_j^T unchanged
        h2 = h.copy()
        h2[j] = (h2[j] + 3) % b
        assert oracle.rel_frob(oracle.oversketch(A, B, h2, s, b, mask), C) < 1e-14
        # flipping half of a block's signs changes S_j S_j^T
        s2 = s.copy()
        s2[j, : n // 2] *= -1
        C2 = oracle.oversketch(A, B, h, s2, b, mask)
        if (mask >> j) & 1:
            assert oracle.rel_frob(C2, C) > 1e-3
        else:
            assert np.array_equal(C2, C)
    with pytest.raises(ValueError):
        oracle.oversketch(A, B, h, s, b, 0)
    with pytest.raises(ValueError):
        oracle.oversketch(A, B, h, s, b, 1 << (N + e))


# ---------------------------------------------- statistics (appendix) ----

def test_unbiased_gram():
    # Lemma "sketch_properties": E[S_sel S_sel^T] = I (per-seed mean of
    # k blocks); off-diagonal entries average k terms that are +-1 w.p. 1/b.
    n, b, N, e = 24, 4, 3, 1
    mask = 0b1011
    k = 3
    T = 4000
    acc = np.zeros((n, n))
    for seed in range(T):
        h, s = oracle.hash_tables(n, b, N, e, 1000 + seed)
        S = oracle.sketch_matrix(h, s, b)[:, oracle.selected_columns(mask, N + e, b)]
        acc += S @ S.T / k
    mean = acc / T
    off = mean[~np.eye(n, dtype=bool)]
    sd = np.sqrt(1.0 / (k * b) / T)
    assert np.abs(off).max() < 5.5 * sd
    assert np.allclose(np.diag(mean), 1.0)


def test_expected_error_closed_form_and_bounds():
    # Lemma "countEV" exact variance summed over entries (Lemma "lemma2"):
    # Monte-Carlo mean of ||AB - C||^2 over seeds matches the closed form,
    # the closed form is below the (2/d)||A||^2||B||^2 bound (d = k b), and
    # the Markov step of Thm 4.1 holds for eps*theta = 2/d.
    rng = _rng(9)
    m, n, l, b, N, e = 6, 96, 5, 8, 4, 1
    A = rng.standard_normal((m, n))
    B = rng.standard_normal((n, l)) + 0.5 * A.T[:, :l]
    mask = 0b11101
    k = 4
    AB = A @ B
    errs = []
    for seed in range(3000):
        h, s = oracle.hash_tables(n, b, N, e, 50_000 + seed)
        C = oracle.oversketch(A, B, h, s, b, mask)
        errs.append(((C - AB) ** 2).sum())
    errs = np.array(errs)
    expect = oracle.expected_sq_error(A, B, k, b)
    se = errs.std() / np.sqrt(len(errs))
    assert abs(errs.mean() - expect) < 5 * se
    nA, nB = (A * A).sum(), (B * B).sum()
    d = k * b
    assert expect <= 2.0 / d * nA * nB
    theta = 0.25
    eps = 2.0 / d / theta
    assert (errs > eps * nA * nB).mean() <= theta


def test_scale_is_one_over_kept_blocks():
    # graceful degradation: keeping k < N blocks stays unbiased with 1/k
    rng = _rng(10)
    m, n, l, b, N, e = 3, 40, 3, 4, 4, 1
    A = rng.standard_normal((m, n))
    B = rng.standard_normal((n, l))
    AB = A @ B
    acc = np.zeros_like(AB)
    T = 3000
    for seed in range(T):
        h, s = oracle.hash_tables(n, b, N, e, 7000 + seed)
        acc += oracle.oversketch(A, B, h, s, b, 0b00101)   # k = 2 < N
    mean = acc / T
    sd = np.sqrt(oracle.expected_sq_error(A, B, 2, b) / AB.size / T)
    assert np.abs(mean - AB).max() < 6 * sd


# ----------------------------------------------------------- gradient ----

def test_gradient_matches_finite_differences():
    # C is linear in X for fixed G (and in G for fixed X): central
    # differences of L = <dC, C> are exact up to rounding for any step.
    from paper_1811_02653_gb300 import workloads as W
    w = W.AUTOGRAD_FD
    X = w.left().astype(np.float64)
    G = w.right().astype(np.float64)
    dC = w.upstream_grad().astype(np.float64)
    h, s = oracle.hash_tables(w.n, w.b, w.N, w.e, w.hash_seed)
    dX, dG = oracle.gradients(X, G, dC, h, s, w.b, w.mask)
    L = lambda X_, G_: (dC * oracle.oversketch(X_, G_, h, s, w.b, w.mask)).sum()
    rng = _rng(11)
    for _ in range(3):
        DX = rng.standard_normal(X.shape)
        DG = rng.standard_normal(G.shape)
        t = 0.5
        fdX = (L(X + t * DX, G) - L(X - t * DX, G)) / (2 * t)
        fdG = (L(X, G + t * DG) - L(X, G - t * DG)) / (2 * t)
        assert abs(fdX - (dX * DX).sum()) < 1e-10 * max(1.0, abs(fdX))
        assert abs(fdG - (dG * DG).sum()) < 1e-10 * max(1.0, abs(fdG))
    for (r, i) in [(0, 0), (5, 77), (63, 511)]:
        E = np.zeros_like(X)
        E[r, i] = 1.0
        fd = (L(X + E, G) - L(X - E, G)) / 2.0
        assert abs(fd - dX[r, i]) < 1e-10 * max(1.0, abs(fd))


# --------------------------------------------------------- quantisers ----

def test_round_bf16_matches_torch_rne():
    torch = pytest.importorskip("torch")
    rng = _rng(12)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32),
                        (rng.standard_normal(2000) * 1e-39).astype(np.float32),   # subnormal
                        (rng.standard_normal(2000) * 1e30).astype(np.float32),
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, -0.0,
                                  2 ** -133, 3 * 2 ** -134], dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_bf16(x), ref)
    # ties go to even
    assert oracle.round_bf16(np.float32(1 + 2 ** -8)) == 1.0
    assert oracle.round_bf16(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def test_round_fp8_e4m3_definition():
    # OCP FP8 E4M3: 3 mantissa bits, bias 7, largest finite 448, smallest
    # subnormal 2^-9, saturating.
    r = oracle.round_fp8_e4m3
    assert r(448.0) == 448.0 and r(1000.0) == 448.0 and r(-1e9) == -448.0
    assert r(2.0 ** -9) == 2.0 ** -9 and r(2.0 ** -10) == 0.0 and r(1.5 * 2 ** -10) == 2.0 ** -9
    assert r(1.0625) == 1.0 and r(1.1875) == 1.25 and r(240.0) == 240.0 and r(232.0) == 224.0
    vals = np.array([m / 8 * 2.0 ** ex for ex in range(-6, 9) for m in range(8, 16)] +
                    [m / 8 * 2.0 ** -6 for m in range(0, 8)])
    vals = vals[vals <= 448]
    assert np.array_equal(r(vals), vals)            # every finite code is a fixed point
    torch = pytest.importorskip("torch")
    if hasattr(torch, "float8_e4m3fn"):
        x = np.clip(_rng(13).standard_normal(20000) * 50, -440, 440).astype(np.float32)
        ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
        assert np.array_equal(r(x), ref)


def test_fp8_scale_exponent():
    f = oracle.fp8_scale_exponent
    assert list(f(np.array([448.0, 448.0001, 224.0, 225.0, 1.0, 0.0]))) == [0, 1, -1, 0, -8, 0]
    x = _rng(14).standard_normal((5, 300)) * 3
    q, e = oracle.quantize_fp8_rows(x)
    assert e.shape == (5, 3)
    assert np.abs(q).max() <= 448
    deq = oracle.dequantize_fp8_rows(q, e)
    assert oracle.rel_frob(deq, x) < 0.05


def test_masked_product_blocks_reduces_to_one_mask():
    # the same kept set in every block of C is the single-mask product
    rng = np.random.default_rng(41)
    b, P = 8, 5
    At = rng.standard_normal((21, P * b))
    Bt = rng.standard_normal((P * b, 13))
    mask = 0b10110
    masks = [[mask] * 4 for _ in range(6)]                    # 4 x 4 blocks, ragged edges
    C = oracle.masked_product_blocks(At, Bt, b, masks, 4, 4)
    assert np.allclose(C, oracle.masked_product(At, Bt, b, mask), rtol=1e-13, atol=1e-13)


def test_masked_product_blocks_brute_force():
    # block (i, j) of C from the explicit sketch: A (S_ij S_ij^T / k_ij) B with S_ij the
    # kept columns of Eq. 3's S; an empty kept set gives a zero block
    rng = np.random.default_rng(42)
    n, b, N, e = 40, 4, 3, 2
    P = N + e
    h, s = oracle.hash_tables(n, b, N, e, 3)
    S = oracle.sketch_matrix(h, s, b)
    A = rng.standard_normal((10, n))
    B = rng.standard_normal((n, 7))
    bm, bn = 4, 3
    masks = [[int(rng.integers(1, 1 << P)) for _ in range(3)] for _ in range(3)]
    masks[1][2] = 0
    C = oracle.masked_product_blocks(A @ S, S.T @ B, b, masks, bm, bn)
    for i in range(3):
        for j in range(3):
            rs, cs = slice(i * bm, min(10, (i + 1) * bm)), slice(j * bn, min(7, (j + 1) * bn))
            if masks[i][j] == 0:
                assert (C[rs, cs] == 0).all()
                continue
            cols = [t * b + q for t in range(P) if (masks[i][j] >> t) & 1 for q in range(b)]
            Ssel = S[:, cols]
            k = bin(masks[i][j]).count("1")
            ref = A[rs] @ (Ssel @ Ssel.T / k) @ B[:, cs]
            assert np.allclose(C[rs, cs], ref, rtol=1e-12, atol=1e-12)


def test_expected_error_factored_equals_the_dense_form():
    # the factored closed form is the same number as the dense one: random
    # factors, and Sec. 5.1's rank-2 matrix A(x, y) = x + y with B = A^T
    rng = _rng(21)
    U, V = rng.standard_normal((6, 2)), rng.standard_normal((96, 2))
    Y, W = rng.standard_normal((96, 3)), rng.standard_normal((5, 3))
    dense = oracle.expected_sq_error(U @ V.T, Y @ W.T, 4, 8)
    assert abs(oracle.expected_sq_error_factored(U, V, Y, W, 4, 8) - dense) <= 1e-10 * dense
    m, n = 40, 240
    x, y = np.arange(1, m + 1.0), np.arange(1, n + 1.0)
    A = x[:, None] + y[None, :]
    Uf, Vf = np.stack([x, np.ones(m)], 1), np.stack([np.ones(n), y], 1)
    dense = oracle.expected_sq_error(A, A.T, 26, 16)
    assert abs(oracle.expected_sq_error_factored(Uf, Vf, Vf, Uf, 26, 16) - dense) <= 1e-10 * dense


def test_per_block_kept_sets_keep_the_expected_error():
    # Alg. 3's rule per block of C: every block keeps k of its own P sketch
    # blocks; each entry's variance is still (1/k) times one block's, so the
    # expected squared error is the same closed form (Monte Carlo over seeds)
    rng = _rng(22)
    m, n, l, b, N, e = 8, 96, 8, 8, 4, 1
    P = N + e
    A = rng.standard_normal((m, n))
    B = rng.standard_normal((n, l)) + 0.5 * A.T
    AB = A @ B
    errs = []
    for seed in range(2000):
        h, s = oracle.hash_tables(n, b, N, e, 90_000 + seed)
        masks = [[((1 << P) - 1) & ~(1 << int(t)) for t in rng.integers(0, P, size=2)] for _ in range(2)]
        C = oracle.masked_product_blocks(oracle.sketch_left(A, h, s, b), oracle.sketch_right(B, h, s, b),
                                         b, masks, 4, 4)
        errs.append(((C - AB) ** 2).sum())
    errs = np.array(errs)
    expect = oracle.expected_sq_error(A, B, N, b)
    assert abs(errs.mean() - expect) < 5 * errs.std() / np.sqrt(len(errs))


def test_sec51_operands_and_exact_product():
    # Sec. 5.1's A(x, y) = x + y: the factors reproduce A, B = A^T, and the closed-form
    # A A^T used as the exact reference equals a plain FP64 product
    torch = pytest.importorskip("torch")
    from paper_1811_02653_gb300 import workloads
    m, n = 40, 300
    A, B, AB = workloads.sec51_device(m, n, "cpu")
    U, V = workloads.sec51_factors(m, n)
    A64 = U @ V.T
    assert np.array_equal(A.numpy().astype(np.float64), A64)
    assert np.array_equal(B.numpy(), A.numpy().T)
    ref = A64 @ A64.T
    assert np.allclose(AB.numpy().astype(np.float64), ref, rtol=2.0 ** -23, atol=0)
