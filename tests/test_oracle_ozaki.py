"""Pins of the slice-product FP64 matrix product (oracle/ozaki.py) against exact rational
arithmetic, integer arithmetic and the bounds of the splitting."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rand(rng, d, n, spread=6):
    """Columns of mixed magnitude (2^-spread .. 2^spread) and sign."""
    X = rng.standard_normal((d, n))
    return X * np.ldexp(1.0, rng.integers(-spread, spread + 1, size=n))[None, :]


def test_column_exponents_are_ceil_log2():
    X = np.array([[0.5, 3.0, 0.0, -1.0, 1e-3],
                  [0.25, -4.0, 0.0, 0.75, 0.0]])
    # max |x|: 0.5 -> -1, 4 -> 2, 0 -> 0 (zero column), 1 -> 0, 1e-3 -> ceil(log2 1e-3) = -9
    assert list(ozaki.column_exponents(X)) == [-1, 2, 0, 0, -9]


@pytest.mark.parametrize("beta,s", [(9, 6), (8, 7), (7, 4)])
def test_split_reconstructs_exactly_with_bounded_integer_slices(beta, s):
    rng = np.random.default_rng(101 + beta)
    X = _rand(rng, 40, 4)
    X[:, 3] = 0.0  # an all-zero column
    a, u, res = ozaki.split(X, beta, s)
    E = ozaki.column_exponents(X)
    assert np.all(np.abs(a) <= 2 ** (beta - 1))
    assert np.all(a[:, :, 3] == 0) and np.all(u[:, 3] == 0) and np.all(res[:, 3] == 0)
    for j in range(3):
        # units are the stated powers of two
        for k in range(s):
            assert u[k, j] == 2.0 ** (E[j] - (beta - 1) - k * beta)
        # residual bound |res| <= 2^(E - s beta)
        assert np.max(np.abs(res[:, j])) <= 2.0 ** (E[j] - s * beta)
        # x = sum_k a_k u_k + res, exactly (rational arithmetic)
        for r in range(0, 40, 7):
            lhs = Fraction(float(X[r, j]))
            rhs = sum((Fraction(int(a[k, r, j])) * Fraction(float(u[k, j])) for k in range(s)),
                      Fraction(0)) + Fraction(float(res[r, j]))
            assert lhs == rhs


def test_slices_fit_bf16_exactly_up_to_beta_9():
    rng = np.random.default_rng(7)
    a, _, _ = ozaki.split(_rand(rng, 200, 3), 9, 6)
    f = a.astype(np.float32)
    assert np.array_equal(ozaki.bf16_roundtrip(f), f)
    # one bit more (beta = 10: integers up to 512) no longer fits
    big = np.arange(257, 512, 2, dtype=np.float32)  # odd integers above 256
    assert not np.array_equal(ozaki.bf16_roundtrip(big), big)


def test_bf16_roundtrip_rounds_to_nearest_even():
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, 256.0, 257.0, 259.0,
                  -257.0, 0.0], dtype=np.float32)
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, 256.0, 256.0, 260.0, -256.0, 0.0],
                    dtype=np.float32)
    assert np.array_equal(ozaki.bf16_roundtrip(x), want)


@pytest.mark.parametrize("beta", [8, 9])
def test_fp32_chunk_accumulation_is_exact_within_the_bound(beta):
    K = ozaki.max_exact_chunk(beta)
    assert K == 2 ** (26 - 2 * beta)
    rng = np.random.default_rng(beta)
    m = 2 ** (beta - 1)
    for trial in range(3):
        a = rng.integers(-m, m + 1, size=3 * K)
        b = rng.integers(-m, m + 1, size=3 * K)
        if trial == 2:  # worst case: every product at the maximum
            a[:] = m
            b[:] = m
        exact = int(np.dot(a.astype(np.int64), b.astype(np.int64)))
        assert ozaki.fp32_chunk_sum(a, b, K) == exact


def test_fp32_accumulation_past_the_bound_loses_bits():
    """With 4x the chunk length, odd products of size ~2^16 push the FP32 running sum past
    2^24: the chunk limit is necessary, not just sufficient."""
    beta = 9
    K = ozaki.max_exact_chunk(beta)
    a = np.full(4 * K, 255, dtype=np.int64)
    b = np.full(4 * K, 255, dtype=np.int64)
    exact = int(np.dot(a, b))
    assert ozaki.fp32_chunk_sum(a, b, K) == exact
    assert ozaki.fp32_chunk_sum(a, b, 4 * K) != exact


def test_slice_products_are_exact_integers():
    rng = np.random.default_rng(3)
    a, _, _ = ozaki.split(_rand(rng, 300, 2), 9, 6)
    b, _, _ = ozaki.split(_rand(rng, 300, 3), 9, 6)
    P = ozaki.slice_product(a[1], b[2])
    for i in range(2):
        for j in range(3):
            assert P[i, j] == sum(int(x) * int(y) for x, y in zip(a[1][:, i], b[2][:, j]))


@pytest.mark.parametrize("beta,s", [(9, 6), (8, 7)])
def test_gram_matches_exact_rational_product_within_bound(beta, s):
    rng = np.random.default_rng(11 * beta)
    A = _rand(rng, 64, 3)
    B = _rand(rng, 64, 4)
    B[:, 2] = A[:, 0]  # a column shared with A (a Gram diagonal entry)
    C = ozaki.gram(A, B, beta, s)
    Ce = ozaki.exact_gram(A, B)
    bound = ozaki.error_bound(A, B, beta, s) + np.abs(Ce) * 2.0 ** -53
    assert np.all(np.abs(C - Ce) <= bound)
    # FP64-class: within a few units of the FP64 product's own accuracy
    scale = np.abs(A).T @ np.abs(B)
    assert np.max(np.abs(C - Ce) / scale) < 64 * 2.0 ** -53


def test_gram_with_too_few_slices_stays_within_its_larger_bound():
    """s = 3 (27 bits) truncates visibly; the error respects the truncation term of the bound
    and is far above FP64 rounding, so the bound is not vacuous."""
    rng = np.random.default_rng(5)
    A = _rand(rng, 64, 3, spread=2)
    B = _rand(rng, 64, 3, spread=2)
    C = ozaki.gram(A, B, 9, 3)
    Ce = ozaki.exact_gram(A, B)
    err = np.abs(C - Ce)
    assert np.all(err <= ozaki.error_bound(A, B, 9, 3) + np.abs(Ce) * 2.0 ** -53)
    assert np.max(err / (np.abs(A).T @ np.abs(B))) > 1e-12


def test_gram_at_the_workload_length_agrees_with_fp64():
    """d = 46128 (the 32-atom cluster's basis), 8 columns: agreement with numpy's FP64
    product to the FP64 rounding level of a sum of that length."""
    rng = np.random.default_rng(46128)
    A = _rand(rng, 46128, 8, spread=3)
    B = _rand(rng, 46128, 8, spread=3)
    C = ozaki.gram(A, B)
    ref = A.T @ B
    scale = np.abs(A).T @ np.abs(B)
    assert np.max(np.abs(C - ref) / scale) < 1e-14


def test_zero_and_power_of_two_columns():
    A = np.zeros((10, 2))
    A[3, 1] = 2.0 ** -20
    B = np.zeros((10, 2))
    B[3, 0] = -(2.0 ** 7)
    B[5, 1] = 1.0
    C = ozaki.gram(A, B)
    assert np.array_equal(C, np.array([[0.0, 0.0], [-(2.0 ** -13), 0.0]]))


def test_digits_needed():
    assert ozaki.digits_needed(9) == 6 and ozaki.digits_needed(8) == 7
    assert ozaki.digits_needed(7) == 8


def test_rotation_shape_matches_exact_product():
    """The dense step's rotations X Q (d x n times n x n) are the same scheme with the
    contraction over n: gram(X^T, Q), with one exponent per row of X. Checked against exact
    rational arithmetic within the bound."""
    rng = np.random.default_rng(2024)
    X = rng.standard_normal((12, 5)) * np.ldexp(1.0, rng.integers(-5, 6, size=12))[:, None]
    Q = np.linalg.qr(rng.standard_normal((5, 5)))[0]
    C = ozaki.gram(X.T, Q)
    Ce = ozaki.exact_gram(X.T, Q)
    bound = ozaki.error_bound(X.T, Q, 9, 6) + np.abs(Ce) * 2.0 ** -53
    assert C.shape == (12, 5)
    assert np.all(np.abs(C - Ce) <= bound)
    assert np.max(np.abs(C - X @ Q) / (np.abs(X) @ np.abs(Q))) < 64 * 2.0 ** -53


def test_gram_is_the_truncated_sum_rounded_once():
    """gram() is the exact value of the kept slice pairs' scaled products rounded once to FP64:
    checked against exact rational sums over the pairs (k, l) themselves, rounded by
    float(Fraction), entry by entry and bit for bit."""
    rng = np.random.default_rng(31)
    A = _rand(rng, 50, 3)
    B = _rand(rng, 50, 3)
    beta, s = 7, 8
    a, u, _ = ozaki.split(A, beta, s)
    b, v, _ = ozaki.split(B, beta, s)
    C = ozaki.gram(A, B, beta, s)
    for i in range(3):
        for j in range(3):
            tot = Fraction(0)
            for k in range(s):
                for l in range(s - k):
                    P = sum(int(x) * int(y) for x, y in zip(a[k][:, i], b[l][:, j]))
                    tot += Fraction(P) * Fraction(float(u[k, i])) * Fraction(float(v[l, j]))
            assert C[i, j] == float(tot)
