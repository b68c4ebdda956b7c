"""FP64 matrix products from exact products of small-integer slices (the error-free splitting
of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012), in its integer-slice form).

Test infrastructure only (see oracle/__init__.py).

The dense steps of the ChFSI iteration (Sec. 3.2: the Gram matrices of Cholesky-QR and
Rayleigh-Ritz, and the rotations by their small factors) are FP64 products C = A^T B with a
long contraction over the basis. On hardware whose FP64 rate is low, such a product can be
taken from low-precision products that are exact:
- **Split.** Each column x of A (and of B) with mu = max|x| > 0 and E = ceil(log2 mu) is written
  as x = sum_{k=1..s} a_k u_k + res. The unit of slice k is u_k = 2^(E - (beta-1) - (k-1) beta).
  The slice is a_k = round_to_nearest_even(r_{k-1} / u_k), with r_0 = x and
  r_k = r_{k-1} - a_k u_k. Every a_k is an integer with |a_k| <= 2^(beta-1), so a BF16 value holds
  it exactly for beta <= 9, and |res| = |r_s| <= u_s / 2 = 2^(E - s beta).
- **Exact slice products.** P_kl = a_k^T b_l is a sum of integer products of magnitude at most
  2^(2 beta - 2). Accumulated in FP32 over chunks of at most 2^(26 - 2 beta) rows, every partial
  sum is an integer below 2^24 and so exact. The chunk sums are integers that FP64 adds exactly
  while they stay below 2^53.
- **Sum.** C_ij ~= sum over pairs (k, l) with k + l <= s + 1 of u_k(i) v_l(j) P_kl(i, j). Every
  term is an integer times a power of two, so the truncated sum has an exact value; C_ij is that
  value rounded once to FP64 (round to nearest, ties to even). The method fixes no order for
  this sum; rounding the exact sum once is the one result that does not depend on an order.
  Dropping the pairs with k + l > s + 1 and the residuals leaves an error of order
  2^(2 - s beta) mu_i nu_j d, like that of an FP64 product for s beta >= 53.

Here P_kl is computed in int64 (its plain definition); `fp32_chunk_sum` states the FP32
accumulation that a tensor-core kernel would use, and the tests check that it is exact within
the bound.
"""
from __future__ import annotations

import math

import numpy as np


def column_exponents(X: np.ndarray) -> np.ndarray:
    """E_j = ceil(log2 max_r |X[r, j]|) per column (0 for an all-zero column)."""
    X = np.asarray(X, dtype=np.float64)
    mu = np.max(np.abs(X), axis=0) if X.shape[0] else np.zeros(X.shape[1])
    E = np.zeros(X.shape[1], dtype=np.int64)
    nz = mu > 0
    # frexp: mu = m 2^e with 0.5 <= m < 1, so ceil(log2 mu) = e, or e - 1 when m = 0.5
    m, e = np.frexp(mu[nz])
    E[nz] = np.where(m == 0.5, e - 1, e)
    return E


def split(X: np.ndarray, beta: int, s: int):
    """Slices of every column of X (d x n, FP64): integers a (s x d x n, int64), units
    u (s x n, FP64 powers of two), and the residual (d x n) left after s slices."""
    X = np.asarray(X, dtype=np.float64)
    d, n = X.shape
    E = column_exponents(X)
    a = np.zeros((s, d, n), dtype=np.int64)
    u = np.zeros((s, n), dtype=np.float64)
    r = X.copy()
    for k in range(s):
        uk = np.ldexp(1.0, (E - (beta - 1) - k * beta).astype(np.int64))
        q = np.rint(r / uk[None, :])  # round half to even; r / uk is exact (power of two)
        a[k] = q.astype(np.int64)
        r = r - q * uk[None, :]  # exact: q uk is the nearest multiple of uk to r
        u[k] = uk
    zero = np.max(np.abs(X), axis=0) == 0 if d else np.ones(n, dtype=bool)
    u[:, zero] = 0.0
    return a, u, r


def slice_product(a_k: np.ndarray, b_l: np.ndarray) -> np.ndarray:
    """P = a_k^T b_l exactly (int64). Where every partial sum stays below 2^53 in magnitude
    (d max|a| max|b| < 2^53) an FP64 matrix product is exact in any order of summation and
    takes its place (int64 products have no BLAS)."""
    d = a_k.shape[0]
    m = max(int(np.abs(a_k).max(initial=0)), 1) * max(int(np.abs(b_l).max(initial=0)), 1)
    if d * m < 2 ** 53:
        return np.rint(a_k.T.astype(np.float64) @ b_l.astype(np.float64)).astype(np.int64)
    return a_k.T.astype(np.int64) @ b_l.astype(np.int64)


def fp32_chunk_sum(a: np.ndarray, b: np.ndarray, chunk: int) -> float:
    """sum_r a[r] b[r] for integer vectors, accumulated as a tensor-core kernel would: each
    product and each running sum in FP32 within chunks of `chunk` rows, the chunk sums in
    FP64."""
    total = 0.0
    for c0 in range(0, len(a), chunk):
        acc = np.float32(0.0)
        for x, y in zip(a[c0:c0 + chunk], b[c0:c0 + chunk]):
            acc = np.float32(acc + np.float32(np.float32(x) * np.float32(y)))
        total += float(acc)
    return total


def max_exact_chunk(beta: int) -> int:
    """Rows whose integer slice products always sum exactly in FP32: 2^(26 - 2 beta)."""
    return 1 << (26 - 2 * beta)


def max_exact_diagonal_window(beta: int, s: int) -> int:
    """Rows over which the products of all pairs on one diagonal k + l = t (at most s pairs)
    always sum exactly in FP32: s 2^(2 beta - 2) per row, so the largest power of two with
    rows s 2^(2 beta - 2) <= 2^24."""
    w = (1 << 24) // (s << (2 * beta - 2))
    return 1 << (w.bit_length() - 1)


def gram(A: np.ndarray, B: np.ndarray, beta: int = 9, s: int = 6) -> np.ndarray:
    """C = A^T B (A: d x na, B: d x nb, FP64) from the exact slice products of the pairs
    (k, l) with k + l <= s + 1 (1-based): their scaled sum, exact, rounded once to FP64.

    All pairs with the same k + l = t (0-based) share the unit 2^(E_i + F_j - 2 (beta - 1) -
    t beta), so the exact value is 2^(E_i + F_j - 2 (beta - 1) - (s - 1) beta) times the
    integer sum over t of D_t 2^((s - 1 - t) beta), D_t = sum_{k + l = t} P_kl. Python
    integers hold it exactly, and float() of an integer rounds to nearest even."""
    a, _, _ = split(A, beta, s)
    b, _, _ = split(B, beta, s)
    E = column_exponents(A)
    F = column_exponents(B)
    D = [sum(slice_product(a[k], b[t - k]) for k in range(t + 1)) for t in range(s)]
    # T = sum_t D_t 2^((s - 1 - t) beta) in Python integers (object arrays: exact, any size)
    T = np.zeros(D[0].shape, dtype=object)
    for t in range(s):
        T = T + (D[t].astype(object) << ((s - 1 - t) * beta))
    e = (E[:, None] + F[None, :]).astype(object) - (2 * (beta - 1) + (s - 1) * beta)
    return np.frompyfunc(lambda v, x: math.ldexp(float(v), x), 2, 1)(T, e).astype(np.float64)


def error_bound(A: np.ndarray, B: np.ndarray, beta: int, s: int) -> np.ndarray:
    """A bound on |gram(A, B) - A^T B| per entry. The dropped pairs (k + l > s + 1) and the two
    residuals contribute at most (s + 2) 2^(E_i + F_j - s beta) d; the final rounding adds at
    most 2^-53 of the result, which the term below (written for a sum that rounds after every
    pair) covers."""
    d = A.shape[0]
    E = column_exponents(A)
    F = column_exponents(B)
    scale = np.ldexp(1.0, (E[:, None] + F[None, :]).astype(np.int64))
    npairs = s * (s + 1) // 2
    trunc = (s + 2) * scale * d * 2.0 ** (-s * beta)
    rnd = npairs * 2.0 ** -53 * (np.abs(A).T @ np.abs(B)) * (1 + 2.0 ** -50)
    return trunc + rnd + 4 * np.finfo(float).tiny


def bf16_roundtrip(x: np.ndarray) -> np.ndarray:
    """x rounded to BF16 (round to nearest even on the FP32 bits) and back to FP32."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> 16) & 1
    r = ((f + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def exact_gram(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^T B in exact rational arithmetic, rounded once to FP64 (small inputs only)."""
    from fractions import Fraction

    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    C = np.zeros((A.shape[1], B.shape[1]))
    for i in range(A.shape[1]):
        fa = [Fraction(float(x)) for x in A[:, i]]
        for j in range(B.shape[1]):
            C[i, j] = float(sum((x * Fraction(float(y)) for x, y in zip(fa, B[:, j])),
                                Fraction(0)))
    return C


def digits_needed(beta: int) -> int:
    """Slices for an FP64-class split: the smallest s with s beta >= 54."""
    return math.ceil(54 / beta)
