"""A CPU model of the split-product arithmetic the tensor-core row passes use, checked against
exact arithmetic, and a small rand_cholQR built on it.

This pins the numerical design of the tensor-core path (products with explicit triangular
inverses, Algorithm 3's two solves; eight balanced 7-bit digits of a 54-bit fixed point; slice
pairs s + t <= 7 kept exactly, s + t = 8 folded in at weight 2^-7; integer recombination) on
the CPU.  It is a model written from that description, independent of the CUDA sources and of
the oracle; the GPU tests check the kernels themselves against the oracle.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.linalg import cholesky, solve_triangular

import synthetic

BIAS = sum(64 << (7 * p) for p in range(8))


def scale_exp(A, axis):
    """E with max |a| < 2^E along `axis`, clamped below at -100 (zero rows/columns)."""
    mx = np.max(np.abs(A), axis=axis, keepdims=True)
    E = np.frexp(mx)[1]
    return np.where(mx > 0, np.maximum(E, -100), -100)


def fix54(A, E):
    """trunc(a 2^(54 - E)) exactly, as int64 (|.| < 2^54)."""
    F = np.trunc(np.ldexp(np.abs(A), (54 - E) * np.ones(A.shape, dtype=np.int64)))
    F = F.astype(np.int64)
    return np.where(A < 0, -F, F)


def digits(Xi):
    """Balanced digits d_p in [-64, 63], X = sum_p d_p 2^(7p); returned by slice s = 7 - p."""
    Y = Xi + BIAS
    assert Y.min() >= 0 and Y.max() < 2 ** 56
    return [((Y >> (7 * (7 - s))) & 127) - 64 for s in range(8)]


def split_product(X, B):
    """Y = X B the way the solve kernel forms it (row scales of X, column scales of B)."""
    E, F = scale_exp(X, 1), scale_exp(B, 0)
    dx, db = digits(fix54(X, E)), digits(fix54(B, F))
    D = []
    for g in range(9):
        acc = np.zeros((X.shape[0], B.shape[1]), dtype=np.int64)
        for s in range(8):
            t = g - s
            if 0 <= t < 8:
                acc += dx[s] @ db[t]
        assert np.abs(acc).max() <= 2 ** 21
        D.append(acc)
    # region 8 summed first in region 7's FP32 accumulator, scaled by 2^-7 (scale-input-d),
    # then region 7's products added: one FP32 rounding, then the exact integer conversion
    r7 = (D[7].astype(np.float32) + D[8].astype(np.float32) * np.float32(2.0 ** -7)).astype(np.float32)
    D7 = np.rint(r7.astype(np.float64)).astype(np.int64)
    th = (D[0] << 21) + (D[1] << 14) + (D[2] << 7) + D[3]
    tl = (D[4] << 21) + (D[5] << 14) + (D[6] << 7) + D7
    t = (th << 25) + (tl >> 3)  # T / 8
    return np.ldexp(t.astype(np.float64), E + F - 56)


def test_split_product_error_is_below_the_scale_product():
    rng = synthetic.rng(11)
    m, n = 40, 64
    X = rng.standard_normal((m, n)) * np.exp(rng.uniform(-20, 20, (m, 1)))
    X[3] = 0.0                                         # a zero row
    X[5, ::3] *= 1e-12                                 # a row with a wide spread
    B = np.triu(rng.standard_normal((n, n)) * np.exp(rng.uniform(-15, 15, (1, n))))
    Y = split_product(X, B)
    E, F = scale_exp(X, 1), scale_exp(B, 0)
    worst = 0.0
    for i in range(m):
        for k in range(0, n, 7):
            exact = sum(Fraction(float(X[i, j])) * Fraction(float(B[j, k])) for j in range(n))
            err = abs(Fraction(float(Y[i, k])) - exact) / Fraction(2) ** int(E[i, 0] + F[0, k])
            worst = max(worst, float(err))
    assert np.all(Y[3] == 0.0)
    assert worst <= 2.0 ** -50, worst


def test_split_product_is_exact_on_short_integers():
    # entries with few significant bits: the fixed point and the kept pairs hold them exactly
    rng = synthetic.rng(12)
    X = rng.integers(-2 ** 10, 2 ** 10, (17, 32)).astype(np.float64)
    B = np.triu(rng.integers(-2 ** 10, 2 ** 10, (32, 32)).astype(np.float64))
    np.testing.assert_array_equal(split_product(X, B), X @ B)


def _inverse_by_columns(R):
    n = R.shape[0]
    X = np.zeros((n, n))
    for k in range(n):
        x = np.zeros(n)
        x[k] = 1.0 / R[k, k]
        for i in range(k - 1, -1, -1):
            x[i] = -np.dot(R[i, i + 1:k + 1], x[i + 1:k + 1]) / R[i, i]
        X[:, k] = x
    return X


@pytest.mark.parametrize("kappa", [1e4, 1e12, 1e15])
def test_rand_cholqr_with_split_solves_meets_the_targets(kappa):
    """Algorithm 3 with both solves as split products by column-wise inverses: the residual
    and orthogonality targets hold up to kappa = 1e15 (reading of the tensor-core path)."""
    m, n = 4096, 32
    V = synthetic.make_v(m, n, kappa, seed=3)
    S = synthetic.rng(4).standard_normal((4 * n, m)) / np.sqrt(4 * n)
    Rs = np.linalg.qr(S @ V, mode="r")
    Rs = Rs * np.sign(np.diag(Rs))[:, None]
    W = split_product(V, _inverse_by_columns(Rs))
    Rc = cholesky(W.T @ W, lower=False)
    Q = split_product(W, _inverse_by_columns(Rc))
    R = Rc @ Rs
    orth = np.linalg.norm(Q.T @ Q - np.eye(n), 2)
    resid = np.linalg.norm(V - Q @ R) / np.linalg.norm(V)
    assert orth <= 1e-14, orth
    assert resid <= 1e-14, resid
    # the same steps with row-wise substitution, for scale
    W2 = solve_triangular(Rs, V.T, trans="T").T
    Rc2 = cholesky(W2.T @ W2, lower=False)
    Q2 = solve_triangular(Rc2, W2.T, trans="T").T
    assert np.linalg.norm(V - Q2 @ (Rc2 @ Rs)) / np.linalg.norm(V) <= 1e-15
