"""A CPU model of the split-product arithmetic the tensor-core row passes use, checked against
exact arithmetic, and a small rand_cholQR built on it.

This pins the numerical design of the tensor-core path (products with explicit triangular
inverses, Algorithm 3's two solves; seven balanced byte digits of a 54-bit fixed point; slice
pairs s + t <= 7 kept exactly; integer recombination) on
the CPU.  It is a model written from that description, independent of the CUDA sources and of
the oracle; the GPU tests check the kernels themselves against the oracle.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.linalg import cholesky, solve_triangular

import synthetic

BIAS = sum(128 << (8 * p) for p in range(7))
M23, M24, M35 = np.float32(1.5 * 2 ** 23), np.float32(1.5 * 2 ** 24), np.float32(1.5 * 2 ** 35)


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
    """Balanced byte digits d_p in [-128, 127], X = sum_p d_p 2^(8p); by slice s = 6 - p.
    |X| < 2^54 keeps the leading digit within [-64, 64]."""
    Y = Xi + BIAS
    assert Y.min() >= 0 and Y.max() < 2 ** 56
    d = [((Y >> (8 * (6 - s))) & 255) - 128 for s in range(7)]
    assert np.abs(d[0]).max() <= 64
    return d


def _bits(f32):
    return np.asarray(f32, dtype=np.float32).view(np.uint32).astype(np.int64)


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def recombine(D):
    """T / 2^12 from the eight region accumulators (exact FP32 integers), T = sum_g D_g 2^(8(7-g)),
    with the kernel's steps: regions 0-4 through the 1.5 * 2^23 offset (exact for
    |D| <= 2^22); region 5 split into an even part (1.5 * 2^24 offset) and a remainder in
    {-1, 0, 1}; the remainder, region 6 and region 7 merged by two FP32 fused multiply-adds
    (|r| < 2^31) and taken at a resolution of 2^12 (1.5 * 2^35 offset); the bit patterns summed
    modulo 2^64, regions 0 and 1 in the high word."""
    v = [_f32(d) for d in D]
    for g in range(8):
        assert np.array_equal(v[g].astype(np.int64), D[g])           # exact in FP32
    a = [_bits(v[g] + M23) for g in range(5)]
    for g in range(5):
        assert np.array_equal(a[g] - 0x4B400000, D[g])
    c5 = (v[5] + M24).astype(np.float32)
    q5 = _bits(c5)
    lo = (v[5] - (c5 - M24).astype(np.float32)).astype(np.float32)
    assert np.array_equal(2 * (q5 - 0x4BC00000) + lo.astype(np.int64), D[5])
    r = _f32(v[6].astype(np.float64) * 256 + v[7].astype(np.float64))        # fmaf
    r = _f32(lo.astype(np.float64) * 65536 + r.astype(np.float64))             # fmaf
    assert np.abs(r).max() < 2 ** 31
    qr = _bits((r + M35).astype(np.float32))
    o23, o24, o35 = 0x4B400000, 0x4BC00000, 0x51400000
    c_hi = (o23 * 4096 + o23 * 16) % 2 ** 32
    c_lo = (o23 * 2 ** 28 + o23 * 2 ** 20 + o23 * 2 ** 12 + o24 * 32 + o35) % 2 ** 64
    out = np.empty(D[0].shape, dtype=np.int64)
    for idx in np.ndindex(D[0].shape):  # Python integers: exact modular arithmetic
        hw = (int(a[0][idx]) * 4096 + int(a[1][idx]) * 16 - c_hi) % 2 ** 32
        lw = (int(qr[idx]) + int(q5[idx]) * 32 + int(a[4][idx]) * 2 ** 12 + int(a[3][idx]) * 2 ** 20 +
              int(a[2][idx]) * 2 ** 28 - c_lo) % 2 ** 64
        t = (lw + (hw << 32)) % 2 ** 64
        out[idx] = t - 2 ** 64 if t >= 2 ** 63 else t
    return out


def split_product(X, B, nda=7):
    """Y = X B the way the solve kernel forms it: row scales of X, column scales of B, byte
    digits, slice pairs s + t <= 7 in eight regions per column half; half h (columns
    32h .. 32h + 31) takes the K range j < 32 (h + 1) that an upper-triangular B reaches.
    nda = 6 keeps only X's six leading digits and the pairs s + t <= 6 (seven regions, the
    46-bit products of RANDQR_F32X2)."""
    m, n = X.shape
    assert B.shape == (n, n) and n <= 64
    Xp = np.zeros((m, 64)); Xp[:, :n] = X
    Bp = np.zeros((64, 64)); Bp[:n, :n] = B
    assert np.array_equal(Bp, np.triu(Bp))
    E, F = scale_exp(Xp, 1), scale_exp(Bp, 0)
    dx, db = digits(fix54(Xp, E)), digits(fix54(Bp, F))
    T = np.zeros((m, 64), dtype=np.int64)
    for h in range(2):
        kk, jj = slice(32 * h, 32 * h + 32), slice(0, 32 * (h + 1))
        D = []
        for g in range(8):
            acc = np.zeros((m, 32), dtype=np.int64)
            for s in range(nda):
                t = g - s
                if 0 <= t < 7 and g <= nda:  # the pairs s + t <= nda (nda + 1 regions)
                    acc += dx[s][:, jj] @ db[t][jj, kk]
            assert np.abs(acc).max() <= (2 ** 22 if g <= 4 else 2 ** 23 - 1)
            D.append(acc)
        T[:, kk] = recombine(D)
    return np.ldexp(T.astype(np.float64), E + F - 56)[:, :n]


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


def test_split_product_at_the_digit_extremes():
    # every digit below the leading one at -128 (products of +2^14) and the leading digit at
    # -63: the region sums come within a few percent of the bounds the recombination relies on
    X0 = 63 * 2 ** 48 + sum(128 << (8 * p) for p in range(6))
    x0 = -np.ldexp(float(X0), -54)
    assert np.ldexp(float(X0), -54) < 1.0 and int(np.ldexp(-x0, 54)) == X0
    n = 64
    X = np.full((3, n), x0)
    B = np.triu(np.full((n, n), x0))
    Y = split_product(X, B)
    exact = [sum(Fraction(x0) * Fraction(x0) for _ in range(k + 1)) for k in range(n)]
    # the final rounding to FP64 of results up to 64 x0^2 dominates
    for k in range(n):
        assert abs(Fraction(float(Y[0, k])) - exact[k]) <= Fraction(2) ** -52 * abs(exact[k])


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


def test_gram_recombination_bounds():
    """The Gram's read-back (events of up to 1024 rows, 7-bit digits): every region is an exact
    FP32 integer (|D| <= 2^24; |D_1| <= 2^22, |D_0| <= 2^21 because leading digits are at most
    32), the high word D_0 2^9 + D_1 2^2 fits in 32 bits, and the int64 result is T / 256 to
    within one unit, for random and extreme region values."""
    rng = synthetic.rng(21)
    bounds = [2 ** 21, 2 ** 22] + [2 ** 24] * 6
    # extreme digit products reach the bounds: 4 pairs x 1024 rows x 64 x 64
    assert 4 * 1024 * 64 * 64 == 2 ** 24 and 1024 * 32 * 64 == 2 ** 21 and 1024 * 64 * 64 == 2 ** 22
    for trial in range(2000):
        if trial < 16:
            D = [int(b) * (1 if (trial >> (i % 4)) & 1 else -1) for i, b in enumerate(bounds)]
        else:
            D = [int(rng.integers(-b, b + 1)) for b in bounds]
        for d in D:
            assert float(np.float32(d)) == d
        hw = D[0] * 512 + D[1] * 4
        assert -2 ** 31 <= hw < 2 ** 31
        lw = ((D[6] * 128 + D[7]) >> 8) + D[5] * 64 + D[4] * 2 ** 13 + D[3] * 2 ** 20 + D[2] * 2 ** 27
        t = (lw + (hw << 32)) % 2 ** 64
        t = t - 2 ** 64 if t >= 2 ** 63 else t
        exact = sum(D[g] * 2 ** (7 * (7 - g)) for g in range(8))
        assert abs(t * 256 - exact) < 256


# ---- the sketch GEMM: dense B, K in chunks of 64 with per-chunk scales ---------------------

def split_gemm(A, B, chunk=64):
    """C = A B the way the sketch kernel forms it: for each chunk of 64 along K, row scales of
    A's chunk and column scales of B's chunk, byte digits, slice pairs s + t <= 7 in eight
    regions, integer recombination; the chunks' FP64 values summed in order."""
    M, K = A.shape
    n = B.shape[1]
    C = np.zeros((M, n))
    for c0 in range(0, K, chunk):
        a, b = A[:, c0:c0 + chunk], B[c0:c0 + chunk]
        E, F = scale_exp(a, 1), scale_exp(b, 0)
        da, db = digits(fix54(a, E)), digits(fix54(b, F))
        D = []
        for g in range(8):
            acc = np.zeros((M, n), dtype=np.int64)
            for s in range(7):
                if 0 <= g - s < 7:
                    acc += da[s] @ db[g - s]
            assert np.abs(acc).max() <= (2 ** 22 if g <= 4 else 2 ** 23 - 1)
            D.append(acc)
        C += np.ldexp(recombine(D).astype(np.float64), E + F - 56)
    return C


def test_sketch_split_gemm_error_per_chunk():
    # each term of a chunk errs by less than 2^-51 of (largest |a| in the chunk's row) x
    # (largest |b| in the chunk's column), whatever the spread inside the chunk: truncation of
    # both factors (2^-53 each, the scales being below twice the maxima), the dropped digit
    # pairs and the recombination's last unit; checked exactly
    rng = synthetic.rng(31)
    M, K, n = 6, 150, 5  # a ragged last chunk
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-25, 25, (1, K)))
    B = rng.standard_normal((K, n)) * np.exp(rng.uniform(-25, 25, (K, 1)))
    A[2] = 0.0
    C = split_gemm(A, B)
    for i in range(M):
        for j in range(n):
            exact = sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K))
            allowed = Fraction(0)
            for c0 in range(0, K, 64):
                L = min(64, K - c0)
                amax = np.abs(A[i, c0:c0 + 64]).max()
                bmax = np.abs(B[c0:c0 + 64, j]).max()
                allowed += L * Fraction(float(amax)) * Fraction(float(bmax)) * Fraction(2) ** -51
            # plus the roundings of the chunk values and of their FP64 sum
            allowed += 4 * Fraction(2) ** -53 * sum(abs(Fraction(float(A[i, k])) * Fraction(float(B[k, j])))
                                                    for k in range(K))
            assert abs(Fraction(float(C[i, j])) - exact) <= allowed
    assert np.all(C[2] == 0.0)


def test_sketch_split_gemm_exact_for_signs_times_integers():
    # +-1 entries of A (and the identity) with integer B: every chunk value is an exact
    # integer, so the result equals A B exactly (the GPU test's bit-exact case)
    rng = synthetic.rng(32)
    K, n = 200, 7
    A = np.where(rng.random((9, K)) < 0.5, -1.0, 1.0)
    B = rng.integers(-2 ** 20, 2 ** 20, (K, n)).astype(np.float64)
    np.testing.assert_array_equal(split_gemm(A, B), A @ B)
    I = np.eye(K)[:70]
    np.testing.assert_array_equal(split_gemm(I, B), B[:70])


def test_sketch_split_gemm_at_the_digit_extremes():
    # a full chunk of entries whose lower digits are all -128 on both sides: the region sums
    # reach the recombination's bounds (asserted inside split_gemm) and the result is right
    X0 = 63 * 2 ** 48 + sum(128 << (8 * p) for p in range(6))
    x0 = -np.ldexp(float(X0), -54)
    A = np.full((2, 64), x0)
    B = np.full((64, 3), x0)
    C = split_gemm(A, B)
    exact = 64 * Fraction(x0) * Fraction(x0)
    assert abs(Fraction(float(C[0, 0])) - exact) <= Fraction(2) ** -52 * exact


# ---- the add-to-reference epilogue of the blocked solves (T = V2 - W1 R12 formed as one sum) --
def add_to_reference(ref, t, u0):
    """ref + t 2^u0 as the blocked solves form it: one integer sum at the unit 2^u1, u1 = u0 or
    coarser so that ref (truncated to that unit) needs at most 61 bits, then one rounding to
    FP64 (nearest, as an int64 -> FP64 conversion rounds).  Returns (value, u1, integer sum)."""
    import struct
    b = struct.unpack("<Q", struct.pack("<d", ref))[0]
    ef = (b >> 52) & 0x7FF
    u1 = max(u0, ef - 1023 - 60)
    ts = t >> min(u1 - u0, 63)  # floor, as an arithmetic shift
    sh = ef - 1075 - u1
    mant = (b & ((1 << 52) - 1)) | (1 << 52)
    rf = 0 if ef == 0 else (mant << sh if sh >= 0 else (mant >> -sh if -sh < 63 else 0))
    rf = -rf if b >> 63 else rf
    total = ts + rf
    return float(np.ldexp(float(total), u1)), u1, total


def test_add_to_reference_is_one_rounding_of_the_exact_sum():
    """Against the exact rational ref + t 2^u0, over references from 2^-300 to 2^300 (and zeros,
    subnormals, both signs) and products of up to 62 bits at units that make either term
    dominate: the integer sum fits 63 bits, and the result is within two units 2^u1 (the two
    truncations) plus half an ulp (the one rounding) of the exact sum, a subnormal reference
    counting as zero -- for a dominant reference 2^u1 is 2^-60 of its binade, so the reference
    moves by at most 2^-58 of its magnitude."""
    rng = np.random.default_rng(3)
    for _ in range(4000):
        kind = rng.integers(0, 6)
        if kind == 0:
            ref = 0.0
        elif kind == 1:
            ref = float(rng.choice([-1.0, 1.0]) * np.ldexp(float(rng.uniform(1, 2)), -1040))  # subnormal
        else:
            ref = float(rng.choice([-1.0, 1.0]) * np.ldexp(float(rng.uniform(1, 2)), int(rng.integers(-300, 300))))
        bits = int(rng.integers(0, 63))
        t = int(rng.integers(-(1 << bits), 1 << bits)) if bits else 0
        e_ref = int(np.frexp(ref)[1]) if ref else 0
        u0 = e_ref - int(rng.integers(0, 130))  # the product from far below to far above ref
        val, u1, total = add_to_reference(ref, t, u0)
        assert abs(total) < (1 << 63)
        exact = Fraction(ref) + Fraction(t) * Fraction(2) ** u0
        err = abs(Fraction(val) - exact)
        ulp = Fraction(2) ** (int(np.frexp(val)[1]) - 53) if val else Fraction(0)
        # a subnormal reference counts as zero: at most 2^-1022 more
        assert err <= 2 * Fraction(2) ** u1 + ulp / 2 + Fraction(2) ** -1022, (ref, t, u0)
        if abs(ref) >= 2.0 ** -1022 and u1 > u0:  # a dominant (normal) reference, relative to itself
            assert 2 * Fraction(2) ** u1 <= Fraction(abs(ref)) * Fraction(2) ** -58


def test_six_digit_products_meet_the_pair_arithmetic_bound():
    """RANDQR_F32X2's solves keep six of X's seven digits: each term then loses less than one
    unit of the dropped digit, 2^(E - 46) of the row scale, so the product's error stays below
    2^-42 of the scale product over 64 terms -- the accuracy of FP32-pair arithmetic -- while
    seven digits stay below 2^-50."""
    rng = synthetic.rng(5)
    m, n = 24, 64
    X = rng.standard_normal((m, n)) * np.exp(rng.uniform(-10, 10, (m, 1)))
    B = np.triu(rng.standard_normal((n, n)) * np.exp(rng.uniform(-10, 10, (1, n))))
    E, F = scale_exp(X, 1), scale_exp(B, 0)
    worst = {}
    for nda in (6, 7):
        Y = split_product(X, B, nda=nda)
        w = 0.0
        for i in range(m):
            for k in range(0, n, 5):
                exact = sum(Fraction(float(X[i, j])) * Fraction(float(B[j, k])) for j in range(n))
                w = max(w, float(abs(Fraction(float(Y[i, k])) - exact) / Fraction(2) ** int(E[i, 0] + F[0, k])))
        worst[nda] = w
    assert worst[7] <= 2.0 ** -50, worst
    assert 2.0 ** -52 < worst[6] <= 2.0 ** -42, worst  # coarser than seven digits, within the bound
