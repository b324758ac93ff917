"""Pins for the CPU oracle: each oracle function is checked against something other than
itself -- a library routine it does not call, a closed form, brute force on tiny inputs,
an invariant or bound the paper proves -- chosen so that a dropped term, a wrong sign or
index, or a transposed operand fails at least one test.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U52 = 2.0 ** -52  # the paper's unit roundoff (Sec. 6.1)


def _posdiag(R):
    s = np.sign(np.diag(R))
    s[s == 0] = 1
    return R * s[:, None]


# ---------------------------------------------------------------------------------
# Generators
# ---------------------------------------------------------------------------------
def test_splitmix64_known_answer():
    # First output of splitmix64 started from state 0 (Vigna's public-domain reference).
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF


def test_philox_matches_numpy_bitgenerator():
    # numpy.random.Philox is Philox4x64-10; it increments the counter before each block,
    # so its first block is the Philox function at counter+1.
    for key, ctr in [((5, 7), (0, 0, 0, 0)), ((2**64 - 1, 3), (41, 9, 0, 2**63)),
                     ((123456789, 0), (2**64 - 2, 0, 0, 0))]:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array(ctr, dtype=np.uint64))
        raw = [int(x) for x in bg.random_raw(4)]
        c = list(ctr)
        c[0] = (c[0] + 1) % 2**64
        if c[0] == 0:
            c[1] = (c[1] + 1) % 2**64
        assert oracle.philox4x64_10(c, key) == raw


def test_cs_hash_uniform_and_independent():
    m, s1 = 400_000, 544
    b, s = oracle.cs_hash(0, m, s1)
    assert b.min() >= 0 and b.max() < s1
    assert set(np.unique(s)) == {-1, 1}
    counts = np.bincount(b, minlength=s1)
    chi2 = ((counts - m / s1) ** 2 / (m / s1)).sum()
    # chi-square with s1-1 dof: mean 543, sd ~33; 6 sd band
    assert abs(chi2 - (s1 - 1)) < 6 * math.sqrt(2 * (s1 - 1))
    assert abs(s.astype(np.float64).mean()) < 6 / math.sqrt(m)
    # sign independent of bucket parity
    tab = np.zeros((2, 2))
    np.add.at(tab, (b % 2, (s > 0).astype(int)), 1)
    _, p, _, _ = scipy.stats.chi2_contingency(tab)
    assert p > 1e-4
    b2, _ = oracle.cs_hash(1, m, s1)
    assert (b2 != b).mean() > 0.99


def test_cs_hash_single_bucket_and_large_s1():
    b, _ = oracle.cs_hash(7, 1000, 1)
    assert (b == 0).all()
    b, _ = oracle.cs_hash(7, 100_000, 2**31 - 1)
    assert b.min() >= 0 and b.max() < 2**31 - 1 and len(np.unique(b)) > 99_990


def test_gauss_sketch_distribution():
    s2, s1 = 64, 3000
    S2 = oracle.gauss_sketch(3, s2, s1)
    z = (S2 * math.sqrt(s2)).ravel()
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2 / z.size)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # entries are independent of position: row means and column means look N(0, 1/k)
    assert abs((z.reshape(s2, s1).mean(axis=1) * math.sqrt(s1)).std() - 1) < 0.3


def test_rademacher_sketch_entries_and_moments():
    s2, s1 = 48, 5000
    S2 = oracle.rademacher_sketch(9, s2, s1)
    scale = 1.0 / math.sqrt(s2)
    assert set(np.unique(S2)) == {-scale, scale}
    z = np.sign(S2)
    # unbiased overall, in every bit position of the sign words, and in every row
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    per_bit = np.array([z[:, b::64].mean() for b in range(64)])
    assert np.abs(per_bit).max() < 5 / math.sqrt(z.size / 64)
    assert np.abs(z.mean(axis=1)).max() < 5 / math.sqrt(s1)
    # neighbours uncorrelated: along a row (inside and across sign words) and across rows
    k = (s1 - 1 - 63) // 64 + 1  # pairs (63 + 64 i, 64 + 64 i) inside the row
    for a, b in ((z[:, :-1], z[:, 1:]), (z[:, 63::64][:, :k], z[:, 64::64][:, :k]), (z[:-1], z[1:])):
        assert abs((a * b).mean()) < 5 / math.sqrt(a.size)
    # S2^T S2 has an exact unit diagonal and off-diagonal entries of variance 1/s2
    C = S2.T[:400] @ S2[:, :400]
    np.testing.assert_allclose(np.diag(C), 1.0, rtol=0, atol=1e-15)
    off = C[np.triu_indices(400, 1)]
    assert abs(off.std() * math.sqrt(s2) - 1) < 0.05


def test_rademacher_sketch_embeds_a_subspace():
    # subspace embedding (Sec. 3): singular values of S2 U within 1 +- eps for orthonormal U
    s1, n = 3000, 8
    U, _ = np.linalg.qr(synthetic.rng(4).standard_normal((s1, n)))
    for s2 in (128, 512):
        sv = np.linalg.svd(oracle.rademacher_sketch(2, s2, s1) @ U, compute_uv=False)
        eps = 3.0 * math.sqrt(n / s2)
        assert sv.max() < 1 + eps and sv.min() > 1 - eps


def test_rand_cholqr_with_a_rademacher_sketch(kappa=1e12):
    m, n = 4000, 12
    s1, s2 = 2 * (n * n + n), 4 * n
    V = synthetic.make_v(m, n, kappa, seed=8)
    Q, R = oracle.rand_cholqr(V, s1, s2, 0, S2=oracle.rademacher_sketch(1, s2, s1))
    e2, _ = oracle.orth_err(Q)
    assert e2 <= 1e-13 and oracle.resid(V, Q, R) <= 1e-14
    Qh, Rh = oracle.householder_qr(V)
    np.testing.assert_allclose(R, _posdiag(Rh), rtol=0, atol=1e-12 * kappa * 1e-3 * np.abs(R).max())


def test_gauss_sketch_counter_layout():
    # entry (r, c) depends only on (seed, r*s1 + c): a wider sketch with the same flat
    # counters gives the same numbers up to the 1/sqrt(s2) scaling.
    A = oracle.gauss_sketch(11, 4, 6) * 2.0
    B = oracle.gauss_sketch(11, 1, 24)
    np.testing.assert_array_equal(A.ravel(), B.ravel())


# ---------------------------------------------------------------------------------
# Steps
# ---------------------------------------------------------------------------------
def _dense_s1(b, s, s1):
    S1 = np.zeros((s1, len(b)))
    S1[b, np.arange(len(b))] = s
    return S1


def test_countsketch_vs_explicit_matrix_integer_exact():
    m, n, s1 = 3000, 7, 97
    V = synthetic.integer_matrix(m, n, seed=1)
    b, s = oracle.cs_hash(42, m, s1)
    W1 = oracle.countsketch(V, s1, 42)
    np.testing.assert_array_equal(W1, _dense_s1(b, s, s1) @ V)


def test_countsketch_vs_explicit_matrix_float():
    m, n, s1 = 2000, 5, 60
    V = synthetic.make_v(m, n, 1e6, seed=2)
    b, s = oracle.cs_hash(9, m, s1)
    W1 = oracle.countsketch(V, s1, 9)
    ref = _dense_s1(b, s, s1) @ V
    tol = m * U52 * (np.abs(_dense_s1(b, s, s1)) @ np.abs(V))
    assert (np.abs(W1 - ref) <= tol).all()


def test_cs_hash_at_is_a_window_of_the_global_hash():
    # Sec. 4.1: a row block is sketched with the S1 columns of its global rows.
    b, s = oracle.cs_hash(5, 1000, 313)
    for row0, m in ((0, 10), (1, 999), (517, 200), (999, 1)):
        bk, sk = oracle.cs_hash_at(5, row0, m, 313)
        np.testing.assert_array_equal(bk, b[row0:row0 + m])
        np.testing.assert_array_equal(sk, s[row0:row0 + m])


def test_countsketch_rows_blocks_sum_to_the_global_sketch():
    m, n, s1 = 2500, 6, 41
    V = synthetic.integer_matrix(m, n, seed=3)
    b, s = oracle.cs_hash(11, m, s1)
    S1 = _dense_s1(b, s, s1)
    cuts = [0, 1, 700, 701, 2500]
    total = np.zeros((s1, n))
    for r0, r1 in zip(cuts[:-1], cuts[1:]):
        Wk = oracle.countsketch_rows(V[r0:r1], s1, 11, r0)
        np.testing.assert_array_equal(Wk, S1[:, r0:r1] @ V[r0:r1])
        total += Wk
    np.testing.assert_array_equal(total, S1 @ V)


def test_gemm_vs_numpy():
    A = synthetic.rng(3).standard_normal((33, 129))
    B = synthetic.rng(4).standard_normal((129, 17))
    C = oracle.gemm(A, B)
    tol = 129 * U52 * (np.abs(A) @ np.abs(B))
    assert (np.abs(C - A @ B) <= tol).all()
    # non-square orientation check: (A B)^T = B^T A^T
    np.testing.assert_allclose(oracle.gemm(B.T, A.T), C.T, rtol=0, atol=1e-12)


def test_hhqr_closed_forms():
    np.testing.assert_allclose(oracle.hhqr_r(np.array([[3.0], [4.0]])), [[5.0]], rtol=1e-15)
    np.testing.assert_allclose(oracle.hhqr_r(np.array([[-3.0], [4.0]])), [[5.0]], rtol=1e-15)
    # columns orthogonal: R is diagonal with the column norms
    A = np.array([[1.0, 2.0], [1.0, -2.0], [1.0, 2.0], [1.0, -2.0]])
    np.testing.assert_allclose(oracle.hhqr_r(A), [[2.0, 0.0], [0.0, 4.0]], atol=1e-14)
    # upper-triangular input with positive diagonal is its own R
    T = np.triu(synthetic.rng(5).standard_normal((6, 6))) + 3 * np.eye(6)
    T = _posdiag(T)
    np.testing.assert_allclose(oracle.hhqr_r(T), T, atol=1e-13)


@pytest.mark.parametrize("rows,n,kappa", [(64, 16, 1e2), (300, 40, 1e10), (128, 128, 1e4)])
def test_hhqr_vs_lapack(rows, n, kappa):
    A = synthetic.make_v(rows, n, kappa, seed=rows + n)
    R = oracle.hhqr_r(A)
    assert np.allclose(np.tril(R, -1), 0) and (np.diag(R) > 0).all()
    R_np = _posdiag(np.linalg.qr(A, mode="r"))
    # backward-stable QR: both R are exact for nearby matrices; compare R^T R = A^T A
    np.testing.assert_allclose(R.T @ R, A.T @ A, atol=50 * n * U52 * np.linalg.norm(A) ** 2)
    # and each row of R against LAPACK's, relative to that row's size (rows are graded)
    scale = np.abs(R_np).max(axis=1, keepdims=True)
    assert (np.abs(R - R_np) <= 1e-9 * scale * max(1.0, kappa * 1e-6)).all()


def test_householder_qr_explicit_q():
    V = synthetic.make_v(500, 12, 1e8, seed=6)
    Q, R = oracle.householder_qr(V)
    assert np.linalg.norm(Q.T @ Q - np.eye(12), 2) < 1e-14
    assert np.linalg.norm(V - Q @ R) / np.linalg.norm(V) < 1e-14
    assert (np.diag(R) > 0).all()
    Qn, Rn = np.linalg.qr(V)
    s = np.sign(np.diag(Rn))
    np.testing.assert_allclose(Q[:, :4], (Qn * s)[:, :4], atol=1e-12)


def test_trsm_vs_scipy():
    m, n = 700, 20
    V = synthetic.rng(7).standard_normal((m, n))
    R = np.triu(synthetic.rng(8).standard_normal((n, n))) + 4 * np.eye(n)
    W = oracle.trsm(V, R)
    ref = scipy.linalg.solve_triangular(R, V.T, trans="T", lower=False).T
    np.testing.assert_allclose(W, ref, rtol=1e-12, atol=1e-13)
    # row-wise backward error of forward substitution (eq. triSys): |W R - V| <= g |W||R|
    assert (np.abs(W @ R - V) <= 2 * n * U52 * (np.abs(W) @ np.abs(R))).all()


def test_gram_and_trmm_vs_numpy():
    W = synthetic.rng(9).standard_normal((1000, 9))
    G = oracle.gram(W)
    np.testing.assert_allclose(G, W.T @ W, rtol=1e-13, atol=1e-12)
    np.testing.assert_array_equal(G, G.T)
    A = np.triu(synthetic.rng(10).standard_normal((8, 8)))
    B = np.triu(synthetic.rng(11).standard_normal((8, 8)))
    np.testing.assert_allclose(oracle.trmm(A, B), A @ B, rtol=1e-14, atol=1e-14)


def test_chol_vs_numpy_and_breakdown():
    X = synthetic.rng(12).standard_normal((50, 10))
    G = X.T @ X
    R = oracle.chol(G)
    np.testing.assert_allclose(R, np.linalg.cholesky(G).T, rtol=1e-12, atol=1e-13)
    with pytest.raises(oracle.OracleError) as e:
        oracle.chol(np.diag([1.0, 2.0, -1.0, 4.0]))
    assert e.value.status == -2 and e.value.info == 3
    with pytest.raises(oracle.OracleError) as e:
        oracle.chol(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert e.value.info == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.chol(np.array([[0.0, 0.0], [0.0, 1.0]]))
    assert e.value.info == 1


def test_error_measures_vs_numpy():
    Q = np.linalg.qr(synthetic.rng(13).standard_normal((300, 11)))[0]
    Q = Q @ (np.eye(11) + 1e-6 * np.diag(np.arange(11)))
    e2, eF = oracle.orth_err(Q)
    M = Q.T @ Q - np.eye(11)
    assert abs(e2 - np.abs(np.linalg.eigvalsh(M)).max()) < 1e-12
    assert abs(eF - np.linalg.norm(M, "fro")) < 1e-12
    A = synthetic.rng(14).standard_normal((9, 9))
    A = A + A.T
    assert abs(oracle.sym_absmax_eig(A) - np.abs(np.linalg.eigvalsh(A)).max()) < 1e-12
    V = synthetic.rng(15).standard_normal((40, 6))
    Qv, Rv = np.linalg.qr(V)
    R2 = Rv.copy()
    R2[0, 5] += 1e-3
    ref = np.linalg.norm(V - Qv @ np.triu(R2)) / np.linalg.norm(V)
    assert abs(oracle.resid(V, Qv, R2) - ref) < 1e-15


# ---------------------------------------------------------------------------------
# The algorithms
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8, 1e12, 1e14])
def test_rand_cholqr_invariants(kappa):
    m, n = 3000, 16
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=0)
    Q, R = oracle.rand_cholqr(V, s1, s2, seed=0)
    e2, _ = oracle.orth_err(Q)
    assert e2 <= 1e-12
    assert oracle.resid(V, Q, R) <= 1e-13
    assert np.allclose(np.tril(R, -1), 0) and (np.diag(R) > 0).all()
    # sigma(R) = sigma(V) (known by construction) since Q has orthonormal columns; the
    # small ones to ~u*kappa relative
    sv = np.linalg.svd(R, compute_uv=False)
    ref = synthetic.sigmas(n, kappa)
    assert (np.abs(sv - ref) <= 1e-13 + 1e-13 * kappa * ref).all()


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_rand_cholqr_unique_factor_matches_householder(kappa):
    # With positive diagonals the thin QR factorization is unique: rand_cholQR must
    # agree with Householder QR (oracle's own and LAPACK's) to perturbation-theory size.
    m, n = 2000, 10
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, kappa, seed=4)
    Q, R = oracle.rand_cholqr(V, s1, s2, seed=1)
    Qh, Rh = oracle.householder_qr(V)
    Qn, Rn = np.linalg.qr(V)
    sg = np.sign(np.diag(Rn))
    tol = 1e-13 * kappa
    assert np.abs(Q - Qh).max() < tol and np.abs(Q - Qn * sg).max() < tol
    assert np.abs(R - Rh).max() < tol * np.abs(R).max()


def _embedding_eps(S, U):
    sv = np.linalg.svd(S @ U, compute_uv=False)
    return max(1 - sv.min() ** 2, sv.max() ** 2 - 1)


@pytest.mark.parametrize("kappa", [10.0, 1e3])
def test_randqr_theorems_51_52_53(kappa):
    """Thm 5.1 (S2S1-orthogonality <= 3 delta, ||V - Q0 R0||_2 <= delta/10 sigma_min),
    Thm 5.2 (kappa(Q0) <= 33 / (25 sqrt((1-eL)/(1+eH)) - 3)) and Thm 5.3
    (||Q^T Q - I||_2 <= 5445 (mn + n(n+1)) u / (25 sqrt(.) - 3)^2), with eps1, eps2 the
    measured distortions of S1 on range(V) and of S2 on range(S1 V), delta from eq. delta."""
    n = 8
    s1, s2 = synthetic.paper_multisketch_sizes(n)  # 594, 475 at n = 8
    m = 6000
    seed = 3
    V = synthetic.make_v(m, n, kappa, seed=seed)
    b, sg = oracle.cs_hash(seed, m, s1)
    S1 = _dense_s1(b, sg, s1)
    S2 = oracle.gauss_sketch(seed + 1, s2, s1)
    U = np.linalg.qr(V)[0]
    e1 = _embedding_eps(S1, U)
    e2 = _embedding_eps(S2, np.linalg.qr(S1 @ U)[0])
    eL, eH = e1 + e2 - e1 * e2, e1 + e2 + e1 * e2
    assert eL < 616 / 625 - 9 / 625 * eH, "sketch outside Assumptions 5.1; pick another seed"
    delta = (383 * (math.sqrt(1 + eH) * s2 * n ** 1.5
                    + math.sqrt(n) * np.linalg.norm(S2, 2)
                    * (s1 * math.sqrt(s2) * math.sqrt(1 + e1) + m * np.linalg.norm(S1, "fro")))
             / math.sqrt(1 - eL) * U52 * kappa)
    assert delta <= 1
    Q0, R0, _, _ = oracle.randqr(V, s1, s2, seed)
    SQ = S2 @ (S1 @ Q0)
    assert np.linalg.norm(SQ.T @ SQ - np.eye(n), 2) <= 3 * delta
    assert np.linalg.norm(V - Q0 @ R0, 2) <= delta / 10 * (1 / kappa)
    ratio = math.sqrt((1 - eL) / (1 + eH))
    assert np.linalg.cond(Q0) <= 33 / (25 * ratio - 3)
    Q, R = oracle.rand_cholqr(V, s1, s2, seed)
    bound = 5445 / (25 * ratio - 3) ** 2 * (m * n + n * (n + 1)) * U52
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= bound


def test_randqr_exact_arithmetic_remark():
    # Remark 4.1: S2 S1 Q0 = Q_tmp, the orthonormal Householder factor of S2 S1 V, so in
    # floating point S2 S1 Q0 is orthonormal to O(u kappa); also Q0 R0 = V.
    m, n = 4000, 12
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e5, seed=8)
    Q0, R0, W1, Ws = oracle.randqr(V, s1, s2, seed=5)
    b, sg = oracle.cs_hash(5, m, s1)
    S1 = _dense_s1(b, sg, s1)
    S2 = oracle.gauss_sketch(6, s2, s1)
    np.testing.assert_allclose(Ws, S2 @ (S1 @ V), atol=1e-13)
    SQ = S2 @ (S1 @ Q0)
    assert np.linalg.norm(SQ.T @ SQ - np.eye(n), 2) < 1e-9
    assert np.linalg.norm(V - Q0 @ R0) / np.linalg.norm(V) < 1e-14
    assert np.linalg.cond(Q0) < 10


def test_single_sketch_reduces_to_multisketch_with_identity():
    # Sec. 5.5 remark: a single sketch is the multisketch with S2 = I.
    m, n = 1500, 6
    s1 = 2 * (n * n + n)
    V = synthetic.make_v(m, n, 1e3, seed=9)
    Q0, R0, W1, Ws = oracle.randqr(V, s1, s1, seed=2, S2=np.eye(s1))
    np.testing.assert_array_equal(Ws, W1)
    np.testing.assert_allclose(R0, oracle.hhqr_r(oracle.countsketch(V, s1, 2)), rtol=0, atol=0)


def test_explicit_s2_matches_seeded_s2():
    m, n = 800, 5
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e3, seed=10)
    S2 = oracle.gauss_sketch(8, s2, s1)
    a = oracle.rand_cholqr(V, s1, s2, seed=7)
    b = oracle.rand_cholqr(V, s1, s2, seed=7, S2=S2)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_cholqr2_and_scholqr3_accuracy_and_failure_points():
    """Sec. 6.3: cholQR2 fails past kappa ~ 1e8 and sCholQR3 past ~1e12, while
    rand_cholQR keeps O(u) orthogonality; below those points all three are accurate."""
    consts = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))["failure_points"]
    m, n = 3000, 16
    for algo, ok_kappa, bad_kappa in [(oracle.cholqr2, 1e5, 1e3 * consts["cholqr2"]),
                                      (oracle.scholqr3, 1e9, 1e3 * consts["scholqr3"])]:
        V = synthetic.make_v(m, n, ok_kappa, seed=1)
        Q, R = algo(V)
        assert oracle.orth_err(Q)[0] < 1e-13 and oracle.resid(V, Q, R) < 1e-14
        V = synthetic.make_v(m, n, bad_kappa, seed=1)
        try:
            Q, R = algo(V)
            failed = oracle.orth_err(Q)[0] > 1e-6 or not np.isfinite(Q).all()
        except oracle.OracleError as e:
            failed = e.status == -2
        assert failed, algo.__name__
    s1, s2 = synthetic.default_sketch_sizes(n)
    V = synthetic.make_v(m, n, 1e15, seed=1)
    Q, R = oracle.rand_cholqr(V, s1, s2, seed=0)
    assert oracle.orth_err(Q)[0] < 1e-12


def test_cholqr_plain_is_one_pass():
    V = synthetic.make_v(500, 6, 10.0, seed=12)
    Q, R = oracle.cholqr(V)
    np.testing.assert_allclose(R.T @ R, V.T @ V, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(Q @ R, V, atol=1e-14)


def test_paper_printed_constants():
    c = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    e = c["multisketch_eps"]
    eL = e["eps1"] + e["eps2"] - e["eps1"] * e["eps2"]
    eH = e["eps1"] + e["eps2"] + e["eps1"] * e["eps2"]
    assert round(eL, 4) == e["eps_L"] and round(eH, 4) == e["eps_H"]
    num = 2 * 11 * 55**2 * 3**2 + 55**2 * 3**2 + 24 * 6 * 25 * 11 * 55 * 3 + 6**2 * 25**2 * 11**2
    assert num / (11**2 * 55**2 * 3**2) == c["thm51_constant"]["value"]
    assert abs(c["assumption_ratio"]["bound_sq"] - 625 / 9) < 1e-12
    # the multisketch in the paper's experiment satisfies Assumptions 5.1's eps condition
    assert eL < 616 / 625 - 9 / 625 * eH


def test_scholqr3_shift_is_the_cited_shift():
    """The shifted pass of sCholQR3 factors V^T V + s I with the cited method's shift
    s = 11 (m n + n (n+1)) u ||V||_F^2, u = 2^-53 (Fukaya et al., SISC 2020).  On V = c U
    with orthonormal U (||V||_F^2 = n c^2 to rounding), R0^T R0 - V^T V must be s I to
    within the Cholesky's O(u) backward error: a coefficient of 1 instead of 11, u = 2^-52,
    or the shift on ||V||_2 instead of ||V||_F^2 all miss by a factor of 2 or more."""
    m, n = 2000, 8
    U = np.linalg.qr(synthetic.rng(5).standard_normal((m, n)))[0]
    for c in (1.0, 2.0 ** -3, 2.0 ** 5):
        V = c * U
        _, _, R0 = oracle.scholqr3(V, return_r0=True)
        D = R0.T @ R0 - V.T @ V
        s = 11.0 * (m * n + n * (n + 1)) * 2.0 ** -53 * (n * c * c)
        assert np.abs(np.diag(D) / s - 1.0).max() < 1e-3
        assert np.abs(D - np.diag(np.diag(D))).max() < 1e-3 * s


def test_scholqr3_kappa_sweep():
    """sCholQR3 past CholeskyQR2's limit: with the shift, the shifted pass succeeds at any
    kappa and Q0 = V R0^{-1} has kappa(Q0) ~ sqrt(s) kappa(V), so CholeskyQR2 of Q0 holds
    O(u) orthogonality while that stays below ~u^{-1/2} (here up to 1e13) and breaks down
    past it (1e14, 1e15) -- the failure point Sec. 6.3 reports near 1e12-1e15.  Without the
    shift the first Cholesky would already fail at 1e12 (kappa(V^T V) = 1e24 > 1/u)."""
    m, n = 3000, 16
    for kappa in (1e12, 1e13):
        V = synthetic.make_v(m, n, kappa, seed=1)
        Q, R = oracle.scholqr3(V)
        assert oracle.orth_err(Q)[0] < 1e-13 and oracle.resid(V, Q, R) < 1e-14
        with pytest.raises(oracle.OracleError) as e:  # no shift: plain CholeskyQR2 fails
            oracle.cholqr2(V)
        assert e.value.status == -2
    for kappa in (1e14, 1e15):
        V = synthetic.make_v(m, n, kappa, seed=1)
        with pytest.raises(oracle.OracleError) as e:
            oracle.scholqr3(V)
        assert e.value.status == -2
