/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for rand_cholQR.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant generator with the CUDA library; each side writes
 * the two counter-based generators (splitmix64, Philox4x64-10) from their published
 * definitions.
 *
 * Method: Higgins, Szyld, Boman & Yamazaki, "Analysis of Randomized Householder-Cholesky
 * QR Factorization with Multisketching" (arXiv 2309.05868).  The paper writes the input
 * as V in R^{n x m} (n rows); this file uses the opposite letters: V is m x n, m rows,
 * n columns, sketch sizes s1 (paper p1) and s2 (paper p2).
 *
 * Everything is FP64, row-major, computed in the order the paper's algorithms state,
 * with no blocking, fusion or reordering.  Build: -O2 -fno-fast-math -ffp-contract=off
 * (no FMA contraction, so every product and sum rounds exactly once).
 *
 * Return codes shared with the Python wrapper:
 *    0  ok
 *   -2  Cholesky breakdown (non-positive pivot); *info holds the 1-based pivot
 *   -3  zero diagonal in a triangular factor from Householder QR (rank deficiency)
 *   -5  allocation failure
 *
 * Parity pins: every function below is checked in tests/test_oracle_*.py against
 * something other than itself (library routines, closed forms, invariants the paper
 * states, brute force on tiny inputs).  Functions without such a pin say so.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void orc_cs_hash_at(uint64_t seed, int64_t row0, int64_t m, int64_t s1, int32_t *bucket,
                    int8_t *sign);
int orc_countsketch_rows(const double *V, int64_t m, int64_t n, int64_t ldv, int64_t s1,
                         uint64_t seed, int64_t row0, double *W1);

#define ORC_OK 0
#define ORC_NOT_SPD (-2)
#define ORC_RANK (-3)
#define ORC_NOMEM (-5)

/* ------------------------------------------------------------------------------------
 * Random numbers the method draws.
 * ---------------------------------------------------------------------------------- */

/* splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014; constants as in Vigna's
 * public-domain splitmix64): one step of the generator whose state is x. */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* CountSketch column i of S1 (Sec. 3, the sparse embedding with one +-1 per column whose
 * row and sign are uniform): x = splitmix64(seed XOR splitmix64(i)); row (bucket) =
 * floor(hi32(x) * s1 / 2^32); sign = -1 if the low bit of x is set, else +1. */
void orc_cs_hash(uint64_t seed, int64_t m, int64_t s1, int32_t *bucket, int8_t *sign) {
  orc_cs_hash_at(seed, 0, m, s1, bucket, sign);
}

/* The same columns row0 .. row0 + m - 1 of S1: a row block V_k of a matrix split by rows
 * (Sec. 4.1, the distributed sketch) is sketched with the S1 columns of its global rows. */
void orc_cs_hash_at(uint64_t seed, int64_t row0, int64_t m, int64_t s1, int32_t *bucket,
                    int8_t *sign) {
  for (int64_t i = 0; i < m; ++i) {
    uint64_t x = orc_splitmix64(seed ^ orc_splitmix64((uint64_t)(row0 + i)));
    bucket[i] = (int32_t)(((x >> 32) * (uint64_t)s1) >> 32);
    sign[i] = (x & 1ULL) ? (int8_t)-1 : (int8_t)1;
  }
}

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC 2011): ten rounds of the 4x64 Philox
 * S-box with the published multipliers and Weyl key increments. */
void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c0, &hi0, &lo0);
    mulhilo64(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Gaussian sketch S2 in R^{s2 x s1} with entries N(0, 1/s2) (Sec. 3: S = G / sqrt(p)).
 * Entry (r, c) takes Philox4x64-10 at counter (r*s1 + c, 0, 0, 0) with key (seed, 0);
 * u1 = (x0>>11 + 1) 2^-53 in (0,1], u2 = (x1>>11) 2^-53 in [0,1), and the Box-Muller
 * transform z = sqrt(-2 ln u1) cos(2 pi u2). */
void orc_gauss_sketch(uint64_t seed, int64_t s2, int64_t s1, double *S2) {
  const double two_m53 = 1.1102230246251565404e-16; /* 2^-53 */
  const double two_pi = 6.283185307179586476925286766559;
  const double scale = 1.0 / sqrt((double)s2);
  for (int64_t r = 0; r < s2; ++r) {
    for (int64_t c = 0; c < s1; ++c) {
      uint64_t ctr[4] = {(uint64_t)(r * s1 + c), 0, 0, 0}, key[2] = {seed, 0}, x[4];
      orc_philox4x64_10(ctr, key, x);
      double u1 = (double)((x[0] >> 11) + 1) * two_m53;
      double u2 = (double)(x[1] >> 11) * two_m53;
      double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
      S2[r * s1 + c] = z * scale;
    }
  }
}

/* Rademacher sketch S2 in R^{s2 x s1} with entries +-1/sqrt(s2) (the paper's alternative
 * dense sketch, Sec. 7): entry (r, c) is -1/sqrt(s2) when bit (c mod 64) of
 * splitmix64(seed XOR splitmix64(r * ceil(s1 / 64) + floor(c / 64))) is set, else +1/sqrt(s2). */
void orc_rademacher_sketch(uint64_t seed, int64_t s2, int64_t s1, double *S2) {
  const double scale = 1.0 / sqrt((double)s2);
  const int64_t nw = (s1 + 63) / 64;
  for (int64_t r = 0; r < s2; ++r) {
    for (int64_t c = 0; c < s1; ++c) {
      uint64_t word = orc_splitmix64(seed ^ orc_splitmix64((uint64_t)(r * nw + c / 64)));
      S2[r * s1 + c] = ((word >> (c % 64)) & 1ULL) ? -scale : scale;
    }
  }
}

/* ------------------------------------------------------------------------------------
 * Algorithm 1 (randQR), step 1: W = S2 S1 V, split as W1 = S1 V then W = S2 W1 (Sec. 4.2).
 * ---------------------------------------------------------------------------------- */

/* W1 = S1 V: W1 (s1 x n) starts at zero, and each row i of V is added, with its sign, to
 * row bucket(i) of W1, rows taken in ascending i. */
int orc_countsketch(const double *V, int64_t m, int64_t n, int64_t ldv, int64_t s1,
                    uint64_t seed, double *W1) {
  return orc_countsketch_rows(V, m, n, ldv, s1, seed, 0, W1);
}

/* W1_k = S1_k V_k for a row block whose first row is global row row0 (Sec. 4.1): the S1
 * columns are those of the global rows, so that S1 V = sum_k S1_k V_k. */
int orc_countsketch_rows(const double *V, int64_t m, int64_t n, int64_t ldv, int64_t s1,
                         uint64_t seed, int64_t row0, double *W1) {
  int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int8_t *sg = (int8_t *)malloc((size_t)(m > 0 ? m : 1));
  if (!b || !sg) { free(b); free(sg); return ORC_NOMEM; }
  orc_cs_hash_at(seed, row0, m, s1, b, sg);
  memset(W1, 0, sizeof(double) * (size_t)(s1 * n));
  for (int64_t i = 0; i < m; ++i) {
    double s = (double)sg[i];
    for (int64_t j = 0; j < n; ++j) W1[(int64_t)b[i] * n + j] += s * V[i * ldv + j];
  }
  free(b); free(sg);
  return ORC_OK;
}

/* C (p x n) = A (p x k) B (k x n), plain triple loop, inner index ascending. */
void orc_gemm(const double *A, const double *B, int64_t p, int64_t k, int64_t n, double *C) {
  for (int64_t i = 0; i < p; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int64_t l = 0; l < k; ++l) acc += A[i * k + l] * B[l * n + j];
      C[i * n + j] = acc;
    }
}

/* ------------------------------------------------------------------------------------
 * Householder QR (Algorithm 1 step 2; Sec. 5.2.2 uses its backward error).
 * LAPACK dgeqr2 recurrence (Golub & Van Loan, Alg. 5.2.1): reflector H_j = I - tau v v^T
 * with v_j = 1 zeroes A[j+1:, j]; the new diagonal is beta = -sign(a_jj) ||A[j:, j]||.
 * ---------------------------------------------------------------------------------- */

/* In place on A (rows x n, row-major, rows >= n).  On return the upper triangle of
 * A[0:n, :] holds R, the strictly-lower part holds v (unit leading entry implied), tau[j]
 * holds the reflector scalars. */
static void householder_inplace(double *A, int64_t rows, int64_t n, double *tau) {
  for (int64_t j = 0; j < n; ++j) {
    double sigma = 0.0;
    for (int64_t i = j + 1; i < rows; ++i) sigma += A[i * n + j] * A[i * n + j];
    double x0 = A[j * n + j];
    if (sigma == 0.0) { tau[j] = 0.0; continue; } /* column already reduced */
    double alpha = sqrt(x0 * x0 + sigma);
    double beta = (x0 >= 0.0) ? -alpha : alpha;
    double v0 = x0 - beta;
    tau[j] = (beta - x0) / beta;
    for (int64_t i = j + 1; i < rows; ++i) A[i * n + j] /= v0;
    A[j * n + j] = beta;
    for (int64_t k = j + 1; k < n; ++k) {
      double w = A[j * n + k];
      for (int64_t i = j + 1; i < rows; ++i) w += A[i * n + j] * A[i * n + k];
      w *= tau[j];
      A[j * n + k] -= w;
      for (int64_t i = j + 1; i < rows; ++i) A[i * n + k] -= A[i * n + j] * w;
    }
  }
}

/* R factor only (Q is not formed), normalised to a positive diagonal by flipping the sign
 * of each row of R whose diagonal is negative; the matching column flip of the implicit
 * orthogonal factor leaves Q_tmp R unchanged.  Returns ORC_RANK if a diagonal is zero. */
int orc_hhqr_r(const double *A_in, int64_t rows, int64_t n, double *R) {
  double *A = (double *)malloc(sizeof(double) * (size_t)(rows * n));
  double *tau = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!A || !tau) { free(A); free(tau); return ORC_NOMEM; }
  memcpy(A, A_in, sizeof(double) * (size_t)(rows * n));
  householder_inplace(A, rows, n, tau);
  int status = ORC_OK;
  for (int64_t i = 0; i < n; ++i) {
    double sg = (A[i * n + i] < 0.0) ? -1.0 : 1.0;
    if (A[i * n + i] == 0.0) status = ORC_RANK;
    for (int64_t j = 0; j < n; ++j) R[i * n + j] = (j >= i) ? sg * A[i * n + j] : 0.0;
  }
  free(A); free(tau);
  return status;
}

/* Full Householder QR with explicit thin Q (m x n): Q = H_0 H_1 ... H_{n-1} [I_n; 0], the
 * comparison method of Sec. 6 (dgeqrf + dorgqr).  Positive diagonal as above. */
int orc_householder_qr(const double *V, int64_t m, int64_t n, int64_t ldv, double *Q, double *R) {
  double *A = (double *)malloc(sizeof(double) * (size_t)(m * n));
  double *tau = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!A || !tau) { free(A); free(tau); return ORC_NOMEM; }
  for (int64_t i = 0; i < m; ++i) memcpy(A + i * n, V + i * ldv, sizeof(double) * (size_t)n);
  householder_inplace(A, m, n, tau);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) Q[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int64_t j = n - 1; j >= 0; --j) {
    if (tau[j] == 0.0) continue;
    for (int64_t c = 0; c < n; ++c) {
      double w = Q[j * n + c];
      for (int64_t i = j + 1; i < m; ++i) w += A[i * n + j] * Q[i * n + c];
      w *= tau[j];
      Q[j * n + c] -= w;
      for (int64_t i = j + 1; i < m; ++i) Q[i * n + c] -= A[i * n + j] * w;
    }
  }
  int status = ORC_OK;
  for (int64_t i = 0; i < n; ++i) {
    double sg = (A[i * n + i] < 0.0) ? -1.0 : 1.0;
    if (A[i * n + i] == 0.0) status = ORC_RANK;
    for (int64_t j = 0; j < n; ++j) R[i * n + j] = (j >= i) ? sg * A[i * n + j] : 0.0;
    for (int64_t r = 0; r < m; ++r) Q[r * n + i] *= sg;
  }
  free(A); free(tau);
  return status;
}

/* ------------------------------------------------------------------------------------
 * Triangular solve, Gram, Cholesky, product (Algorithms 1-4).
 * ---------------------------------------------------------------------------------- */

/* W = V R^{-1}, R upper triangular (n x n): per row, forward substitution
 * w_j = (v_j - sum_{k<j} w_k r_kj) / r_jj with k ascending (the row-wise solve whose
 * backward error is the model of Sec. 5.2.3, eq. triSys). */
void orc_trsm(const double *V, int64_t m, int64_t n, int64_t ldv, const double *R, double *W,
              int64_t ldw) {
  for (int64_t i = 0; i < m; ++i) {
    const double *v = V + i * ldv;
    double *w = W + i * ldw;
    for (int64_t j = 0; j < n; ++j) {
      double s = v[j];
      for (int64_t k = 0; k < j; ++k) s -= w[k] * R[k * n + j];
      w[j] = s / R[j * n + j];
    }
  }
}

/* G = W^T W (n x n), rows summed in ascending order (Algorithm 2 step 1). */
void orc_gram(const double *W, int64_t m, int64_t n, int64_t ldw, double *G) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t k = 0; k < n; ++k) {
      double acc = 0.0;
      for (int64_t i = 0; i < m; ++i) acc += W[i * ldw + j] * W[i * ldw + k];
      G[j * n + k] = acc;
    }
}

/* Upper Cholesky G = R^T R (Algorithm 2 step 2), Cholesky-Banachiewicz order.  On a
 * non-positive (or NaN) pivot returns ORC_NOT_SPD with *info = 1-based pivot index. */
int orc_chol(const double *G, int64_t n, double *R, int32_t *info) {
  memset(R, 0, sizeof(double) * (size_t)(n * n));
  if (info) *info = 0;
  for (int64_t j = 0; j < n; ++j) {
    double d = G[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= R[k * n + j] * R[k * n + j];
    if (!(d > 0.0)) { if (info) *info = (int32_t)(j + 1); return ORC_NOT_SPD; }
    double rjj = sqrt(d);
    R[j * n + j] = rjj;
    for (int64_t l = j + 1; l < n; ++l) {
      double s = G[j * n + l];
      for (int64_t k = 0; k < j; ++k) s -= R[k * n + j] * R[k * n + l];
      R[j * n + l] = s / rjj;
    }
  }
  return ORC_OK;
}

/* C = A B for upper-triangular A, B (n x n) (Algorithm 3 step 3: R = R1 R0). */
void orc_trmm(const double *A, const double *B, int64_t n, double *C) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int64_t k = i; k <= j; ++k) acc += A[i * n + k] * B[k * n + j];
      C[i * n + j] = (j >= i) ? acc : 0.0;
    }
}

/* ------------------------------------------------------------------------------------
 * The algorithms.
 * ---------------------------------------------------------------------------------- */

/* Algorithm 1, randQR: Ws = S2 S1 V; R0 = R(hhqr(Ws)); Q0 = V R0^{-1}.  If S2 is NULL it
 * is generated from seed+1 by orc_gauss_sketch; the CountSketch uses seed.  Optional
 * outputs W1 (s1 x n) and Ws (s2 x n) may be NULL. */
int orc_randqr(const double *V, int64_t m, int64_t n, int64_t ldv, int64_t s1, int64_t s2,
               uint64_t seed, const double *S2_in, double *Q0, double *R0, double *W1_out,
               double *Ws_out) {
  double *W1 = (double *)malloc(sizeof(double) * (size_t)(s1 * n));
  double *Ws = (double *)malloc(sizeof(double) * (size_t)(s2 * n));
  double *S2g = S2_in ? NULL : (double *)malloc(sizeof(double) * (size_t)(s2 * s1));
  if (!W1 || !Ws || (!S2_in && !S2g)) { free(W1); free(Ws); free(S2g); return ORC_NOMEM; }
  const double *S2 = S2_in;
  if (!S2) { orc_gauss_sketch(seed + 1, s2, s1, S2g); S2 = S2g; }
  int st = orc_countsketch(V, m, n, ldv, s1, seed, W1);
  if (st == ORC_OK) {
    orc_gemm(S2, W1, s2, s1, n, Ws);
    st = orc_hhqr_r(Ws, s2, n, R0);
  }
  if (st == ORC_OK) orc_trsm(V, m, n, ldv, R0, Q0, n);
  if (W1_out) memcpy(W1_out, W1, sizeof(double) * (size_t)(s1 * n));
  if (Ws_out) memcpy(Ws_out, Ws, sizeof(double) * (size_t)(s2 * n));
  free(W1); free(Ws); free(S2g);
  return st;
}

/* Algorithm 2, cholQR: G = V^T V; R = chol(G); Q = V R^{-1}. */
int orc_cholqr(const double *V, int64_t m, int64_t n, int64_t ldv, double *Q, double *R,
               int32_t *info) {
  double *G = (double *)malloc(sizeof(double) * (size_t)(n * n));
  if (!G) return ORC_NOMEM;
  orc_gram(V, m, n, ldv, G);
  int st = orc_chol(G, n, R, info);
  if (st == ORC_OK) orc_trsm(V, m, n, ldv, R, Q, n);
  free(G);
  return st;
}

/* Algorithm 3, rand_cholQR: [Q0, R0] = randQR(V); [Q, R1] = cholQR(Q0); R = R1 R0.
 * Optional outputs Rs (= R0) and Rc (= R1) may be NULL. */
int orc_rand_cholqr(const double *V, int64_t m, int64_t n, int64_t ldv, int64_t s1, int64_t s2,
                    uint64_t seed, const double *S2, double *Q, double *R, double *Rs_out,
                    double *Rc_out, int32_t *info) {
  double *Q0 = (double *)malloc(sizeof(double) * (size_t)(m * n));
  double *R0 = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *R1 = (double *)malloc(sizeof(double) * (size_t)(n * n));
  if (!Q0 || !R0 || !R1) { free(Q0); free(R0); free(R1); return ORC_NOMEM; }
  if (info) *info = 0;
  int st = orc_randqr(V, m, n, ldv, s1, s2, seed, S2, Q0, R0, NULL, NULL);
  if (st == ORC_OK) st = orc_cholqr(Q0, m, n, n, Q, R1, info);
  if (st == ORC_OK) orc_trmm(R1, R0, n, R);
  if (Rs_out) memcpy(Rs_out, R0, sizeof(double) * (size_t)(n * n));
  if (Rc_out && st == ORC_OK) memcpy(Rc_out, R1, sizeof(double) * (size_t)(n * n));
  free(Q0); free(R0); free(R1);
  return st;
}

/* Algorithm 4, cholQR2: [Q0, R0] = cholQR(V); [Q, R1] = cholQR(Q0); R = R1 R0. */
int orc_cholqr2(const double *V, int64_t m, int64_t n, int64_t ldv, double *Q, double *R,
                int32_t *info) {
  double *Q0 = (double *)malloc(sizeof(double) * (size_t)(m * n));
  double *R0 = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *R1 = (double *)malloc(sizeof(double) * (size_t)(n * n));
  if (!Q0 || !R0 || !R1) { free(Q0); free(R0); free(R1); return ORC_NOMEM; }
  int st = orc_cholqr(V, m, n, ldv, Q0, R0, info);
  if (st == ORC_OK) st = orc_cholqr(Q0, m, n, n, Q, R1, info);
  if (st == ORC_OK) orc_trmm(R1, R0, n, R);
  free(Q0); free(R0); free(R1);
  return st;
}

/* Shifted CholeskyQR3.  The paper cites but never states it; this follows the cited
 * method (Fukaya, Kannan, Nakatsukasa, Yamamoto & Yanagisawa, SISC 2020): shift
 * s = 11 (m n + n (n+1)) u ||V||_F^2 with u = 2^-53; G = V^T V + s I; R0 = chol(G);
 * Q0 = V R0^{-1}; [Q, R12] = cholQR2(Q0); R = R12 R0.  R0_out (may be NULL) receives the
 * shifted pass's factor, so that R0^T R0 - V^T V (= s I up to rounding) can be checked
 * against the cited shift. */
int orc_scholqr3(const double *V, int64_t m, int64_t n, int64_t ldv, double *Q, double *R,
                 double *R0_out, int32_t *info) {
  double *G = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *R0 = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *R12 = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *Q0 = (double *)malloc(sizeof(double) * (size_t)(m * n));
  if (!G || !R0 || !R12 || !Q0) { free(G); free(R0); free(R12); free(Q0); return ORC_NOMEM; }
  const double u = 1.1102230246251565404e-16;
  double fro2 = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) fro2 += V[i * ldv + j] * V[i * ldv + j];
  double shift = 11.0 * ((double)m * (double)n + (double)n * (double)(n + 1)) * u * fro2;
  orc_gram(V, m, n, ldv, G);
  for (int64_t j = 0; j < n; ++j) G[j * n + j] += shift;
  int st = orc_chol(G, n, R0, info);
  if (st == ORC_OK) {
    orc_trsm(V, m, n, ldv, R0, Q0, n);
    st = orc_cholqr2(Q0, m, n, n, Q, R12, info);
  }
  if (st == ORC_OK) orc_trmm(R12, R0, n, R);
  if (R0_out) memcpy(R0_out, R0, sizeof(double) * (size_t)(n * n));
  free(G); free(R0); free(R12); free(Q0);
  return st;
}

/* ------------------------------------------------------------------------------------
 * Error measures of Sec. 6.3 (and the 2-norm the stability theorems bound).
 * ---------------------------------------------------------------------------------- */

/* Largest |eigenvalue| of a symmetric n x n matrix by cyclic Jacobi rotations
 * (Golub & Van Loan Alg. 8.5.3), used for the spectral norm of Q^T Q - I. */
double orc_sym_absmax_eig(const double *A_in, int64_t n) {
  double *A = (double *)malloc(sizeof(double) * (size_t)(n * n));
  if (!A) return NAN;
  memcpy(A, A_in, sizeof(double) * (size_t)(n * n));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int64_t p = 0; p < n; ++p)
      for (int64_t q = 0; q < n; ++q) {
        tot += A[p * n + q] * A[p * n + q];
        if (p != q) off += A[p * n + q] * A[p * n + q];
      }
    if (off == 0.0 || off <= 1e-30 * tot) break;
    for (int64_t p = 0; p < n - 1; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int64_t k = 0; k < n; ++k) { /* columns p, q */
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int64_t k = 0; k < n; ++k) { /* rows p, q */
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  double mx = 0.0;
  for (int64_t i = 0; i < n; ++i) if (fabs(A[i * n + i]) > mx) mx = fabs(A[i * n + i]);
  free(A);
  return mx;
}

/* ||I - Q^T Q||_2 and ||I - Q^T Q||_F. */
void orc_orth_err(const double *Q, int64_t m, int64_t n, int64_t ldq, double *e2, double *eF) {
  double *G = (double *)malloc(sizeof(double) * (size_t)(n * n));
  if (!G) { *e2 = NAN; *eF = NAN; return; }
  orc_gram(Q, m, n, ldq, G);
  double f = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    G[j * n + j] -= 1.0;
    for (int64_t k = 0; k < n; ++k) f += G[j * n + k] * G[j * n + k];
  }
  *eF = sqrt(f);
  *e2 = orc_sym_absmax_eig(G, n);
  free(G);
}

/* ||V - Q R||_F / ||V||_F. */
double orc_resid(const double *V, int64_t m, int64_t n, int64_t ldv, const double *Q,
                 int64_t ldq, const double *R) {
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int64_t k = 0; k <= j; ++k) acc += Q[i * ldq + k] * R[k * n + j];
      double d = V[i * ldv + j] - acc;
      num += d * d;
      den += V[i * ldv + j] * V[i * ldv + j];
    }
  return sqrt(num) / sqrt(den);
}
