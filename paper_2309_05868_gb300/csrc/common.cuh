// common.cuh -- device helpers and the context shared by the librandqr translation units.
//
// Counter-based generators are written here from their published definitions
// (splitmix64: Steele, Lea & Flood 2014; Philox4x64-10: Salmon et al. 2011); nothing is
// shared with the CPU checker.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/randqr.h"

namespace rq {

// ---------------------------------------------------------------------------------------
// Device status word.  The first kernel that meets a numerical failure records
// (code, info, stage) with an atomicCAS on code; every kernel checks it on entry and
// returns at once if it is set, so a failed factorization drains without faulting.
// ---------------------------------------------------------------------------------------
struct DevStatus {
  int32_t code;        // randqr_status (0 = ok)
  int32_t info;        // 1-based failing pivot
  int32_t stage;       // which factorization stage failed
  int32_t wait_limit;  // 0: each wait's default bound; k + 1: k polls (randqr_set_wait_limit)
  double dmin, dmax;   // min / max diagonal of the first triangular factor
};

__device__ __forceinline__ bool status_failed(const DevStatus *st) {
  return *(volatile const int32_t *)&st->code != 0;
}

// The poll bound of a kernel's waits: its default unless the context set one.
__device__ __forceinline__ int wait_bound(const DevStatus *st, int dflt) {
  const int v = st->wait_limit;
  return v > 0 ? v - 1 : dflt;
}

__device__ __forceinline__ void status_fail(DevStatus *st, int32_t code, int32_t info,
                                            int32_t stage) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->info = info;
    st->stage = stage;
  }
}

// ---------------------------------------------------------------------------------------
// splitmix64 output function and the CountSketch hash built on it.
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Row i of V goes to bucket floor(hi32(x) * s1 / 2^32) with sign bit (x & 1), where
// x = splitmix64(seed ^ splitmix64(i)).  Returned as bucket | (signbit << 31).
__device__ __forceinline__ uint32_t cs_bucket_sign(uint64_t seed, uint64_t i, uint32_t s1) {
  uint64_t x = splitmix64(seed ^ splitmix64(i));
  uint32_t b = (uint32_t)(((x >> 32) * (uint64_t)s1) >> 32);
  return b | ((uint32_t)(x & 1ULL) << 31);
}

// ---------------------------------------------------------------------------------------
// Philox4x64-10.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
    uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

// Flip the sign of a double by its bit pattern (no FP64 pipe instruction).
__device__ __forceinline__ double flip_if(double v, uint32_t signbit) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)signbit << 63));
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

// Packed storage of an n x n upper-triangular matrix, column by column:
// element (k, j), k <= j, lives at j (j + 1) / 2 + k.
__host__ __device__ __forceinline__ int tri_idx(int k, int j) { return j * (j + 1) / 2 + k; }

}  // namespace rq

// ---------------------------------------------------------------------------------------
// Context.
// ---------------------------------------------------------------------------------------
struct randqr_ctx {
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;
  // one growable workspace slab
  void *ws = nullptr;
  size_t ws_bytes = 0;
  // device staging of randqr_factor_host (V uploaded and factored in place, R)
  void *hstage = nullptr;
  size_t hstage_bytes = 0;
  // cached Gaussian sketch S2 (seed, s1, s2)
  double *s2_buf = nullptr;
  size_t s2_bytes = 0;
  bool s2_valid = false;
  uint64_t s2_seed = 0;
  int64_t s2_s1 = 0, s2_s2 = 0;
  int32_t s2_kind_cached = 0;  // randqr_sketch_kind of the cached S2
  int32_t s2_kind = 0;         // randqr_sketch_kind generated when a call passes S2 = NULL
  // status word on the device, and a pinned host copy
  rq::DevStatus *status_dev = nullptr;
  rq::DevStatus *status_host = nullptr;
  char last_err[256] = {0};
  // Gram on the tensor cores (split products) when n <= 128
  bool use_tc = true;
  bool fuse_first_pass = false;  // rand_cholQR n = 64: first solve and Gram in one launch
  // poll bound of the kernels' waits (randqr_set_wait_limit): < 0 = defaults
  int32_t wait_limit = -1;
  // accuracy measurement (randqr_info.want_accuracy): pinned host copy of Q^T Q (packed) and
  // the two residual sums
  double *acc_host = nullptr;
  // per-kernel timing (randqr_set_profiling)
  bool prof = false;
  struct ProfRec {
    int kind;
    cudaEvent_t beg, end;
  };
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  // request server (randqr_submit / randqr_poll), created on first use
  struct randqr_server *server = nullptr;
  // batched plans (randqr_factor_batched), created on first use
  struct randqr_batcher *batcher = nullptr;
};

// The settings a context passes on to the contexts it runs work on (server slots, batch lanes).
inline void rq_inherit_settings(randqr_ctx *sub, const randqr_ctx *ctx) {
  sub->use_tc = ctx->use_tc;
  sub->fuse_first_pass = ctx->fuse_first_pass;
  sub->wait_limit = ctx->wait_limit;
}

// Tear down a context's request server (waits for its streams).
void rq_server_destroy(randqr_ctx *ctx);
// Wait bound of randqr_sketch_static's kernels (randqr_set_wait_limit with no context).
void rq_static_set_wait_limit(int32_t polls);
// Accuracy of a result (api.cu): enqueue the measurement of Q (and of V - Q R when V is intact,
// rq_accuracy_has_resid) on `s`; after the stream has passed it, rq_accuracy_finish fills *info.
randqr_status rq_accuracy_enqueue(randqr_ctx *ctx, const double *V, int64_t ldv, const double *Q, int64_t ldq,
                                  const double *R, int64_t ldr, int64_t m, int64_t n, cudaStream_t s);
bool rq_accuracy_has_resid(const double *V, const double *Q);
void rq_accuracy_finish(randqr_ctx *ctx, int64_t n, bool have_resid, randqr_info *info);
// Tear down a context's batched plans and their lanes.
void rq_batcher_destroy(randqr_ctx *ctx);

namespace rq {
// Kernel kinds for the per-kernel timing record.
enum KernelKind {
  K_GAUSS_GEN = 0, K_CS_SCATTER, K_SKETCH_GEMM, K_HHQR, K_TRSM, K_GRAM, K_POTRF, K_UNPACK,
  K_CS_HASH, K_PACK_DF, K_TRSM_DF, K_GRAM_DF, K_GRAM_TC, K_TRI_INV, K_TRSM_TC, K_SOLVE_GRAM, K_NUM_KINDS
};
}  // namespace rq

namespace rq {
// Status word reset at the start of a call: zero, with the context's wait bound
// (wait_limit_field: 0 = defaults, k + 1 = k polls).
cudaError_t launch_status_reset(DevStatus *st, int32_t wait_limit_field, cudaStream_t s);
// Accuracy of a result (accuracy.cu): sums[0] += ||V - Q R||_F^2 and sums[1] += ||V||_F^2 for R
// upper triangular (packed), FP64 on the CUDA cores.
cudaError_t launch_resid_f64(const double *V, int64_t ldv, const double *Q, int64_t ldq, int64_t m, int64_t n,
                             const double *Rpacked, double *sums, int num_sms, const DevStatus *st, cudaStream_t s);
// The same sums with Q R formed as a split product on the tensor cores (trsm_tc.cu), n <= 64.
cudaError_t launch_trsm_oz_resid(const double *Q, int64_t ldq, const double *V, int64_t ldv, int64_t m, int64_t n,
                                 const double *Rpacked, double *sums, int num_sms, DevStatus *st, cudaStream_t s);
// Largest |eigenvalue| of the symmetric n x n matrix I - G, G given packed upper (host, Jacobi).
double sym_identity_gap2(const double *Gpacked, int n);
// Kernel launchers (defined in the .cu files; all enqueue on `s`).
cudaError_t launch_cs_hash(uint64_t seed, int64_t m, int64_t s1, int32_t *bucket, int8_t *sign,
                           cudaStream_t s);
cudaError_t launch_gauss_gen(uint64_t seed, int64_t s2, int64_t s1, double *S2, cudaStream_t s);
cudaError_t launch_rad_gen(uint64_t seed, int64_t s2, int64_t s1, double *S2, cudaStream_t s);
// W1 += S1 V for the rows row0 .. row0 + m - 1 of a larger matrix (the hash takes the global index)
cudaError_t launch_cs_scatter(const double *V, int64_t m, int64_t n, int64_t ldv, int64_t s1,
                              uint64_t seed, int64_t row0, double *W1, int num_sms, const DevStatus *st,
                              cudaStream_t s);
// Ws += S2 W1 ((s2 x s1)(s1 x n), Ws zeroed by the caller): split products on the tensor cores
// for n <= 64 when use_tc, else FP64 tiles on the CUDA cores
cudaError_t launch_sketch_gemm(const double *S2, const double *W1, int64_t s2, int64_t s1,
                               int64_t n, double *Ws, bool use_tc, int num_sms, DevStatus *st,
                               cudaStream_t s);
bool sketch_oz_supported(int64_t n);
cudaError_t launch_sketch_oz(const double *A, int64_t lda, const double *B, int64_t ldb, int64_t M, int64_t K,
                             int64_t n, double *C, int num_sms, DevStatus *st, cudaStream_t s);
// C += S2 B with S2 (M x K) the Rademacher sketch of `seed` generated inside the kernel (no buffer),
// entries +-1/sqrt(M) exactly as launch_rad_gen writes them; n <= 64
cudaError_t launch_sketch_oz_rademacher(uint64_t seed, const double *B, int64_t ldb, int64_t M, int64_t K, int64_t n,
                                        double *C, int num_sms, DevStatus *st, cudaStream_t s);
// Householder R of the rows x n sketch; with scratch (hhqr_scratch_doubles) and n >= 32 it runs
// on several co-resident CTAs, otherwise on one.
size_t hhqr_scratch_doubles(int64_t rows, int64_t n);
// The argument checks of the factorization entry points (sizes, leading dimensions, and no
// overlap of V, Q, R except Q == V with equal leading dimensions): true if they fail.
bool factor_args_bad(const double *V, int64_t m, int64_t n, int64_t ldv, const double *Q, int64_t ldq,
                     const double *R, int64_t ldr);
// The same on one cluster of 8 CTAs (hhqr_cluster.cu), for n >= 16 and sketches whose columns fit
// in shared memory; launch_hhqr takes it first.
bool hhqr_cluster_ok(int64_t rows, int64_t n);
cudaError_t launch_hhqr_cluster(const double *A, int64_t rows, int64_t n, double *Rpacked, DevStatus *st,
                                cudaStream_t s);
cudaError_t launch_hhqr(double *A, int64_t rows, int64_t n, double *Rpacked, double *scratch, DevStatus *st,
                        cudaStream_t s);
cudaError_t launch_potrf(double *G, int64_t n, double shift_coeff, double *Rc_packed,
                         const double *Rprev_packed, double *Rout_packed, double *Rout,
                         int64_t ldr, int32_t stage, DevStatus *st, cudaStream_t s);
// dense upper triangle (row-major, ld) -> packed; packed -> dense with zeros (or mirrored) below
cudaError_t launch_pack_upper(const double *R, int64_t ldr, int64_t n, double *Rpacked, const DevStatus *st,
                              cudaStream_t s);
cudaError_t launch_unpack_sym(const double *Rpacked, int64_t n, double *R, int64_t ldr, const DevStatus *st,
                              cudaStream_t s);
cudaError_t launch_unpack(const double *Rpacked, int64_t n, double *R, int64_t ldr,
                          const DevStatus *st, cudaStream_t s);
cudaError_t launch_trsm(const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t m,
                        int64_t n, const double *Rpacked, randqr_precision prec, int num_sms,
                        const DevStatus *st, cudaStream_t s);
cudaError_t launch_gram(const double *W, int64_t ldw, int64_t m, int64_t n, double *Gpacked,
                        randqr_precision prec, int num_sms, const DevStatus *st,
                        cudaStream_t s);
// double-float (RANDQR_F32X2) row passes
size_t pack_df_elems(int64_t n);       // float2 entries of the blocked pair form of R
size_t pack_df_rinv_elems(int64_t n);  // float2 entries of the padded 1/r_jj
cudaError_t launch_pack_df(const double *Rp, int64_t n, float2 *Rdf, float2 *rinv,
                           const DevStatus *st, cudaStream_t s);
cudaError_t launch_trsm_df(const void *X, bool x_f64, int64_t ldx, void *Y, bool y_f64,
                           int64_t ldy, int64_t m, int64_t n, const float2 *Rdf,
                           const float2 *rinv, int num_sms, const DevStatus *st,
                           cudaStream_t s);
cudaError_t launch_gram_df(const float2 *W, int64_t ldw, int64_t m, int64_t n, double *Gpacked,
                           int num_sms, const DevStatus *st, cudaStream_t s);
// X = R^{-1} for packed upper-triangular R (small.cu)
cudaError_t launch_tri_inv(const double *Rpacked, int64_t n, double *Xpacked, const DevStatus *st,
                           cudaStream_t s);
// Y = X B (B upper triangular, packed) from exact split products on the tensor cores
// (trsm_tc.cu), n <= 64; Y may equal X (same ld)
bool trsm_oz_supported(int64_t n);
// The first row pass of rand_cholQR in one launch (trsm_tc.cu): W = V B (B = R_s^{-1}, packed
// upper, 64 x 64) stored into W and G += W^T W (packed upper, zeroed by the caller), on paired
// CTAs.  Only n = 64 with contiguous 16-byte aligned rows (ldv = ldw = 64); W may be V.
bool solve_gram_supported(int64_t n, const double *V, int64_t ldv, const double *W, int64_t ldw, int num_sms);
cudaError_t launch_solve_gram(const double *V, int64_t ldv, double *W, int64_t ldw, int64_t m, int64_t n,
                              const double *Bpacked, double *Gpacked, int num_sms, DevStatus *st, cudaStream_t s,
                              int digits);
// One block product of a blocked solve (64 < n <= 128): Y = X B, or Y = Ref + X B when Ref is
// given (Ref may be Y), for X with nk <= 64 columns, Y with nn <= 64.  B packed upper (b_ld = 0:
// dimension nn, entries with row >= nk ignored), or dense row-major with leading dimension b_ld
// >= nn, of which the entries (j, k) with k < 32 <= j are left out when nn > 32 (the first column
// half takes K < 32 only: a second product adds them); reverse (packed B only): X read as X J and
// Y (and Ref) as Y J (J the column reversal; needs Ref, even nk and nn, 16-byte aligned rows)
cudaError_t launch_trsm_oz_block(const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t m, int64_t nk,
                                 int64_t nn, const double *Bpacked, bool reverse, const double *Ref, int64_t ldref,
                                 int num_sms, DevStatus *st, cudaStream_t s, int b_ld = 0);
// The blocks of an upper-triangular R (packed, dimension n, 64 < n <= 128) split at n1 = n - 64:
// mode 0: R22 (rows and columns n1 .. n-1); mode 1: sign * R12 restricted to its upper part
// (entries (j, k) with j <= k, j < n1); mode 2: sign * J L12 J with L12 the strictly lower part of
// R12 (entry (c, k) = sign * R(n1 - 1 - c, n1 + 63 - k) where that lies below R12's diagonal).
// Output packed upper of dimension 64; mode 3: sign * R12 dense, n1 x 64 row-major (ld 64).
cudaError_t launch_block_prep(const double *Rp, int64_t n, int mode, double sign, double *Bout, const DevStatus *st,
                              cudaStream_t s);
// digits: 7 (each term within 2^-54 of its row x column scales, the FP64 path) or 6 (2^-46: RANDQR_F32X2)
cudaError_t launch_trsm_oz(const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t m, int64_t n,
                           const double *Bpacked, int num_sms, DevStatus *st, cudaStream_t s, int digits = 7);
// Gram from exact split products on the tensor cores, n <= 64 (gram_split.cu)
bool gram_split_supported(int64_t n);
cudaError_t launch_gram_split(const void *W, bool in_df, int64_t ldw, int64_t m, int64_t n, double *Gpacked,
                              int num_sms, DevStatus *st, cudaStream_t s);
// G[:, 64:n] (upper triangle) = W^T W[:, 64:n] for 64 < n <= 128 from exact split products
// (gram_cross.cu); with launch_gram_split on the first 64 columns, the whole Gram
cudaError_t launch_gram_cross(const double *W, int64_t ldw, int64_t m, int64_t n, double *Gpacked, int num_sms,
                              DevStatus *st, cudaStream_t s);
// Gram from exact split products on the tensor cores, n <= 128 (gram_tc.cu)
bool gram_oz_supported(int64_t n);
cudaError_t launch_gram_oz(const void *W, bool in_df, int64_t ldw, int64_t m, int64_t n,
                           double *Gpacked, bool acc_f64, int num_sms, DevStatus *st,
                           cudaStream_t s);
}  // namespace rq
