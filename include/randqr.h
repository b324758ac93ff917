/*
 * randqr.h -- C ABI of librandqr.so: rand_cholQR on one GB300 GPU (sm_103a).
 *
 * Method: Higgins, Szyld, Boman & Yamazaki, "Analysis of Randomized Householder-Cholesky
 * QR Factorization with Multisketching" (arXiv 2309.05868).
 *   Algorithm 1 (randQR):      Ws = S2 S1 V;  R_s = R(hhqr(Ws));  W = V R_s^{-1}
 *   Algorithm 2 (cholQR):      G = W^T W;  R_c = chol(G);  Q = W R_c^{-1}
 *   Algorithm 3 (rand_cholQR): the two above, then R = R_c R_s
 *   Algorithm 4 (cholQR2):     cholQR twice
 *
 * Letters: the paper writes V as n x m (n rows); this API uses V as m x n: m rows, n
 * columns, m >> n.  s1 (the paper's p1) is the CountSketch size, s2 (p2) the Gaussian
 * sketch size.  The sizes of the benchmarked configurations are s1 = 2(n^2+n), s2 = 4n.
 *
 * Layout: every matrix is FP64, row-major, with a leading dimension (ld) counted in
 * elements; ld >= number of columns.  Small outputs (R, n x n) are row-major with ldr.
 * Memory: every pointer named *_dev (or V, Q, R, Ws, S2) is device memory on the
 * context's device, owned by the caller, and must stay valid until the call's work on
 * the stream has finished.  The context owns its workspace (sketch buffers, Gram,
 * triangular factors, the cached S2) and frees it in randqr_destroy.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * Every compute call only enqueues work on that stream and returns RANDQR_OK once the
 * launches succeeded -- except when `info` is non-NULL: then the call waits for the
 * stream, copies the device status word and returns the numerical status (e.g.
 * RANDQR_ERR_NOT_SPD) with the details in *info.  randqr_get_status() does the same
 * wait-and-read for calls made with info == NULL.
 *
 * Errors: argument errors are detected on the host before any launch and return
 * RANDQR_ERR_ARG with nothing enqueued.  Numerical failures are detected on the device:
 * the first failing kernel writes the context's status word and every later kernel of
 * that context returns at once, so outputs are left unspecified but nothing faults.
 * A context is not thread-safe: use one context per host thread or serialise calls.
 */
#ifndef RANDQR_H_
#define RANDQR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RANDQR_OK = 0,
  RANDQR_PENDING = 1,           /* serving: request not finished yet */
  RANDQR_ERR_ARG = -1,          /* bad size, ld, pointer or enum; nothing was enqueued */
  RANDQR_ERR_NOT_SPD = -2,      /* Cholesky met a non-positive pivot; info = 1-based index */
  RANDQR_ERR_RANK = -3,         /* zero or non-finite diagonal of R_s (V numerically rank deficient) */
  RANDQR_ERR_NONFINITE = -4,    /* NaN or Inf reached a factor */
  RANDQR_ERR_NOMEM = -5,        /* workspace allocation failed or exceeds the HBM budget */
  RANDQR_ERR_ADMISSION = -6,    /* serving: request can never fit the HBM budget */
  RANDQR_ERR_TIMEOUT = -7,      /* a bounded device-side wait gave up */
  RANDQR_ERR_CUDA = -8,         /* a CUDA runtime call failed (see randqr_last_cuda_error) */
  RANDQR_ERR_TICKET = -9        /* serving: unknown ticket */
} randqr_status;

/* Arithmetic of rand_cholQR's two triangular solves (and, with the tensor cores off, of its Gram).
 * With the tensor cores on (the default) and n <= 64 the solves are split products: RANDQR_FP64
 * keeps seven byte digits of every row (each term within 2^-54 of the product of its row and
 * column scales, FP64's accuracy), RANDQR_F32X2 six (2^-46 per term, about an FP32 pair's
 * accuracy, with fewer products and digits: the faster mixed-precision form);
 * for 64 < n <= 128 (even n) both take the seven-digit blocked products.  With the tensor cores
 * off, RANDQR_F32X2 selects the pair-arithmetic kernels.  Householder QR, Cholesky and
 * R = R_c R_s are FP64 in every case, and the Gram keeps its full split format. */
typedef enum {
  RANDQR_FP64 = 0,   /* FP64 accuracy throughout */
  RANDQR_F32X2 = 1   /* ~46-bit row passes: six-digit split products on the tensor cores, or
                        double-float (pairs of FP32) on the FP32 pipes with the tensor cores off */
} randqr_precision;

/* Details of a call's outcome.  `want_accuracy` is the one input: set it (nonzero) before
 * passing the struct to randqr_factor, randqr_factor_host, randqr_cholqr2 or
 * randqr_shifted_cholqr3 and the call also measures the result it returns, so that each
 * result states its own orthogonality and residual: after the factorization it forms Q^T Q
 * (the same split-product Gram as the method, or the FP64 Gram with the tensor cores off) and
 * ||I - Q^T Q||_2 (largest |eigenvalue|, cyclic Jacobi on the host), and the residual
 * ||V - Q R||_F / ||V||_F from one more pass over V and Q (Q R as a split product on the tensor
 * cores for n <= 64, FP64 otherwise).  That costs about three more reads of an m x n matrix.
 * The fields are -1 when not measured: want_accuracy == 0, a failed factorization, or (for
 * resid_relF) Q aliasing V, whose input is then gone.  The measurement's own error is a few
 * units of 2^-53 (relative to |Q| for the Gram, to |V| for the residual). */
typedef struct {
  int32_t info;         /* failing Cholesky pivot (1-based), or the failing wait's step, or 0 */
  int32_t stage;        /* which Cholesky failed: 1 = first, 2 = second, 3 = third; else 0 */
  double rs_min_diag;   /* smallest diagonal entry of R_s (rand_cholQR) or of the first R */
  double rs_max_diag;   /* largest diagonal entry of that factor */
  int32_t want_accuracy; /* in: nonzero asks for orth_err2 and resid_relF */
  int32_t reserved;
  double orth_err2;     /* out: ||I - Q^T Q||_2, or -1 */
  double resid_relF;    /* out: ||V - Q R||_F / ||V||_F, or -1 */
} randqr_info;

typedef struct randqr_ctx randqr_ctx;

/* Create a context on `device` (made current for the call).  hbm_budget_bytes caps the
 * context's own workspace (0 = no cap).  No workspace is allocated until first use. */
randqr_status randqr_create(randqr_ctx **ctx, int device, size_t hbm_budget_bytes);

/* Wait for the context's work on all streams it used, free its workspace, destroy it. */
randqr_status randqr_destroy(randqr_ctx *ctx);

/* Static description of a status code. */
const char *randqr_status_string(randqr_status s);

/* The last CUDA error string seen by this context ("" if none). */
const char *randqr_last_cuda_error(const randqr_ctx *ctx);

/* Wait for `stream`, read and clear the context's device status word. */
randqr_status randqr_get_status(randqr_ctx *ctx, void *stream, randqr_info *info);

/* Bytes of workspace the context holds now. */
size_t randqr_workspace_bytes(const randqr_ctx *ctx);

/* Failure detection: every wait inside this library's kernels (an mbarrier phase in the
 * tensor-core kernels, a published reflector's flag in the multi-CTA Householder QR) polls a
 * bounded number of times, then gives up, records RANDQR_ERR_TIMEOUT in the status word and
 * drains (waits for its own copies and products in flight, frees its tensor memory) so that
 * the context stays usable.  The default bound (2^24 polls for mbarriers, 2^22 for the
 * Householder flags: seconds) is far above any legitimate wait.  polls >= 0 replaces it for
 * this context's later launches (0: a wait gives up without polling, so any launch that has
 * to wait at all fails with RANDQR_ERR_TIMEOUT -- a way to exercise the failure path on a
 * healthy GPU); polls < 0 restores the default.  The bound, like the tensor-core and
 * fused-pass switches, also holds for the context's served requests (from their next launch)
 * and batched calls (a change drops the captured batch plans).  With ctx == NULL the bound
 * applies to randqr_sketch_static instead (process-wide; set it while no such call is in
 * flight).  Also: the Gram CTAs of the fused first pass (randqr_set_fused_first_pass) wait on
 * their solver's progress words under the same bound. */
randqr_status randqr_set_wait_limit(randqr_ctx *ctx, int32_t polls);

/* Gram products on the tensor cores (default on): for n <= 128 the Gram G = W^T W of the
 * Cholesky passes is formed from exact integer slices of W (eight balanced 7-bit digits of a
 * 54-bit fixed point per column and row group, each an exact f16) multiplied by tcgen05 MMAs
 * with exact FP32 accumulation, then recombined in 64-bit integers.  The triangular solves whose
 * factor is well conditioned are formed the same way as products with the FP64 inverse (n <= 64,
 * and even n <= 128 blocked at n - 64): both solves of rand_cholQR (Algorithm 3; R_s^{-1} is
 * applied to V so that its truncation error is a row-wise backward error in V, and kappa(R_c) =
 * O(1) by the sketch's embedding property; for n > 64 the first solve's off-diagonal block goes
 * by substitution order, T = V2 - W1 R12, W2 = T R22^{-1}) and every pass of CholeskyQR2 and
 * of shifted CholeskyQR3 (their R is within the methods' own condition limit, kappa(R) below
 * about u^{-1/2}, where the computed inverse's right perturbation, of order n u kappa(R), stays
 * below the loss of orthogonality that pass has anyway, of order u kappa(R)^2, and the next pass
 * removes both).  The sketch GEMM Ws = S2 W1 is a split product too for n <= 128.  enable = 0
 * selects the CUDA-core kernels of the chosen precision everywhere. */
randqr_status randqr_set_tensor_cores(randqr_ctx *ctx, int enable);

/* The first row pass of rand_cholQR in one launch (Algorithm 3 with the Gram of Algorithm 2
 * step 1; default off): for n = 64 with the tensor cores on, contiguous rows (ldv = ldq = 64) and
 * 16-byte aligned V and Q, W = V R_s^{-1} and G = W^T W come from one kernel on pairs of CTAs --
 * one forms and stores W, the other takes the Gram of the rows just stored (from L2) -- so V is
 * read once and W written once before the Cholesky factorization, instead of a solve pass
 * followed by a Gram pass that reads W again: 16 m n fewer bytes of HBM traffic per
 * factorization.  The arithmetic is that of the two separate kernels.  Both passes are bound by
 * their instruction issue rather than by HBM on this path, and the fused launch runs each of
 * them on half of the SMs, so it is not faster; enable = 1 selects it (randQR's shard stage,
 * randqr_shard_gram, follows the same switch).  Returns RANDQR_ERR_ARG for a null ctx. */
randqr_status randqr_set_fused_first_pass(randqr_ctx *ctx, int enable);

/* ---- Per-kernel timing (tracing) ------------------------------------------------------
 * While profiling is on, every kernel the context launches is bracketed by two CUDA events
 * recorded on the call's stream.  randqr_get_kernel_times waits for those events, writes
 * for each kernel kind k < *n_kinds (at most max_kinds) the summed device time in ms and
 * the launch count, and clears the record.  randqr_kernel_name(k) names kind k.  The
 * events cost a few microseconds per launch; nothing is recorded while profiling is off. */
randqr_status randqr_set_profiling(randqr_ctx *ctx, int enable);
randqr_status randqr_get_kernel_times(randqr_ctx *ctx, int32_t max_kinds, double *total_ms,
                                      int64_t *launches, int32_t *n_kinds);
const char *randqr_kernel_name(int32_t kind);

/* ---- Step 1 of Algorithm 1, split into its parts (Sec. 4.2) --------------------------
 * CountSketch S1 (Sec. 3: one +-1 per column of S1, row and sign uniform): column i of
 * S1 has its nonzero in row bucket[i] with value sign[i], where
 *   x = splitmix64(seed XOR splitmix64(i)),  bucket = floor(hi32(x) * s1 / 2^32),
 *   sign = -1 if (x & 1) else +1,
 * splitmix64 being the output function of Steele, Lea & Flood's generator.  Writes m
 * int32 buckets and m int8 signs to device memory.  Requires 1 <= s1 < 2^31, m >= 0. */
randqr_status randqr_cs_hash(randqr_ctx *ctx, uint64_t seed, int64_t m, int64_t s1,
                             int32_t *bucket_dev, int8_t *sign_dev, void *stream);

/* Gaussian sketch S2 (s2 x s1, row-major, device) with N(0, 1/s2) entries (Sec. 3,
 * S = G / sqrt(p)).  Entry (r, c) takes Philox4x64-10 (Salmon et al. 2011) at counter
 * (r*s1 + c, 0, 0, 0) with key (seed, 0), u1 = ((x0>>11)+1) 2^-53, u2 = (x1>>11) 2^-53,
 * and Box-Muller z = sqrt(-2 ln u1) cos(2 pi u2).  The integers are exact; the
 * transcendental functions are CUDA's, so entries agree with a host libm to a few ulp. */
randqr_status randqr_gauss_sketch(randqr_ctx *ctx, uint64_t seed, int64_t s2, int64_t s1,
                                  double *S2_dev, void *stream);

/* Rademacher sketch S2 (s2 x s1, row-major, device) with entries +-1/sqrt(s2), the dense
 * alternative to the Gaussian the paper mentions (Sec. 7): entry (r, c) is -1/sqrt(s2) when bit
 * (c mod 64) of splitmix64(seed XOR splitmix64(r * ceil(s1 / 64) + floor(c / 64))) is set, else
 * +1/sqrt(s2).  Integer arithmetic only: bit-exact with any host implementation. */
randqr_status randqr_rademacher_sketch(randqr_ctx *ctx, uint64_t seed, int64_t s2, int64_t s1,
                                      double *S2_dev, void *stream);

/* The sketch of Algorithm 1 step 1 on this context:
 *   RANDQR_SKETCH_GAUSSIAN (default): S2 S1 with S2 from randqr_gauss_sketch(seed + 1) when the
 *     call passes S2 = NULL;
 *   RANDQR_SKETCH_RADEMACHER: the same with S2 from randqr_rademacher_sketch(seed + 1);
 *   RANDQR_SKETCH_COUNT_ONLY: the single CountSketch S1 (S2 = I; the call must pass s2 == s1,
 *     and any S2 is ignored);
 *   RANDQR_SKETCH_GAUSSIAN_ONLY: the single Gaussian sketch S2 (S1 = I; the call must pass
 *     s1 == m; S2 is s2 x m; not for randqr_shard_sketch).
 * The single-sketch kinds are the paper's comparison points (Sec. 6.2, sizes ceil(6.8 (n^2+n))
 * and ceil(36.01 ln n)); a call whose sizes do not fit the kind returns RANDQR_ERR_ARG.
 * Generated sketches are cached per (seed, s1, s2, kind); a Rademacher S2 on the tensor-core path
 * (n <= 128) is not materialised at all: the sketch GEMM draws its signs itself, the same values
 * randqr_rademacher_sketch would write.  Applies to randqr_sketch,
 * randqr_factor, randqr_randqr and randqr_shard_sketch on this context; the batched and
 * serving calls keep the Gaussian multisketch. */
typedef enum {
  RANDQR_SKETCH_GAUSSIAN = 0,
  RANDQR_SKETCH_RADEMACHER = 1,
  RANDQR_SKETCH_COUNT_ONLY = 2,
  RANDQR_SKETCH_GAUSSIAN_ONLY = 3
} randqr_sketch_kind;
randqr_status randqr_set_sketch_kind(randqr_ctx *ctx, int32_t kind);

/* Ws = S2 S1 V (Algorithm 1 step 1), s2 x n row-major (ld n) in device memory.
 * W1 = S1 V is formed in the context's workspace by a scatter-add of V's rows (CountSketch
 * with `seed`), then Ws = S2 W1.  S2 may be NULL: the context then uses (and caches) the
 * sketch randqr_gauss_sketch would give for seed + 1.  Requires 1 <= n <= s2 <= s1,
 * m >= 1, ldv >= n.
 * Accuracy of Ws = S2 W1: with the tensor cores on (the default) and n <= 128, the product is
 * formed from exact integer digit products over chunks of 64 along s1; each term carries an
 * error below 2^-53 of the chunk's largest |S2| entry in its row times the chunk's largest
 * |W1| entry in its column, and integer W1 with +-1 S2 gives the exact result.  Otherwise an
 * FP64 GEMM (error below (s1 / splits + splits) u |S2| |W1|). */
randqr_status randqr_sketch(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                            int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                            const double *S2, double *Ws, void *stream);

/* Ws = S2 S1 V as randqr_sketch computes it on a context with the tensor cores on (the
 * default): the split-product sketch GEMM (n <= 128) with its stated error bound -- but without a
 * context and without allocating any device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc where they need the sketch (a framework that owns
 * every device allocation through its own pool, a host callback or latency-critical path
 * where an allocation's implicit synchronisation is not allowed, a library that must not
 * grow its host application's device footprint).
 * Scratch: the CountSketch accumulator W1 lives in a fixed device array of 2^20 doubles
 * (8 MiB) plus a 64-byte status word, held by every GPU that loads the library until the
 * process exits; requires s1 * n <= 1048576 (else RANDQR_ERR_ARG, nothing enqueued).
 * S2 (s2 x s1, device) is required (NULL -> RANDQR_ERR_ARG), since generating it would need
 * scratch too.  Runs on the current device and `stream`; Ws (s2 x n, ld n) is overwritten.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.  Every call
 * shares the one array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and give wrong results -- serialise them.  Each call clears W1 before use.
 * Same size rules as randqr_sketch otherwise; RANDQR_ERR_CUDA if a launch fails. */
randqr_status randqr_sketch_static(const double *V, int64_t m, int64_t n, int64_t ldv,
                                   int64_t s1, int64_t s2, uint64_t seed, const double *S2,
                                   double *Ws, void *stream);

/* The device status of the last randqr_sketch_static call on the current device: waits for
 * `stream` (the stream that call used), copies the fixed status word to the host (into
 * *info when non-NULL; no allocation) and returns its code -- RANDQR_OK, or
 * RANDQR_ERR_TIMEOUT when a bounded wait of the sketch kernels gave up (Ws is then
 * incomplete).  The word belongs to the last call: the next randqr_sketch_static clears it. */
randqr_status randqr_sketch_static_status(void *stream, randqr_info *info);

/* ---- The factorizations -------------------------------------------------------------
 * All three return Q (m x n, ldq) with orthonormal columns and R (n x n upper, ldr,
 * strictly-lower part zeroed, positive diagonal) with V = Q R.  Q may alias V (ldq ==
 * ldv) for an in-place factorization; otherwise Q and V must not overlap.  Requires
 * 1 <= n <= 128, n <= m, ld >= n. */

/* rand_cholQR (Algorithm 3): randQR with the multisketch S2 S1 (sizes s1, s2, CountSketch
 * seed `seed`, Gaussian S2 as in randqr_sketch), then cholQR of W = V R_s^{-1}, and
 * R = R_c R_s.  R_s is normalised to a positive diagonal.  Requires n <= s2 <= s1.
 * `prec` selects the arithmetic of the row passes (randqr_precision). */
randqr_status randqr_factor(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                            int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                            const double *S2, randqr_precision prec, double *Q, int64_t ldq,
                            double *R, int64_t ldr, randqr_info *info, void *stream);

/* rand_cholQR of a matrix in HOST memory: V (m x n, ldv), Q (m x n, ldq) and R (n x n, ldr)
 * are host pointers; S2 (optional, as in randqr_factor) is device memory.  On `stream`, the
 * call uploads V into a staging area of the context (m n doubles plus n^2, kept for later
 * calls and counted against the HBM budget; growing it waits for the device), runs
 * randqr_factor in place there, and downloads Q and R.  Q may alias V (ldq == ldv); R must
 * not overlap V or Q.  With pinned host memory (cudaMallocHost / cudaHostRegister) the
 * call is asynchronous: V must stay unchanged, and Q and R are complete, only once the
 * stream has reached the end of the call's work (info != NULL waits for it).  Pageable host
 * memory works, with copies that block the host.  One call at a time per context (the
 * staging area is the context's); callers that overlap consecutive factorizations use one
 * context per stream.  Errors as randqr_factor (argument errors before any copy), plus
 * RANDQR_ERR_NOMEM when the staging area cannot be allocated within the budget. */
randqr_status randqr_factor_host(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                                 int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                                 const double *S2, randqr_precision prec, double *Q, int64_t ldq,
                                 double *R, int64_t ldr, randqr_info *info, void *stream);

/* randQR alone (Algorithm 1): Q0 = V R_s^{-1} (S2S1-orthogonal, kappa(Q0) = O(1)) and
 * R0 = R_s.  Same arguments as randqr_factor.  With the tensor cores on (n <= 64, or even
 * n <= 128 with 16-byte aligned rows) the solve is the split-product solve of randqr_factor's
 * first pass; otherwise FP64 forward substitution. */
randqr_status randqr_randqr(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                            int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                            const double *S2, double *Q0, int64_t ldq, double *R0,
                            int64_t ldr, randqr_info *info, void *stream);

/* CholeskyQR2 (Algorithm 4), FP64.  Fails with RANDQR_ERR_NOT_SPD once kappa(V) is near
 * u^{-1/2} (about 1e8, Sec. 6.3). */
randqr_status randqr_cholqr2(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                             int64_t ldv, double *Q, int64_t ldq, double *R, int64_t ldr,
                             randqr_info *info, void *stream);

/* Shifted CholeskyQR3 (cited by the paper, Sec. 1 and 6; defined by Fukaya, Kannan,
 * Nakatsukasa, Yamamoto & Yanagisawa, SISC 2020), FP64: G = V^T V + s I with
 * s = 11 (m n + n (n+1)) u ||V||_F^2, u = 2^-53; R0 = chol(G); Q0 = V R0^{-1}; then
 * CholeskyQR2 of Q0 and R = R12 R0. */
randqr_status randqr_shifted_cholqr3(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                                     int64_t ldv, double *Q, int64_t ldq, double *R,
                                     int64_t ldr, randqr_info *info, void *stream);

/* ---- Row-sharded rand_cholQR (Sec. 4.1) -----------------------------------------------
 * V (M x n) split by rows over P shards, shard k holding rows [row0_k, row0_k + m_k).  The
 * sketch is linear in V and the CountSketch hash is a function of the GLOBAL row index, so
 * Ws = sum_k S2 S1_k V_k and G = sum_k W_k^T W_k: the method needs exactly two sums of small
 * buffers across shards (s2 x n, then n x n), which the caller performs (an allreduce, a
 * host loop, ...).  The stages, in order, every shard with its own context and data:
 *   1. randqr_shard_sketch -> Ws_k;           caller: Ws = sum_k Ws_k
 *   2. randqr_sketch_r(Ws) -> R_s            (deterministic: equal on every shard)
 *   3. randqr_shard_gram(V_k, R_s) -> W_k = V_k R_s^{-1} in Q_k, G_k = W_k^T W_k;
 *                                             caller: G = sum_k G_k
 *   4. randqr_shard_finish(Q_k, G, R_s) -> Q_k = W_k R_c^{-1} in place, R = R_c R_s.
 * With P = 1 (row0 = 0, m_1 = M) the stages compute what randqr_factor computes, kernel for
 * kernel.  All matrices are row-major device buffers; m_k >= 1 (a shard may hold fewer rows
 * than columns); 1 <= n <= 128.  Errors as for the calls above (RANDQR_ERR_ARG before
 * anything is enqueued). */

/* Ws_k = S2 S1_k V_k (s2 x n, ld n): the sketch of shard V_k (m x n, ldv) whose first row is
 * global row row0 >= 0; S1_k holds the CountSketch columns row0 .. row0 + m - 1 of the global
 * S1 (seed, s1), S2 as in randqr_sketch (NULL: generated for seed + 1 and cached). */
randqr_status randqr_shard_sketch(randqr_ctx *ctx, const double *V, int64_t m, int64_t n, int64_t ldv,
                                  int64_t row0, int64_t s1, int64_t s2, uint64_t seed, const double *S2,
                                  double *Ws, void *stream);

/* R_s from the summed sketch Ws (s2 x n, ld n, device; not modified): Householder QR
 * (Algorithm 1 step 2), positive diagonal, written dense to Rs (n x n, ldr, zeros below the
 * diagonal).  Requires n <= s2 <= 2^20.  With info non-NULL, waits and reports the status. */
randqr_status randqr_sketch_r(randqr_ctx *ctx, const double *Ws, int64_t s2, int64_t n, double *Rs,
                              int64_t ldr, randqr_info *info, void *stream);

/* W_k = V_k R_s^{-1} into Q (m x n, ldq; may equal V with ldq == ldv) and G_k = W_k^T W_k
 * into G (n x n, ldg, both triangles written).  Rs (n x n, ldrs) is read from its upper
 * triangle.  The solve and the Gram use the same kernels as randqr_factor. */
randqr_status randqr_shard_gram(randqr_ctx *ctx, const double *V, int64_t m, int64_t n, int64_t ldv,
                                const double *Rs, int64_t ldrs, double *Q, int64_t ldq, double *G,
                                int64_t ldg, void *stream);

/* From the summed G (n x n, ldg, upper triangle read): R_c = chol(G) (Algorithm 2 step 2),
 * Q_k = W_k R_c^{-1} in place (Q, m x n, ldq), and R = R_c R_s (n x n, ldr, dense upper with
 * zeros below).  RANDQR_ERR_NOT_SPD through info (or randqr_get_status) if G is not
 * numerically positive definite. */
randqr_status randqr_shard_finish(randqr_ctx *ctx, double *Q, int64_t m, int64_t n, int64_t ldq,
                                  const double *G, int64_t ldg, const double *Rs, int64_t ldrs, double *R,
                                  int64_t ldr, randqr_info *info, void *stream);

/* ---- Batched: many independent rand_cholQR factorizations in one graph launch ----------
 * The paper factors one matrix at a time; this call factors `count` matrices of uneven
 * sizes (Algorithm 3 on each, sketch sizes 0 -> 2(n^2+n), 4n; S2 from seed + 1) with their
 * kernel chains captured as parallel branches of one CUDA graph over L stream lanes, each
 * lane with its own workspace.  The first call with a given item array (the descriptors'
 * bytes and `prec` are the key) builds a plan: uncaptured warm-up runs size the lanes'
 * workspaces, then an autotuner captures schedules with L = 4, 8, 16, 32 lanes (items dealt
 * to lanes largest-first) and keeps the fastest by timing replays; that first call blocks
 * and allocates.  Later calls with the same items replay the kept graph on `stream` (one
 * launch, no allocation).  With `statuses` non-NULL the call waits and writes each item's
 * status (returning the first error); otherwise it returns after the launch.  The caller
 * keeps V, Q, R alive while a launch runs and does not free them while the plan is cached
 * (the graph holds their addresses; randqr_destroy drops the plans). */
typedef struct {
  const double *V;
  int64_t m, n, ldv;
  double *Q;
  int64_t ldq;
  double *R;
  int64_t ldr;
  int64_t s1, s2;
  uint64_t seed;
} randqr_batch_item;

randqr_status randqr_factor_batched(randqr_ctx *ctx, const randqr_batch_item *items,
                                    int32_t count, randqr_precision prec,
                                    randqr_status *statuses, void *stream);
/* The cached plan of a batch: its lane count and the autotuner's timed replay (ms).
 * RANDQR_ERR_TICKET if no plan exists for these items. */
randqr_status randqr_batch_plan_info(randqr_ctx *ctx, const randqr_batch_item *items,
                                     int32_t count, randqr_precision prec, int32_t *lanes,
                                     float *ms);

/* ---- Serving: continuous batching of factorization requests ---------------------------
 * The paper has no serving layer; these calls run its Algorithms 3 and 4 (and shifted
 * CholeskyQR3) as requests.  A context's server owns `slots` CUDA streams, each with its own
 * workspace, so admitted requests overlap on the device.  Requests are admitted in FIFO
 * order as soon as a slot is free and their footprint (V, Q, R and workspace bytes) fits
 * the HBM budget beside everything in flight; a request larger than the whole budget is
 * refused at submit with RANDQR_ERR_ADMISSION.  Gaussian sketches are generated once per
 * (seed + 1, s1, s2) and shared by all slots.  Submit and poll never block on the device
 * (except the first use of a sketch shape, which generates it); randqr_wait blocks.  The
 * caller keeps V, Q and R alive and untouched until poll/wait returns a status other than
 * RANDQR_PENDING; the ticket is retired by that call.  Single host thread per context. */
typedef enum {
  RANDQR_ALGO_RAND_CHOLQR = 0,
  RANDQR_ALGO_CHOLQR2 = 1,
  RANDQR_ALGO_SHIFTED_CHOLQR3 = 2
} randqr_algo;

typedef struct {
  int32_t algo;        /* randqr_algo */
  int32_t prec;        /* randqr_precision of rand_cholQR's row passes */
  const double *V;     /* m x n, row-major, ldv (device) */
  int64_t m, n, ldv;
  int64_t s1, s2;      /* rand_cholQR sketch sizes; 0 selects 2(n^2+n) and 4n */
  uint64_t seed;       /* CountSketch seed; S2 uses seed + 1 */
  double *Q;           /* m x n, ldq (device); may equal V with ldq == ldv */
  int64_t ldq;
  double *R;           /* n x n, ldr (device) */
  int64_t ldr;
  double max_orth_err; /* loss of orthogonality the caller accepts; with prec = RANDQR_FP64
                          and a value >= 1e-12 rand_cholQR may run its row passes as
                          RANDQR_F32X2, whose results meet ||I - Q^T Q||_2 <= 1e-12 and
                          ||V - QR||_F/||V||_F <= 1e-13 in this library's tests; 0 = FP64 */
  int32_t want_accuracy; /* nonzero: the request's randqr_info carries orth_err2 and
                            resid_relF measured on the device (randqr_info) */
  int32_t reserved;      /* must be 0 */
} randqr_request;

typedef struct {
  uint64_t submitted, completed, queued, running;
  size_t bytes_in_flight;
  int32_t slots;
  size_t budget;
} randqr_serve_stats;

/* (Re)configure the server: number of slots (1..256) and HBM budget in bytes (0 = 64 GiB).
 * Only while nothing is queued or running.  Without this call the first submit creates a
 * server with 8 slots and the context's budget (64 GiB if that is 0). */
randqr_status randqr_serve_config(randqr_ctx *ctx, int32_t slots, size_t hbm_budget_bytes);
/* A descriptor is checked whole before anything is queued: an unknown algo or prec, sizes or
 * leading dimensions out of range, NULL or overlapping V, Q, R (Q == V needs ldq == ldv),
 * sketch sizes that do not fit, or a nonzero reserved field return RANDQR_ERR_ARG and queue
 * nothing; requests already queued or running are not affected.  submit_batch checks every
 * descriptor first and queues none if one is refused. */
randqr_status randqr_submit(randqr_ctx *ctx, const randqr_request *req, uint64_t *ticket);
randqr_status randqr_submit_batch(randqr_ctx *ctx, const randqr_request *reqs, int32_t count,
                                  uint64_t *tickets);
/* RANDQR_PENDING while queued or running; else the request's status (and *info). */
randqr_status randqr_poll(randqr_ctx *ctx, uint64_t ticket, randqr_info *info);
randqr_status randqr_wait(randqr_ctx *ctx, uint64_t ticket, randqr_info *info);
randqr_status randqr_serve_stats_get(randqr_ctx *ctx, randqr_serve_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* RANDQR_H_ */
