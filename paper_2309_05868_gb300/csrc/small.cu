// small.cu -- the O(poly(n)) steps that sit between the row passes:
//   Householder QR of the s2 x n sketch (Algorithm 1 step 2), R only, positive diagonal;
//   Cholesky of the n x n Gram (Algorithm 2 step 2), optionally shifted (sCholQR3);
//   R = R_c R_prev (Algorithm 3 step 3 / Algorithm 4 step 3).
// Each runs on the device (one CTA, or a few co-resident CTAs for the Householder QR) so no
// host round trip separates it from the row passes; all are FP64.  Triangular factors travel between kernels in packed column-major upper storage
// (tri_idx), which is what the row-pass kernels stage in shared memory.
#include "common.cuh"

namespace rq {

constexpr int SMALL_THREADS = 512;

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (int)(blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------------------
// Householder QR, R only.  Column j: sigma = ||A[j+1:, j]||^2, beta = -sign(a_jj) sqrt(a_jj^2
// + sigma), v = A[j:, j] / (a_jj - beta) with v_j = 1, tau = (beta - a_jj) / beta, then
// A[j:, j+1:] -= tau v (v^T A[j:, j+1:]).  The recurrence is LAPACK's dgeqr2 (Golub & Van
// Loan Alg. 5.2.1).  A is row-major rows x n; in shared memory (row pitch n + 1, so that a
// warp walking down a column touches different banks) when it fits, else updated in place in
// global memory (L2, pitch n).  v is applied as A[i, j] * (1 / (a_jj - beta)) on the fly.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(SMALL_THREADS) k_hhqr(double *Ag, int rows, int n,
                                                        bool use_smem, double *Rp,
                                                        DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double s_tau, s_rv0;
  double *w = sm;                         // n
  double *A = use_smem ? sm + n : Ag;     // rows x ld
  const int ld = use_smem ? n + 1 : n;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (use_smem) {
    for (int e = tid; e < rows * n; e += nt) A[(e / n) * ld + e % n] = Ag[e];
    __syncthreads();
  }
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int j = 0; j < n; ++j) {
    double part = 0.0;
    for (int i = j + 1 + tid; i < rows; i += nt) part = fma(A[i * ld + j], A[i * ld + j], part);
    const double sigma = block_sum(part, red);
    if (tid == 0) {
      const double x0 = A[j * ld + j];
      if (sigma == 0.0) {
        s_tau = 0.0;
      } else {
        const double alpha = sqrt(x0 * x0 + sigma);
        const double beta = (x0 >= 0.0) ? -alpha : alpha;
        s_rv0 = 1.0 / (x0 - beta);
        s_tau = (beta - x0) / beta;
        A[j * ld + j] = beta;
      }
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau == 0.0) continue;
    const double rv0 = s_rv0;
    // w_k = tau (a_jk + sum_{i>j} v_i a_ik), one warp per column k
    for (int k = j + 1 + wid; k < n; k += nw) {
      double acc = 0.0;
      for (int i = j + 1 + lane; i < rows; i += 32) acc = fma(A[i * ld + j], A[i * ld + k], acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) w[k] = tau * fma(acc, rv0, A[j * ld + k]);
    }
    __syncthreads();
    // A[j, k] -= w_k;  A[i, k] -= v_i w_k  (i > j, k > j); 64-column strips, no index division
    for (int i0 = j; i0 < rows; i0 += nt / 64) {
      const int i = i0 + tid / 64;
      if (i >= rows) break;
      for (int k = j + 1 + (tid & 63); k < n; k += 64) {
        if (i == j)
          A[j * ld + k] -= w[k];
        else
          A[i * ld + k] = fma(-A[i * ld + j] * rv0, w[k], A[i * ld + k]);
      }
    }
    __syncthreads();
  }
  // R with rows flipped to a positive diagonal, packed column-major upper.
  for (int e = tid; e < n * (n + 1) / 2; e += nt) {
    int j = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while (j * (j + 1) / 2 > e) --j;
    while ((j + 1) * (j + 2) / 2 <= e) ++j;
    const int k = e - j * (j + 1) / 2;
    const double d = A[k * ld + k];
    Rp[e] = (d < 0.0) ? -A[k * ld + j] : A[k * ld + j];
  }
  if (tid == 0) {
    double dmin = INFINITY, dmax = 0.0;
    int bad = 0;
    for (int k = 0; k < n; ++k) {
      const double d = fabs(A[k * ld + k]);
      if (!(d > 0.0) || !isfinite(d)) bad = bad ? bad : k + 1;
      dmin = fmin(dmin, d);
      dmax = fmax(dmax, d);
    }
    st->dmin = dmin;
    st->dmax = dmax;
    if (bad) status_fail(st, RANDQR_ERR_RANK, bad, 0);
  }
}

// ---------------------------------------------------------------------------------------
// The same Householder QR on HQ_CTAS co-resident CTAs (one cooperative launch).  CTA b keeps
// the columns k with k % HQ_CTAS == b in shared memory (column-major, so a warp walks down a
// column with unit stride).  Step j: the owner of column j forms the reflector (sigma, beta,
// tau, v = A[j+1:, j] / (a_jj - beta)) and publishes tau, beta and v through global memory (L2)
// with a per-step flag; every CTA then applies it to its own columns k > j, one warp per
// column.  The owner of column j + 1 updates that column first and publishes reflector j + 1
// before its other columns (look-ahead), so a step costs about one column update plus one
// flag round trip.  Waits are bounded (RANDQR_ERR_TIMEOUT).  The result equals k_hhqr's up to
// the order of the dot products.
// ---------------------------------------------------------------------------------------
constexpr int HQ_CTAS = 16, HQ_THREADS = 256, HQ_MAX_WAIT = 1 << 22;


// Form reflector j from local column `col` (rows 0..rows-1) and publish it; one warp.
__device__ __forceinline__ void hq_reflect(double *col, int rows, int j, double *pub, volatile int *flag,
                                          int lane) {
  double part = 0.0;
  for (int i = j + 1 + lane; i < rows; i += 32) part = fma(col[i], col[i], part);
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const double x0 = col[j];
  double tau = 0.0, beta = x0, rv0 = 0.0;
  if (part != 0.0) {
    const double alpha = sqrt(x0 * x0 + part);
    beta = (x0 >= 0.0) ? -alpha : alpha;
    rv0 = 1.0 / (x0 - beta);
    tau = (beta - x0) / beta;
  }
  // pub: [tau, beta, v_{j+1} .. v_{rows-1}] at offsets 0, 1, 2 + (i - j - 1)
  for (int i = j + 1 + lane; i < rows; i += 32) {
    const double v = col[i] * rv0;
    col[i] = v;
    pub[2 + (i - j - 1)] = v;
  }
  if (lane == 0) {
    col[j] = beta;
    pub[0] = tau;
    pub[1] = beta;
  }
  __threadfence();  // each lane's part of the reflector is visible device-wide ...
  __syncwarp();
  if (lane == 0) *flag = 1;  // ... before the flag
}

__global__ void __launch_bounds__(HQ_THREADS) k_hhqr_coop(const double *Ag, int rows, int n, double *pub,
                                                          int *flags, double *Rp, DevStatus *st) {
  if (status_failed(st)) return;
  const int lim = wait_bound(st, HQ_MAX_WAIT);
  extern __shared__ double hq_sm[];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ncl = (n - b + HQ_CTAS - 1) / HQ_CTAS;  // local columns: k = b + HQ_CTAS * c
  double *cols = hq_sm;                              // ncl x rows
  double *vsh = hq_sm + (size_t)ncl * rows;          // rows: current reflector
  __shared__ double s_tau;
  __shared__ int s_fail;
  const size_t stride = (size_t)rows + 2;
  for (int e = tid; e < ncl * rows; e += HQ_THREADS) {
    const int c = e / rows, i = e - c * rows;
    cols[e] = Ag[(size_t)i * n + b + HQ_CTAS * c];
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // reflector 0 from its owner
  if (b == 0 && warp == 0) hq_reflect(cols, rows, 0, pub, flags, lane);
  for (int j = 0; j < n; ++j) {
    // wait for reflector j
    if (tid == 0) {
      int ok = 0;
      for (int it = 0; it < lim && !ok; ++it) ok = *(volatile int *)&flags[j];
      if (!ok) {
        s_fail = 1;
        status_fail(st, RANDQR_ERR_TIMEOUT, j + 1, 0);
      }
      __threadfence();
    }
    __syncthreads();
    if (s_fail) return;
    const double *pj = pub + (size_t)j * stride;
    for (int i = j + 1 + tid; i < rows; i += HQ_THREADS) vsh[i] = *(volatile const double *)&pj[2 + (i - j - 1)];
    if (tid == 0) s_tau = *(volatile const double *)&pj[0];
    __syncthreads();
    const double tau = s_tau;
    // local columns k > j; the owner of column j + 1 handles it first and publishes reflector j + 1
    const int c_next = (j + 1 < n && (j + 1) % HQ_CTAS == b) ? (j + 1) / HQ_CTAS : -1;
    if (tau != 0.0) {
      for (int t = warp; t < ncl; t += HQ_THREADS / 32) {
        // order: c_next first (warp 0), then the rest
        int c = t;
        if (c_next >= 0) c = (t == 0) ? c_next : (t <= c_next ? t - 1 : t);
        const int k = b + HQ_CTAS * c;
        if (k <= j) continue;
        double *col = cols + (size_t)c * rows;
        double acc = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) acc = fma(vsh[i], col[i], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double w = tau * (col[j] + acc);
        if (lane == 0) col[j] -= w;
        for (int i = j + 1 + lane; i < rows; i += 32) col[i] = fma(-vsh[i], w, col[i]);
        __syncwarp();
        if (c == c_next) hq_reflect(col, rows, j + 1, pub + (size_t)(j + 1) * stride, flags + j + 1, lane);
      }
    } else if (c_next >= 0 && warp == 0) {
      hq_reflect(cols + (size_t)c_next * rows, rows, j + 1, pub + (size_t)(j + 1) * stride, flags + j + 1, lane);
    }
    __syncthreads();
  }
  // R (rows flipped to a positive diagonal), packed column-major upper: this CTA's columns
  for (int c = 0; c < ncl; ++c) {
    const int k = b + HQ_CTAS * c;
    for (int i = tid; i <= k; i += HQ_THREADS) {
      const double bi = *(volatile const double *)&pub[(size_t)i * stride + 1];
      const double v = cols[(size_t)c * rows + i];
      Rp[tri_idx(i, k)] = bi < 0.0 ? -v : v;
    }
  }
  if (b == 0 && tid == 0) {
    double dmin = INFINITY, dmax = 0.0;
    int bad = 0;
    for (int k = 0; k < n; ++k) {
      const double d = fabs(*(volatile const double *)&pub[(size_t)k * stride + 1]);
      if (!(d > 0.0) || !isfinite(d)) bad = bad ? bad : k + 1;
      dmin = fmin(dmin, d);
      dmax = fmax(dmax, d);
    }
    st->dmin = dmin;
    st->dmax = dmax;
    if (bad) status_fail(st, RANDQR_ERR_RANK, bad, 0);
  }
}

size_t hhqr_scratch_doubles(int64_t rows, int64_t n) { return (size_t)n * (size_t)(rows + 2) + (size_t)(n + 1) / 2 + 1; }

cudaError_t launch_hhqr(double *A, int64_t rows, int64_t n, double *Rpacked, double *scratch, DevStatus *st,
                        cudaStream_t s) {
  if (hhqr_cluster_ok(rows, n)) {
    // one thread-block cluster; where the cluster cannot be placed, the cooperative kernel
    const cudaError_t e = launch_hhqr_cluster(A, rows, n, Rpacked, st, s);
    if (e == cudaSuccess) return e;
    (void)cudaGetLastError();
  }
  const int ncl = (int)ceil_div(n, HQ_CTAS);
  const size_t coop_smem = sizeof(double) * (size_t)(ncl + 1) * (size_t)rows;
  if (scratch && n >= 2 * HQ_CTAS && coop_smem <= 200 * 1024) {
    // scratch: n published reflectors (rows + 2 doubles each), then n flags
    double *pub = scratch;
    int *flags = (int *)(scratch + (size_t)n * (size_t)(rows + 2));
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    if (coop_smem > 48 * 1024) {
      e = cudaFuncSetAttribute(k_hhqr_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)coop_smem);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(HQ_CTAS);
    cfg.blockDim = dim3(HQ_THREADS);
    cfg.dynamicSmemBytes = coop_smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_hhqr_coop, (const double *)A, (int)rows, (int)n, pub, flags, Rpacked, st);
  }
  size_t smem = sizeof(double) * (size_t)(n + rows * (n + 1));
  bool use_smem = smem <= 200 * 1024;
  size_t dyn = use_smem ? smem : sizeof(double) * (size_t)n;
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_hhqr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  k_hhqr<<<1, SMALL_THREADS, dyn, s>>>(A, (int)rows, (int)n, use_smem, Rpacked, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Cholesky G = R^T R (upper), right-looking on the packed upper triangle in shared memory:
// r_jj = sqrt(g_jj); r_jl = g_jl / r_jj; g_kl -= r_jk r_jl for j < k <= l.  A pivot that is
// not > 0 (or NaN) stops the factorization with RANDQR_ERR_NOT_SPD(j+1).  If shift_coeff
// is nonzero, shift_coeff * trace(G) is added to the diagonal first (sCholQR3's shift,
// since trace(V^T V) = ||V||_F^2).  Step j's row of R is copied to a contiguous buffer, and the
// trailing update gives each warp whole columns l (lanes down the rows k <= l of the packed
// column), so no thread divides to find its entry.
// Then, if Rprev is given, Rout = R Rprev (upper x upper, packed); if Rout_dense is given,
// the final factor (Rout, or R itself) is written there row-major with zeros below: a second
// kernel over many CTAs (the product's n^3 / 6 FP64 multiply-adds would take one SM's FP64
// pipe about 0.1 ms at n = 128).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(SMALL_THREADS) k_potrf(double *Gp, int n, double shift_coeff, double *Rcp,
                                                         int stage, DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ double A[];  // packed upper, n(n+1)/2, then row j of R (n)
  __shared__ double red[32];
  __shared__ int s_fail;
  __shared__ double s_inv;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int P = n * (n + 1) / 2;
  double *rowj = A + P;
  for (int e = tid; e < P; e += nt) A[e] = Gp[e];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  if (shift_coeff != 0.0) {
    double part = 0.0;
    for (int j = tid; j < n; j += nt) part += A[tri_idx(j, j)];
    const double tr = block_sum(part, red);
    for (int j = tid; j < n; j += nt) A[tri_idx(j, j)] += shift_coeff * tr;
    __syncthreads();
  }
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double d = A[tri_idx(j, j)];
      if (!(d > 0.0) || !isfinite(d)) {
        s_fail = j + 1;
      } else {
        const double r = sqrt(d);
        A[tri_idx(j, j)] = r;
        s_inv = 1.0 / r;
      }
    }
    __syncthreads();
    if (s_fail) break;
    // row j of R by the pivot's reciprocal (one multiply per entry), kept contiguous as well
    const double inv = s_inv;
    for (int l = j + 1 + tid; l < n; l += nt) {
      const double v = A[tri_idx(j, l)] * inv;
      A[tri_idx(j, l)] = v;
      rowj[l] = v;
    }
    __syncthreads();
    for (int l = j + 1 + warp; l < n; l += nwarps) {
      const double rl = rowj[l];
      double *col = A + l * (l + 1) / 2;  // column l: rows 0 .. l
      for (int k = j + 1 + lane; k <= l; k += 32) col[k] = fma(-rowj[k], rl, col[k]);
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) status_fail(st, RANDQR_ERR_NOT_SPD, s_fail, stage);
    return;
  }
  for (int e = tid; e < P; e += nt) Rcp[e] = A[e];
}

// Rout(i, j) = sum_{k=i..j} R(i, k) Rprev(k, j) (packed, when Routp) and the dense row-major
// Rdense (Rout, or R itself without Rprev), zeros below; both triangles staged in shared memory
// by every CTA, one output per thread.
__global__ void __launch_bounds__(256) k_tri_mul(const double *Rp, const double *Rprev, int n, double *Routp,
                                                 double *Rdense, int64_t ldr, const DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ double tm_sm[];
  const int P = n * (n + 1) / 2;
  double *Ra = tm_sm, *Rb = tm_sm + P;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    Ra[e] = Rp[e];
    if (Rprev) Rb[e] = Rprev[e];
  }
  __syncthreads();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - i * n;
    double v = 0.0;
    if (j >= i) {
      if (Rprev) {
        for (int k = i; k <= j; ++k) v = fma(Ra[tri_idx(i, k)], Rb[tri_idx(k, j)], v);
        if (Routp) Routp[tri_idx(i, j)] = v;
      } else {
        v = Ra[tri_idx(i, j)];
      }
    }
    if (Rdense) Rdense[(int64_t)i * ldr + j] = v;
  }
}

cudaError_t launch_potrf(double *G, int64_t n, double shift_coeff, double *Rc_packed,
                         const double *Rprev_packed, double *Rout_packed, double *Rout,
                         int64_t ldr, int32_t stage, DevStatus *st, cudaStream_t s) {
  const size_t dyn = sizeof(double) * (size_t)(n * (n + 1) / 2 + n);
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  k_potrf<<<1, SMALL_THREADS, dyn, s>>>(G, (int)n, shift_coeff, Rc_packed, stage, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || (Rprev_packed == nullptr && Rout == nullptr)) return e;
  const size_t dyn2 = sizeof(double) * (size_t)(n * (n + 1));
  if (dyn2 > 48 * 1024) {
    e = cudaFuncSetAttribute(k_tri_mul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn2);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (int)std::min<int64_t>(64, std::max<int64_t>(1, (n * n + 255) / 256));
  k_tri_mul<<<blocks, 256, dyn2, s>>>(Rc_packed, Rprev_packed, (int)n, Rout_packed, Rout, ldr, st);
  return cudaGetLastError();
}

// Blocks of a packed upper-triangular R split at n1 = n - 64, as packed 64 x 64 upper matrices
// (launch_block_prep in common.cuh describes the modes).
__global__ void k_block_prep(const double *Rp, int n, int mode, double sign, double *Bout, const DevStatus *st) {
  if (status_failed(st)) return;
  const int n1 = n - 64;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 * 64; e += gridDim.x * blockDim.x) {
    const int j = e >> 6, k = e & 63;  // row j, column k of the output (j <= k stored)
    if (mode == 3) {  // dense R12: R(j, n1 + k), j < n1 <= n1 + k
      if (j < n1) Bout[j * 64 + k] = sign * Rp[tri_idx(j, n1 + k)];
      continue;
    }
    if (j > k) continue;
    double v = 0.0;
    if (mode == 0) {
      v = Rp[tri_idx(n1 + j, n1 + k)];
    } else if (mode == 1) {
      if (j < n1) v = sign * Rp[tri_idx(j, n1 + k)];
    } else {
      const int rj = n1 - 1 - j, ck = 63 - k;  // R12 entry (rj, ck), in R12's strictly lower part
      if (rj >= 0 && rj > ck) v = sign * Rp[tri_idx(rj, n1 + ck)];
    }
    Bout[tri_idx(j, k)] = v;
  }
}

cudaError_t launch_block_prep(const double *Rp, int64_t n, int mode, double sign, double *Bout, const DevStatus *st,
                              cudaStream_t s) {
  k_block_prep<<<16, 256, 0, s>>>(Rp, (int)n, mode, sign, Bout, st);
  return cudaGetLastError();
}

__global__ void k_status_reset(DevStatus *st, int32_t wait_limit_field) {
  st->code = 0;
  st->info = 0;
  st->stage = 0;
  st->wait_limit = wait_limit_field;
  st->dmin = 0.0;
  st->dmax = 0.0;
}

cudaError_t launch_status_reset(DevStatus *st, int32_t wait_limit_field, cudaStream_t s) {
  k_status_reset<<<1, 1, 0, s>>>(st, wait_limit_field);
  return cudaGetLastError();
}

// Packed upper -> dense row-major with zeros below the diagonal.
__global__ void k_unpack(const double *Rp, int n, double *R, int64_t ldr, const DevStatus *st) {
  if (status_failed(st)) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e % n;
    R[(int64_t)i * ldr + j] = (j >= i) ? Rp[tri_idx(i, j)] : 0.0;
  }
}

__global__ void k_pack_upper(const double *R, int64_t ldr, int n, double *Rp, const DevStatus *st) {
  if (status_failed(st)) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e % n;
    if (j >= i) Rp[tri_idx(i, j)] = R[(int64_t)i * ldr + j];
  }
}

__global__ void k_unpack_sym(const double *Rp, int n, double *R, int64_t ldr, const DevStatus *st) {
  if (status_failed(st)) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e % n;
    R[(int64_t)i * ldr + j] = Rp[j >= i ? tri_idx(i, j) : tri_idx(j, i)];
  }
}

cudaError_t launch_pack_upper(const double *R, int64_t ldr, int64_t n, double *Rpacked, const DevStatus *st,
                              cudaStream_t s) {
  k_pack_upper<<<(unsigned)ceil_div(n * n, 256), 256, 0, s>>>(R, ldr, (int)n, Rpacked, st);
  return cudaGetLastError();
}

cudaError_t launch_unpack_sym(const double *Rpacked, int64_t n, double *R, int64_t ldr, const DevStatus *st,
                              cudaStream_t s) {
  k_unpack_sym<<<(unsigned)ceil_div(n * n, 256), 256, 0, s>>>(Rpacked, (int)n, R, ldr, st);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const double *Rpacked, int64_t n, double *R, int64_t ldr,
                          const DevStatus *st, cudaStream_t s) {
  k_unpack<<<(unsigned)ceil_div(n * n, 256), 256, 0, s>>>(Rpacked, (int)n, R, ldr, st);
  return cudaGetLastError();
}

// X = R^{-1} for upper-triangular R (packed), FP64, column by column: column k solves
// R x = e_k by back substitution, x_k = 1 / r_kk, x_i = -(sum_{l=i+1..k} r_il x_l) / r_ii for
// i = k-1 .. 0.  Then R X = I + F with |F| <= gamma |R| |X|: the computed inverse is
// R^{-1} (I + F), a perturbation that stays on the right of a product V X, so V X = W (I + F)
// keeps W's conditioning.  One warp per column; lane t owns the partial sums of rows t, t + 32,
// ... and adds r_il x_l to them as soon as x_l is known (the column-oriented form of the same
// recurrence), so one step costs a broadcast, a multiply and a fused multiply-add in
// sequence.  The pivots' reciprocals are formed once.
constexpr int TRI_COLS = 8;  // columns (warps) per CTA
constexpr int TRI_SLOTS = 4;  // rows per lane: n <= 128

__global__ void __launch_bounds__(TRI_COLS * 32) k_tri_inv(const double *Rp, int n, double *Xp,
                                                         const DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ double tri_sm[];
  const int P = n * (n + 1) / 2;
  double *R = tri_sm, *rdiag = tri_sm + P;
  double *x = rdiag + n + (threadIdx.x >> 5) * n;
  for (int e = threadIdx.x; e < P; e += blockDim.x) R[e] = Rp[e];
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) rdiag[e] = 1.0 / R[tri_idx(e, e)];
  __syncthreads();
  const int lane = threadIdx.x & 31, k = blockIdx.x * TRI_COLS + (threadIdx.x >> 5);
  if (k >= n) return;
  const double xk = rdiag[k];
  double acc[TRI_SLOTS];
#pragma unroll
  for (int q = 0; q < TRI_SLOTS; ++q) {
    const int i = lane + 32 * q;
    acc[q] = i < k ? R[tri_idx(i, k)] * xk : 0.0;
  }
  if (lane == 0) x[k] = xk;
  for (int l = k - 1; l >= 0; --l) {
    double mine = acc[0];
#pragma unroll
    for (int q = 1; q < TRI_SLOTS; ++q)
      if ((l >> 5) == q) mine = acc[q];
    const double xl = -__shfl_sync(0xffffffffu, mine, l & 31) * rdiag[l];
    if (lane == 0) x[l] = xl;
#pragma unroll
    for (int q = 0; q < TRI_SLOTS; ++q) {
      const int i = lane + 32 * q;
      if (i < l) acc[q] = fma(R[tri_idx(i, l)], xl, acc[q]);
    }
  }
  __syncwarp();
  for (int i = lane; i <= k; i += 32) Xp[tri_idx(i, k)] = x[i];
}

cudaError_t launch_tri_inv(const double *Rpacked, int64_t n, double *Xpacked, const DevStatus *st,
                           cudaStream_t s) {
  const size_t dyn = sizeof(double) * (size_t)(n * (n + 1) / 2 + n + TRI_COLS * n);
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_tri_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  k_tri_inv<<<(unsigned)ceil_div(n, TRI_COLS), TRI_COLS * 32, dyn, s>>>(Rpacked, (int)n, Xpacked, st);
  return cudaGetLastError();
}

}  // namespace rq
