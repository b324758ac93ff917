// rowpass.cu -- the passes over the tall m x n matrix:
//   Y = X R^{-1} for upper-triangular R (Algorithm 1 step 3 and Algorithm 2 step 3), by
//     row-wise forward substitution, the solve whose backward error the paper's analysis
//     models (Sec. 5.2.3, eq. triSys): every row is solved on its own;
//   G = W^T W (Algorithm 2 step 1), accumulated into the packed upper triangle.
//
// FP64 form.  On GB300 the FP64 pipe issues about 1.7 FMA/clk/SM (1.0 TFLOP/s measured on
// the whole GPU) against 6.7 TB/s of HBM, so an FP64 row pass of n^2/2 FMAs per 8n-byte row
// is bound by the FP64 pipe, not by memory, for every n >= 2.  The kernels are therefore
// written to keep the FP64 pipe busy with useful FMAs only: one thread per row (no idle
// lanes in the triangular loops), rows staged through shared memory with coalesced loads
// and stores, R and the reciprocal diagonal in shared memory, no FP64 division in the loop.
#include <algorithm>

#include "common.cuh"

namespace rq {

constexpr int TRSM_ROWS = 128;  // rows per tile = threads per CTA

__global__ void __launch_bounds__(TRSM_ROWS) k_trsm_f64(const double *__restrict__ X, int64_t ldx,
                                                        double *Y, int64_t ldy, int64_t m, int n,
                                                        const double *__restrict__ Rp,
                                                        const DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ double sm[];
  const int P = n * (n + 1) / 2;
  const int ld = (n & 1) ? n : n + 1;  // odd stride in doubles: rows fall in distinct banks
  double *R = sm;
  double *rinv = R + P;
  double *T = rinv + n;
  const int tid = threadIdx.x;
  for (int e = tid; e < P; e += blockDim.x) R[e] = Rp[e];
  __syncthreads();
  for (int j = tid; j < n; j += blockDim.x) rinv[j] = 1.0 / R[tri_idx(j, j)];
  __syncthreads();
  for (int64_t row0 = (int64_t)blockIdx.x * TRSM_ROWS; row0 < m;
       row0 += (int64_t)gridDim.x * TRSM_ROWS) {
    const int rows = (int)imin64(TRSM_ROWS, m - row0);
    for (int e = tid; e < rows * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      T[r * ld + c] = X[(row0 + r) * ldx + c];
    }
    __syncthreads();
    if (tid < rows) {
      double *w = T + tid * ld;
      for (int j = 0; j < n; ++j) {
        const double *rc = R + j * (j + 1) / 2;
        double s = w[j];
        for (int k = 0; k < j; ++k) s = fma(-w[k], rc[k], s);
        w[j] = s * rinv[j];
      }
    }
    __syncthreads();
    for (int e = tid; e < rows * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      Y[(row0 + r) * ldy + c] = T[r * ld + c];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Gram: each thread owns up to Q packed pairs (k <= j) of G and keeps their sums in
// registers across every tile of its CTA's row range; one atomic per pair at the end.
// ---------------------------------------------------------------------------------------
constexpr int GRAM_THREADS = 256, GRAM_TILE = 32;

template <int Q>
__global__ void __launch_bounds__(GRAM_THREADS) k_gram_f64(const double *__restrict__ W, int64_t ldw,
                                                           int64_t m, int n, int64_t rows_per_cta,
                                                           double *Gp, const DevStatus *st) {
  if (status_failed(st)) return;
  __shared__ double T[GRAM_TILE * 129];
  const int ld = (n & 1) ? n : n + 1;
  const int P = n * (n + 1) / 2;
  const int tid = threadIdx.x;
  int pk[Q], pj[Q];
  double acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int p = tid + q * GRAM_THREADS;
    if (p >= P) p = 0;  // padding pairs compute a harmless duplicate and are not stored
    int j = (int)((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
    while (j * (j + 1) / 2 > p) --j;
    while ((j + 1) * (j + 2) / 2 <= p) ++j;
    pj[q] = j;
    pk[q] = p - j * (j + 1) / 2;
    acc[q] = 0.0;
  }
  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  for (int64_t row0 = r_begin; row0 < r_end; row0 += GRAM_TILE) {
    const int rows = (int)imin64(GRAM_TILE, r_end - row0);
    __syncthreads();
    for (int e = tid; e < rows * n; e += GRAM_THREADS) {
      const int r = e / n, c = e - r * n;
      T[r * ld + c] = W[(row0 + r) * ldw + c];
    }
    __syncthreads();
    for (int r = 0; r < rows; ++r) {
      const double *t = T + r * ld;
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[q] = fma(t[pk[q]], t[pj[q]], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int p = tid + q * GRAM_THREADS;
    if (p < P) atomicAdd(Gp + p, acc[q]);
  }
}

cudaError_t launch_trsm(const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t m,
                        int64_t n, const double *Rpacked, randqr_precision prec, int num_sms,
                        const DevStatus *st, cudaStream_t s) {
  if (prec != RANDQR_FP64) return cudaErrorInvalidValue;
  const int ld = (n & 1) ? (int)n : (int)n + 1;
  const size_t smem = sizeof(double) * ((size_t)(n * (n + 1) / 2) + n + (size_t)TRSM_ROWS * ld);
  cudaError_t e = cudaFuncSetAttribute(k_trsm_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = std::max(1, (int)((220 * 1024) / smem));
  per_sm = std::min(per_sm, 8);
  const int64_t tiles = ceil_div(m, TRSM_ROWS);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms * per_sm));
  k_trsm_f64<<<blocks, TRSM_ROWS, smem, s>>>(X, ldx, Y, ldy, m, (int)n, Rpacked, st);
  return cudaGetLastError();
}

cudaError_t launch_gram(const double *W, int64_t ldw, int64_t m, int64_t n, double *Gpacked,
                        randqr_precision prec, int num_sms, const DevStatus *st,
                        cudaStream_t s) {
  if (prec != RANDQR_FP64) return cudaErrorInvalidValue;
  const int64_t P = n * (n + 1) / 2;
  const int64_t Qn = ceil_div(P, GRAM_THREADS);
  const int blocks_target = num_sms * 2;
  const int64_t rows_per_cta = std::max<int64_t>(GRAM_TILE, ceil_div(ceil_div(m, blocks_target), GRAM_TILE) * GRAM_TILE);
  const int blocks = (int)ceil_div(m, rows_per_cta);
  if (Qn <= 3)
    k_gram_f64<3><<<blocks, GRAM_THREADS, 0, s>>>(W, ldw, m, (int)n, rows_per_cta, Gpacked, st);
  else if (Qn <= 9)
    k_gram_f64<9><<<blocks, GRAM_THREADS, 0, s>>>(W, ldw, m, (int)n, rows_per_cta, Gpacked, st);
  else if (Qn <= 19)
    k_gram_f64<19><<<blocks, GRAM_THREADS, 0, s>>>(W, ldw, m, (int)n, rows_per_cta, Gpacked, st);
  else
    k_gram_f64<33><<<blocks, GRAM_THREADS, 0, s>>>(W, ldw, m, (int)n, rows_per_cta, Gpacked, st);
  return cudaGetLastError();
}

}  // namespace rq
