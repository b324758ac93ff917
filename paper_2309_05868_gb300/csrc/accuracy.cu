// accuracy.cu -- the accuracy a factorization states about itself (randqr_info.want_accuracy):
// ||I - Q^T Q||_2 and ||V - Q R||_F / ||V||_F, the two measures of Sec. 6.3 (with the 2-norm
// for orthogonality, the norm the stability analysis bounds).
//
// The Gram Q^T Q comes from the library's own Gram kernels (api.cu); this file holds the
// FP64 residual pass used when the tensor-core product is not available (n > 64 or tensor
// cores off), and the host-side spectral norm of the small symmetric matrix I - Q^T Q.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace rq {

namespace {

constexpr int RS_THREADS = 256;

// sums[0] += sum_i ||v_i - q_i R||^2, sums[1] += sum_i ||v_i||^2 (R upper triangular, packed by
// columns).  One warp per row at a time: the row of Q goes to shared memory, lane t forms the
// entries k = t, t + 32, ... of q_i R from R in shared memory.
__global__ void __launch_bounds__(RS_THREADS) k_resid_f64(const double *__restrict__ V, int64_t ldv,
                                                          const double *__restrict__ Q, int64_t ldq, int64_t m, int n,
                                                          const double *__restrict__ Rp, double *sums,
                                                          const DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ double rs_sm[];
  const int P = n * (n + 1) / 2;
  double *R = rs_sm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double *qrow = rs_sm + P + warp * n;
  for (int e = threadIdx.x; e < P; e += RS_THREADS) R[e] = Rp[e];
  __syncthreads();
  double res = 0.0, ref = 0.0;
  const int64_t wpb = RS_THREADS / 32;
  for (int64_t i = (int64_t)blockIdx.x * wpb + warp; i < m; i += (int64_t)gridDim.x * wpb) {
    for (int j = lane; j < n; j += 32) qrow[j] = Q[i * ldq + j];
    __syncwarp();
    for (int k = lane; k < n; k += 32) {
      double y = 0.0;
      for (int j = 0; j <= k; ++j) y = fma(qrow[j], R[k * (k + 1) / 2 + j], y);
      const double v = V[i * ldv + k], d = v - y;
      res = fma(d, d, res);
      ref = fma(v, v, ref);
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) {
    res += __shfl_xor_sync(0xffffffffu, res, o);
    ref += __shfl_xor_sync(0xffffffffu, ref, o);
  }
  if (lane == 0) {
    atomicAdd(&sums[0], res);
    atomicAdd(&sums[1], ref);
  }
}

}  // namespace

cudaError_t launch_resid_f64(const double *V, int64_t ldv, const double *Q, int64_t ldq, int64_t m, int64_t n,
                             const double *Rpacked, double *sums, int num_sms, const DevStatus *st, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)(n * (n + 1) / 2 + (RS_THREADS / 32) * n);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_resid_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, RS_THREADS / 32), 4 * (int64_t)num_sms));
  k_resid_f64<<<(unsigned)blocks, RS_THREADS, smem, s>>>(V, ldv, Q, ldq, m, (int)n, Rpacked, sums, st);
  return cudaGetLastError();
}

// Largest |eigenvalue| of A = G - I (G symmetric, given by its packed upper triangle) by cyclic
// Jacobi rotations (Jacobi 1846; the two-sided rotation that zeroes a_pq with
// t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), theta = (a_qq - a_pp) / (2 a_pq)), sweeping
// until the off-diagonal mass is negligible against the diagonal.
double sym_identity_gap2(const double *Gp, int n) {
  std::vector<double> A((size_t)n * n);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k <= j; ++k) {
      const double g = Gp[j * (j + 1) / 2 + k] - (k == j ? 1.0 : 0.0);
      A[(size_t)k * n + j] = g;
      A[(size_t)j * n + k] = g;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int p = 0; p < n; ++p) {
      diag += A[(size_t)p * n + p] * A[(size_t)p * n + p];
      for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    }
    if (off == 0.0 || off <= 1e-36 * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + c * aqk;
        }
      }
  }
  double mx = 0.0;
  for (int p = 0; p < n; ++p) mx = fmax(mx, fabs(A[(size_t)p * n + p]));
  return mx;
}

}  // namespace rq
