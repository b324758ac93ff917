// gram_split.cu -- G = W^T W (Algorithm 2 step 1, the Gram of each Cholesky pass) for n <= 64
// from exact split products on the tensor cores: the kernel and its launch.  The CTA body, its
// number format and its warp roles are in gram_split_body.cuh.
#include "gram_split_body.cuh"

namespace rq {

template <int NP, bool IN_DF>
__global__ void __launch_bounds__(GS_THREADS, 1)
    k_gram_split(const void *Win, int64_t ldw, int64_t m, int n, double *Gp, int64_t rows_per_cta,
                 int load_mode, DevStatus *st) {
  if (status_failed(st)) return;
  gram_split_cta<NP, IN_DF, false>(Win, ldw, m, n, Gp, rows_per_cta, load_mode, st, (int)blockIdx.x, 0u);
}

bool gram_split_supported(int64_t n) { return n >= 1 && n <= 64; }

namespace {
template <int NP, bool IN_DF>
cudaError_t launch_gram_split_t(const void *W, int64_t ldw, int64_t m, int64_t n, double *Gpacked, int num_sms,
                                DevStatus *st, cudaStream_t s) {
  using C = GsCfg<NP>;
  int64_t ctas = std::min<int64_t>(ceil_div(m, C::GROUP), (int64_t)num_sms);
  const int64_t rows_per_cta = ceil_div(ceil_div(m, ctas), C::GROUP) * C::GROUP;
  ctas = ceil_div(m, rows_per_cta);
  const bool aligned = ((uintptr_t)W & 15) == 0;
  const int load_mode = (aligned && n == NP && ldw == NP) ? GLOAD_BLOCK
                        : (aligned && (n * 8) % 16 == 0 && (ldw * 8) % 16 == 0) ? GLOAD_ROWS
                                                                                 : GLOAD_PLAIN;
  cudaError_t e = cudaFuncSetAttribute(k_gram_split<NP, IN_DF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM);
  if (e != cudaSuccess) return e;
  k_gram_split<NP, IN_DF><<<(unsigned)ctas, GS_THREADS, C::SMEM, s>>>(W, ldw, m, (int)n, Gpacked, rows_per_cta,
                                                                      load_mode, st);
  return cudaGetLastError();
}

template <bool IN_DF>
cudaError_t launch_gram_split_w(const void *W, int64_t ldw, int64_t m, int64_t n, double *Gpacked, int num_sms,
                                DevStatus *st, cudaStream_t s) {
  if (n <= 16) return launch_gram_split_t<16, IN_DF>(W, ldw, m, n, Gpacked, num_sms, st, s);
  if (n <= 32) return launch_gram_split_t<32, IN_DF>(W, ldw, m, n, Gpacked, num_sms, st, s);
  return launch_gram_split_t<64, IN_DF>(W, ldw, m, n, Gpacked, num_sms, st, s);
}
}  // namespace

cudaError_t launch_gram_split(const void *W, bool in_df, int64_t ldw, int64_t m, int64_t n, double *Gpacked,
                              int num_sms, DevStatus *st, cudaStream_t s) {
  if (!gram_split_supported(n)) return cudaErrorInvalidValue;
  return in_df ? launch_gram_split_w<true>(W, ldw, m, n, Gpacked, num_sms, st, s)
               : launch_gram_split_w<false>(W, ldw, m, n, Gpacked, num_sms, st, s);
}

}  // namespace rq

