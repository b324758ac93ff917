// rowpass_df.cu -- the row passes in double-float arithmetic (RANDQR_F32X2).
//
// GB300 issues FP32 FMAs ~70x faster than FP64 FMAs (69.5 vs 1.0 TFLOP/s measured), so
// the triangular solves and the Gram run here on pairs of FP32 numbers (hi + lo, a ~48-bit
// significand; Dekker 1971, Knuth's TwoSum, FMA-based TwoProd).  The Householder QR of the
// sketch, the Cholesky and R = R_c R_s stay FP64 (small.cu).
//
// Storage: V and the final Q are FP64; the intermediate W = V R_s^{-1} is stored in the Q
// buffer as (hi, lo) float pairs -- same 8 bytes per entry -- so W never round-trips
// through FP64.  FP64 <-> pair conversions are done with integer bit manipulation and
// FP32 instructions only: on this GPU an FP64 conversion or add would run on the slow
// FP64 pipe.
//
// Range: entries are represented exactly to ~47 bits while |x| >= 2^-74; smaller
// magnitudes keep at least FP32 precision down to 2^-126 and flush to zero below it.
#include <algorithm>

#include "common.cuh"

namespace rq {

// ---------------------------------------------------------------------------------------
// FP64 -> (hi, lo) without FP64 instructions.  hi keeps the top 24 significant bits
// (truncated), lo is the remaining 29-bit tail rounded to FP32 by an integer->float
// conversion and scaled by an exactly representable power of two.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float2 d2df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);  // biased FP64 exponent
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFULL;
  if (e <= 896) return make_float2(__uint_as_float(sign), 0.0f);           // |x| < 2^-126
  if (e >= 1151) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.0f);  // overflow
  const float hi = __uint_as_float(sign | ((unsigned int)(e - 896) << 23) | (unsigned int)(mant >> 29));
  const unsigned int tail = (unsigned int)(mant & 0x1FFFFFFFULL);  // 29 bits, weight 2^(e-1075)
  const int pe = e - 1075 + 127;                                    // biased exponent of 2^(e-1075)
  float lo = 0.0f;
  if (tail != 0 && pe > 0) {
    lo = __uint2float_rn(tail) * __uint_as_float((unsigned int)pe << 23);
    lo = __uint_as_float(__float_as_uint(lo) | sign);
  }
  return make_float2(hi, lo);
}

// (hi, lo) -> FP64 without FP64 instructions: assemble hi's FP64 bit pattern and add lo's
// significand, aligned to hi's FP64 ulp (truncated below it), in 64-bit integer arithmetic.
__device__ __forceinline__ double df2d(float hi, float lo) {
  const unsigned int hb = __float_as_uint(hi), lb = __float_as_uint(lo);
  const int eh = (int)((hb >> 23) & 0xff);
  if (eh == 0) return __longlong_as_double((long long)((unsigned long long)(hb >> 31) << 63));
  if (eh == 255) return __longlong_as_double((long long)(((unsigned long long)(hb >> 31) << 63) | 0x7ff0000000000000ULL));
  long long M = (long long)((1ULL << 52) | ((unsigned long long)(hb & 0x7fffff) << 29));
  int E = eh - 127;  // value = M * 2^(E - 52)
  const int el = (int)((lb >> 23) & 0xff);
  if (el != 0 && el != 255) {
    const long long ml = (long long)((1u << 23) | (lb & 0x7fffff));  // value = ml * 2^(el-127-23)
    const int s = (el - 127 - 23) - (E - 52);                       // shift into hi's units
    long long add = 0;
    if (s >= 0)
      add = (s < 40) ? (ml << s) : 0;
    else
      add = (-s < 63) ? (ml >> (-s)) : 0;
    if ((lb >> 31) != (hb >> 31)) add = -add;
    M += add;
    if (M >= (1LL << 53)) { M >>= 1; ++E; }
    while (M > 0 && M < (1LL << 52)) { M <<= 1; --E; }
  }
  if (M <= 0) return 0.0;
  const unsigned long long out = ((unsigned long long)(hb >> 31) << 63) |
                                 ((unsigned long long)(E + 1023) << 52) |
                                 ((unsigned long long)M & 0xFFFFFFFFFFFFFULL);
  return __longlong_as_double((long long)out);
}

// s -= a * b with s kept as an unnormalised pair (sh, sl).
__device__ __forceinline__ void df_fms(float &sh, float &sl, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float t = __fsub_rn(sh, p);
  const float z = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(-p, z));
  sl = __fadd_rn(__fsub_rn(sl, e), err);
  sh = t;
}

// s += a * b.
__device__ __forceinline__ void df_fma(float &sh, float &sl, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float t = __fadd_rn(sh, p);
  const float z = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
  sl = __fadd_rn(__fadd_rn(sl, e), err);
  sh = t;
}

__device__ __forceinline__ float2 df_norm(float sh, float sl) {
  const float h = __fadd_rn(sh, sl);
  return make_float2(h, __fsub_rn(sl, __fsub_rn(h, sh)));
}

// (sh + sl) * r, normalised.
__device__ __forceinline__ float2 df_mul(float sh, float sl, float2 r) {
  const float p = sh * r.x;
  float e = __fmaf_rn(sh, r.x, -p);
  e = __fmaf_rn(sh, r.y, e);
  e = __fmaf_rn(sl, r.x, e);
  return df_norm(p, e);
}

// ---------------------------------------------------------------------------------------
// Triangular factor in pair form: packed upper R and 1/r_jj, from the FP64 packed factor.
// ---------------------------------------------------------------------------------------
__global__ void k_pack_df(const double *Rp, int n, float2 *Rdf, float2 *rinv, const DevStatus *st) {
  if (status_failed(st)) return;
  const int P = n * (n + 1) / 2;
  for (int e = threadIdx.x; e < P; e += blockDim.x) Rdf[e] = d2df(Rp[e]);
  for (int j = threadIdx.x; j < n; j += blockDim.x) rinv[j] = d2df(1.0 / Rp[tri_idx(j, j)]);
}

// ---------------------------------------------------------------------------------------
// Y = X R^{-1} per row by forward substitution in pair arithmetic, one thread per row, two
// independent partial sums (even / odd k) per dot product to overlap the dependent chains.
// IN_F64: X is FP64 (else pairs); OUT_F64: Y is FP64 (else pairs).  X and Y may alias.
// ---------------------------------------------------------------------------------------
constexpr int DF_ROWS = 128;

template <bool IN_F64, bool OUT_F64>
__global__ void __launch_bounds__(DF_ROWS) k_trsm_df(const void *X, int64_t ldx, void *Y, int64_t ldy,
                                                     int64_t m, int n, const float2 *__restrict__ Rg,
                                                     const float2 *__restrict__ rinvg,
                                                     const DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ float2 smf[];
  const int P = n * (n + 1) / 2;
  const int ld = (n & 1) ? n : n + 1;
  float2 *R = smf;
  float2 *rinv = R + P;
  float2 *T = rinv + n;
  const int tid = threadIdx.x;
  for (int e = tid; e < P; e += blockDim.x) R[e] = Rg[e];
  for (int j = tid; j < n; j += blockDim.x) rinv[j] = rinvg[j];
  __syncthreads();
  for (int64_t row0 = (int64_t)blockIdx.x * DF_ROWS; row0 < m; row0 += (int64_t)gridDim.x * DF_ROWS) {
    const int rows = (int)imin64(DF_ROWS, m - row0);
    for (int e = tid; e < rows * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      if (IN_F64)
        T[r * ld + c] = d2df(((const double *)X)[(row0 + r) * ldx + c]);
      else
        T[r * ld + c] = ((const float2 *)X)[(row0 + r) * ldx + c];
    }
    __syncthreads();
    if (tid < rows) {
      float2 *w = T + tid * ld;
      for (int j = 0; j < n; ++j) {
        const float2 *rc = R + j * (j + 1) / 2;
        float ah = w[j].x, al = w[j].y, bh = 0.f, bl = 0.f;
        int k = 0;
        for (; k + 1 < j; k += 2) {
          df_fms(ah, al, w[k], rc[k]);
          df_fms(bh, bl, w[k + 1], rc[k + 1]);
        }
        if (k < j) df_fms(ah, al, w[k], rc[k]);
        // combine the two partial sums: (ah + al) + (bh + bl)
        const float t = __fadd_rn(ah, bh);
        const float z = __fsub_rn(t, ah);
        const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(t, z)), __fsub_rn(bh, z));
        const float l = __fadd_rn(__fadd_rn(al, bl), err);
        const float2 s = df_norm(t, l);
        w[j] = df_mul(s.x, s.y, rinv[j]);
      }
    }
    __syncthreads();
    for (int e = tid; e < rows * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      const float2 v = T[r * ld + c];
      if (OUT_F64)
        ((double *)Y)[(row0 + r) * ldy + c] = df2d(v.x, v.y);
      else
        ((float2 *)Y)[(row0 + r) * ldy + c] = v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// G = W^T W from pairs.  Each thread owns one 4 x 4 block (jb, kb), kb <= jb, of the upper
// triangle and keeps 16 pair accumulators in registers across its CTA's rows; per row it
// loads 4 + 4 entries for 16 pair-FMAs.  The sums go to FP64 and into G with one atomic each.
// ---------------------------------------------------------------------------------------
constexpr int DFG_TILE = 32;

__global__ void k_gram_df(const float2 *__restrict__ W, int64_t ldw, int64_t m, int n,
                          int64_t rows_per_cta, double *Gp, const DevStatus *st) {
  if (status_failed(st)) return;
  __shared__ float2 T[DFG_TILE * 132];
  const int nb = (n + 3) / 4;
  const int ld = 4 * nb + 1;  // padded row, odd stride in 8-byte words
  const int tid = threadIdx.x;
  const int nblk = nb * (nb + 1) / 2;
  int jb = 0, kb = 0;
  const bool active = tid < nblk;
  if (active) {
    int t = tid;
    jb = 0;
    while (t > jb) { t -= jb + 1; ++jb; }
    kb = t;  // kb <= jb
  }
  float ah[4][4], al[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { ah[a][b] = 0.f; al[a][b] = 0.f; }
  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  for (int64_t row0 = r_begin; row0 < r_end; row0 += DFG_TILE) {
    const int rows = (int)imin64(DFG_TILE, r_end - row0);
    __syncthreads();
    for (int e = tid; e < rows * ld; e += blockDim.x) {
      const int r = e / ld, c = e - r * ld;
      T[e] = (c < n) ? W[(row0 + r) * ldw + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (active) {
      for (int r = 0; r < rows; ++r) {
        const float2 *t = T + r * ld;
        float2 x[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) { x[a] = t[4 * kb + a]; y[a] = t[4 * jb + a]; }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) df_fma(ah[a][b], al[a][b], x[a], y[b]);
      }
    }
  }
  if (!active) return;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int k = 4 * kb + a, j = 4 * jb + b;  // G(k, j), need k <= j < n
      if (j < n && k <= j) atomicAdd(Gp + tri_idx(k, j), (double)ah[a][b] + (double)al[a][b]);
    }
}

cudaError_t launch_pack_df(const double *Rp, int64_t n, float2 *Rdf, float2 *rinv,
                           const DevStatus *st, cudaStream_t s) {
  k_pack_df<<<1, 256, 0, s>>>(Rp, (int)n, Rdf, rinv, st);
  return cudaGetLastError();
}

cudaError_t launch_trsm_df(const void *X, bool x_f64, int64_t ldx, void *Y, bool y_f64, int64_t ldy,
                           int64_t m, int64_t n, const float2 *Rdf, const float2 *rinv, int num_sms,
                           const DevStatus *st, cudaStream_t s) {
  const int ld = (n & 1) ? (int)n : (int)n + 1;
  const size_t smem = sizeof(float2) * ((size_t)(n * (n + 1) / 2) + n + (size_t)DF_ROWS * ld);
  int per_sm = std::max(1, (int)((220 * 1024) / smem));
  per_sm = std::min(per_sm, 8);
  const int64_t tiles = ceil_div(m, DF_ROWS);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms * per_sm));
  cudaError_t e;
#define RQ_TRSM_DF(A, B)                                                                        \
  e = cudaFuncSetAttribute(k_trsm_df<A, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
  if (e != cudaSuccess) return e;                                                               \
  k_trsm_df<A, B><<<blocks, DF_ROWS, smem, s>>>(X, ldx, Y, ldy, m, (int)n, Rdf, rinv, st);
  if (x_f64 && !y_f64) {
    RQ_TRSM_DF(true, false)
  } else if (!x_f64 && y_f64) {
    RQ_TRSM_DF(false, true)
  } else if (x_f64 && y_f64) {
    RQ_TRSM_DF(true, true)
  } else {
    RQ_TRSM_DF(false, false)
  }
#undef RQ_TRSM_DF
  return cudaGetLastError();
}

cudaError_t launch_gram_df(const float2 *W, int64_t ldw, int64_t m, int64_t n, double *Gpacked,
                           int num_sms, const DevStatus *st, cudaStream_t s) {
  const int nb = (int)((n + 3) / 4);
  const int nblk = nb * (nb + 1) / 2;
  const int threads = std::max(32, (nblk + 31) / 32 * 32);
  const int per_sm = std::max(1, std::min(8, 1024 / threads));
  const int blocks_target = num_sms * per_sm;
  const int64_t rows_per_cta =
      std::max<int64_t>(DFG_TILE, ceil_div(ceil_div(m, blocks_target), DFG_TILE) * DFG_TILE);
  const int blocks = (int)ceil_div(m, rows_per_cta);
  k_gram_df<<<blocks, threads, 0, s>>>(W, ldw, m, (int)n, rows_per_cta, Gpacked, st);
  return cudaGetLastError();
}

}  // namespace rq
