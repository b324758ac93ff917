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
#include "df.cuh"

namespace rq {

// ---------------------------------------------------------------------------------------
// Triangular factor in pair form, in column blocks of DF_JB = 16: n is padded to n_pad (a
// multiple of DF_JB) and block b (columns 16b .. 16b+15) stores, for every row k < 16b + 16,
// its 16 entries contiguously: Rb[128 b (b+1) + 16 k + c] = R(k, 16b + c), zero where
// k > 16b + c or the column is padding.  rinv[j] = 1/r_jj, zero on padding, so padded
// columns solve to zero without a branch.
// ---------------------------------------------------------------------------------------
constexpr int DF_JB = 16;

__host__ __device__ __forceinline__ int df_npad(int n) { return (n + DF_JB - 1) / DF_JB * DF_JB; }
__host__ __device__ __forceinline__ int df_block_off(int b) { return DF_JB * DF_JB / 2 * b * (b + 1); }
__host__ __device__ __forceinline__ int df_rb_size(int n) {
  const int nb = df_npad(n) / DF_JB;
  return df_block_off(nb);
}

__global__ void k_pack_df(const double *Rp, int n, float2 *Rb, float2 *rinv, const DevStatus *st) {
  if (status_failed(st)) return;
  const int np = df_npad(n), total = df_rb_size(n);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int b = 0;
    while (df_block_off(b + 1) <= e) ++b;
    const int local = e - df_block_off(b);
    const int k = local / DF_JB, j = DF_JB * b + local % DF_JB;
    Rb[e] = (j < n && k <= j) ? d2df(Rp[tri_idx(k, j)]) : make_float2(0.f, 0.f);
  }
  for (int j = threadIdx.x; j < np; j += blockDim.x)
    rinv[j] = (j < n) ? d2df(1.0 / Rp[tri_idx(j, j)]) : make_float2(0.f, 0.f);
}

// ---------------------------------------------------------------------------------------
// Y = X R^{-1} by blocked forward substitution in pair arithmetic (the blocked form of the
// row-wise solve: diagonal blocks by substitution, never by an explicit inverse).  A CTA
// holds a tile of DF_ROWS rows in shared memory.  For column block J (16 columns):
//   (1) update  T[:, J] -= T[:, <J] R[<J, J]  -- a pair-arithmetic GEMM: warp w owns
//       columns 16J + 4w .. +3, lane l owns rows l, l+32, l+64, l+96, so each thread keeps
//       16 independent accumulators, reads its 4 row entries (consecutive rows: distinct
//       banks) and the 4 R entries (one broadcast per warp) per k;
//   (2) solve the 16 x 16 diagonal block row by row, one thread per row.
// For every output entry the terms are taken in ascending k, as in the row-wise solve.
// IN_F64: X is FP64 (else pairs); OUT_F64: Y is FP64 (else pairs).  X and Y may alias.
// ---------------------------------------------------------------------------------------
constexpr int DF_ROWS = 128;

template <bool IN_F64, bool OUT_F64>
__global__ void __launch_bounds__(DF_ROWS) k_trsm_df(const void *X, int64_t ldx, void *Y, int64_t ldy,
                                                     int64_t m, int n, const float2 *__restrict__ Rg,
                                                     const float2 *__restrict__ rinvg,
                                                     const DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ float4 smf4[];
  const int np = df_npad(n), RB = df_rb_size(n);
  const int ld = np + 1;  // odd stride in 8-byte words
  float2 *Rb = (float2 *)smf4;
  float2 *rinv = Rb + RB;
  float2 *T = rinv + np;
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
  for (int e = tid; e < RB; e += blockDim.x) Rb[e] = Rg[e];
  for (int j = tid; j < np; j += blockDim.x) rinv[j] = rinvg[j];
  __syncthreads();
  for (int64_t row0 = (int64_t)blockIdx.x * DF_ROWS; row0 < m; row0 += (int64_t)gridDim.x * DF_ROWS) {
    const int rows = (int)imin64(DF_ROWS, m - row0);
    for (int e = tid; e < DF_ROWS * np; e += blockDim.x) {
      const int r = e / np, c = e - r * np;
      float2 v = make_float2(0.f, 0.f);
      if (c < n && r < rows) {
        if (IN_F64)
          v = d2df(((const double *)X)[(row0 + r) * ldx + c]);
        else
          v = ((const float2 *)X)[(row0 + r) * ldx + c];
      }
      T[r * ld + c] = v;
    }
    __syncthreads();
    for (int b = 0; b < np / DF_JB; ++b) {
      const int j0 = DF_JB * b;
      const float2 *rb = Rb + df_block_off(b);
      if (j0 > 0) {
        // (1) off-diagonal update of the block, 4 rows x 4 columns per thread
        const int c0 = j0 + 4 * wq;
        float ah[16], al[16];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float2 v = T[(lane + 32 * i) * ld + c0 + c];
            ah[4 * i + c] = v.x;
            al[4 * i + c] = v.y;
          }
        for (int k = 0; k < j0; ++k) {
          float2 w4[4], r4[4], a[16], bb[16];
#pragma unroll
          for (int i = 0; i < 4; ++i) w4[i] = T[(lane + 32 * i) * ld + k];
          const float4 q0 = *(const float4 *)(rb + DF_JB * k + 4 * wq);
          const float4 q1 = *(const float4 *)(rb + DF_JB * k + 4 * wq + 2);
          r4[0] = make_float2(q0.x, q0.y);
          r4[1] = make_float2(q0.z, q0.w);
          r4[2] = make_float2(q1.x, q1.y);
          r4[3] = make_float2(q1.z, q1.w);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              a[4 * i + c] = w4[i];
              bb[4 * i + c] = r4[c];
            }
          df_fms_nn<16>(ah, al, a, bb);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            T[(lane + 32 * i) * ld + c0 + c] = df_norm(ah[4 * i + c], al[4 * i + c]);
        __syncthreads();
      }
      // (2) the diagonal block, one thread per row
      {
        float2 *t = T + tid * ld + j0;
        float2 wl[DF_JB];
#pragma unroll
        for (int c = 0; c < DF_JB; ++c) {
          float sh = t[c].x, sl = t[c].y;
#pragma unroll
          for (int cc = 0; cc < c; ++cc) df_fms(sh, sl, wl[cc], rb[DF_JB * (j0 + cc) + c]);
          const float2 sn = df_norm(sh, sl);
          wl[c] = df_mul(sn.x, sn.y, rinv[j0 + c]);
        }
#pragma unroll
        for (int c = 0; c < DF_JB; ++c) t[c] = wl[c];
      }
      __syncthreads();
    }
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
  // Row r keeps column c at r*ld + (c % 4)*nb + c / 4, so the 4 entries a thread reads
  // for its block (c = 4*kb + a) sit nb apart and neighbouring threads' kb hit distinct
  // banks; the odd row stride spreads rows.
  const int ld = 4 * nb + 1;
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
  // per-tile partial sums (ph, pl) and running totals (th, tl): no pair accumulation
  // chain is longer than one tile, the totals take one accurate pair addition per tile.
  float th[16], tl[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) { th[q] = 0.f; tl[q] = 0.f; }
  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  for (int64_t row0 = r_begin; row0 < r_end; row0 += DFG_TILE) {
    const int rows = (int)imin64(DFG_TILE, r_end - row0);
    __syncthreads();
    const int wpr = 4 * nb;  // padded entries per row
    for (int e = tid; e < rows * wpr; e += blockDim.x) {
      const int r = e / wpr, c = e - r * wpr;
      T[r * ld + (c & 3) * nb + (c >> 2)] = (c < n) ? W[(row0 + r) * ldw + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (active) {
      float ph[16], pl[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) { ph[q] = 0.f; pl[q] = 0.f; }
      for (int r = 0; r < rows; ++r) {
        const float2 *t = T + r * ld;
        float2 x[4], y[4], a[16], bb[16];
#pragma unroll
        for (int i = 0; i < 4; ++i) { x[i] = t[i * nb + kb]; y[i] = t[i * nb + jb]; }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            a[4 * i + c] = make_float2(-x[i].x, -x[i].y);  // s -= (-x) y
            bb[4 * i + c] = y[c];
          }
        df_fms_nn<16>(ph, pl, a, bb);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) df_add(th[q], tl[q], ph[q], pl[q]);
    }
  }
  if (!active) return;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int k = 4 * kb + i, j = 4 * jb + c;  // G(k, j), need k <= j < n
      if (j < n && k <= j) atomicAdd(Gp + tri_idx(k, j), (double)th[4 * i + c] + (double)tl[4 * i + c]);
    }
}

size_t pack_df_elems(int64_t n) { return (size_t)df_rb_size((int)n); }
size_t pack_df_rinv_elems(int64_t n) { return (size_t)df_npad((int)n); }

cudaError_t launch_pack_df(const double *Rp, int64_t n, float2 *Rdf, float2 *rinv,
                           const DevStatus *st, cudaStream_t s) {
  k_pack_df<<<1, 256, 0, s>>>(Rp, (int)n, Rdf, rinv, st);
  return cudaGetLastError();
}

cudaError_t launch_trsm_df(const void *X, bool x_f64, int64_t ldx, void *Y, bool y_f64, int64_t ldy,
                           int64_t m, int64_t n, const float2 *Rdf, const float2 *rinv, int num_sms,
                           const DevStatus *st, cudaStream_t s) {
  const int np = df_npad((int)n);
  const size_t smem = sizeof(float2) * ((size_t)df_rb_size((int)n) + np + (size_t)DF_ROWS * (np + 1));
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
  // at most 64 tiles per CTA: the totals see at most 64 pair additions, then FP64 atomics
  const int64_t rows_per_cta = std::min<int64_t>(
      64 * DFG_TILE,
      std::max<int64_t>(DFG_TILE, ceil_div(ceil_div(m, blocks_target), DFG_TILE) * DFG_TILE));
  const int blocks = (int)ceil_div(m, rows_per_cta);
  k_gram_df<<<blocks, threads, 0, s>>>(W, ldw, m, (int)n, rows_per_cta, Gpacked, st);
  return cudaGetLastError();
}

}  // namespace rq
