// gram_tc.cu -- G = W^T W (Algorithm 2 step 1) from exact split products on the
// fifth-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// The Gram is the one dense contraction with a long reduction (K = m) on the path.  GB300
// multiplies FP64 at 1 TFLOP/s but bf16 at ~2 PFLOP/s, so W is split into integer slices
// that bf16 holds exactly and whose products the tensor cores sum exactly (the splitting
// idea of Ozaki, Ogita, Oishi & Rump; written here from that idea):
//
//   for a chunk of KC rows, column j gets a scale 2^E_j > max |W_ij|; the fixed-point value
//   X_ij = trunc(|W_ij| 2^(56 - E_j)) (< 2^56) is cut into eight 7-bit digits
//   a_s = (X >> (49 - 7 s)) & 127 carrying the sign of W_ij, so W_ij = 2^(E_j - 56) sum_s a_s 2^(49 - 7 s)
//   up to 2^(E_j - 56).  Then  sum_rows W_ij W_ik = 2^(E_j + E_k) sum_g 2^(-14 - 7 g) C_g(j, k),
//   C_g = sum_{s + t = g} sum_rows a_s(j) a_t(k), keeping g <= 7 (the dropped groups are
//   below 2^-56 of the chunk's column scales).
//
// Every C_g is a sum of at most 4 x KC products of magnitude < 2^14 (< 2^23 in total), an
// integer that FP32 accumulation holds exactly, so the tensor cores add the slice products
// with no rounding.  Each chunk's eight groups are read from tensor memory, combined in
// pair arithmetic, scaled by 2^(E_j + E_k) and added into per-thread pair sums (spilled
// into second-level pair totals every 8 chunks); one FP64 atomic per entry at the end.
//
// Pipeline per CTA (one per SM: the eight regions fill the 512 tensor-memory columns):
// the rows of a chunk arrive in shared memory by bulk asynchronous copies (the TMA engine,
// completion on an mbarrier); all 8 warps derive the column scales and the slices from
// shared memory; one thread then starts the copy of the next chunk and issues the MMAs;
// after the MMAs complete (second mbarrier) the warps read the accumulators back.
//
// Layout: an A tile holds 128 rows of slice-planes (SP = 128 / NP slices of NP padded
// columns each), K-major in 8 x 16-byte core matrices without swizzle.  The B operand of
// slice t is a 64-row window of the same tiles, so one copy of the slices serves both
// operands.  Region g' of tensor memory (64 columns) accumulates all (tile, slice) pairs with
// first-slice + t = g'; lane block q of that region then holds group g' + q.
#include <cuda_bf16.h>

#include "common.cuh"
#include "df.cuh"

namespace rq {

namespace {

constexpr int OZ_S = 8;          // slices per value
constexpr int OZ_THREADS = 256;  // 8 warps; warps w and w + 4 share TMEM lane quarter w
constexpr uint32_t OZ_TMEM_COLS = 512;
constexpr int OZ_MAX_WAIT = 1 << 24;
constexpr int OZ_STAGE_BYTES = 64 * 1024;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major, no swizzle: lbo = byte step between core matrices
// along K, sbo = byte step between 8-row groups.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: kind::f16, bf16 A and B (K-major), FP32 D, M x N.
__device__ __forceinline__ uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit = OZ_MAX_WAIT) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
  return done != 0;
}

// Bulk asynchronous copy global -> shared (TMA engine), completion counted in bytes on mbar.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}

// 8 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(addr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n"); }

// Exponent field of an element rebased to the FP64 bias; 0 for zero / subnormal.
template <bool IN_DF>
__device__ __forceinline__ int expfield(const void *p) {
  if (IN_DF) {
    const int ef = (__float_as_uint(((const float2 *)p)->x) >> 23) & 0xff;
    return ef ? ef - 127 + 1023 : 0;
  }
  return (int)(((unsigned long long)__double_as_longlong(*(const double *)p) >> 52) & 0x7ff);
}

// Signed 56-bit fixed point of a float's value relative to 2^E (truncated).
__device__ __forceinline__ long long fix_f32(float f, int E) {
  const unsigned int b = __float_as_uint(f);
  const int ef = (b >> 23) & 0xff;
  if (ef == 0) return 0;
  const long long mant = (long long)((b & 0x7fffff) | 0x800000);
  const int sh = (ef - 127) + 33 - E;  // value = mant 2^(ef-127-23); times 2^(56-E)
  long long x = sh >= 0 ? (sh < 40 ? (mant << sh) : 0) : (-sh < 63 ? (mant >> -sh) : 0);
  return (b >> 31) ? -x : x;
}

template <bool IN_DF>
__device__ __forceinline__ long long fixpt(const void *p, int E) {
  if (IN_DF) {
    const float2 v = *(const float2 *)p;
    return fix_f32(v.x, E) + fix_f32(v.y, E);
  }
  const unsigned long long b = (unsigned long long)__double_as_longlong(*(const double *)p);
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef == 0) return 0;
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
  const int sh = (ef - 1023) + 4 - E;  // value = mant 2^(ef-1023-52); times 2^(56-E)
  long long x = sh >= 0 ? (sh < 8 ? (mant << sh) : 0) : (-sh < 63 ? (mant >> -sh) : 0);
  return (b >> 63) ? -x : x;
}

// bf16 bits of a small integer (|a| < 2^22), exactly, with FP32-pipe and integer ops only.
__device__ __forceinline__ uint32_t int_to_bf16_bits(int a) {
  const float f = __int_as_float(0x4B400000 + a) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}

__device__ __forceinline__ float pow2f(int e) {  // 2^e, e clamped to [-126, 127]
  e = max(min(e, 127), -126);
  return __uint_as_float((uint32_t)(e + 127) << 23);
}

}  // namespace

// One CTA per SM, OZ_THREADS threads; grid.y = column pass (64 columns each).
// bulk: rows of a chunk are contiguous in global memory (ldw == n, 16-byte multiples).
template <bool IN_DF>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_gram_oz(const void *__restrict__ W, int64_t ldw, int64_t m, int n, int np, int kc,
              int64_t rows_per_cta, bool bulk, double *Gp, DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ __align__(1024) uint8_t oz_smem[];
  const int sp = 128 / np, nt = OZ_S / sp;
  const size_t tile_bytes = (size_t)128 * kc * 2;
  uint8_t *A = oz_smem;                                  // nt tiles
  uint8_t *stage = oz_smem + nt * tile_bytes;            // kc x n elements, 8 bytes each
  int *colexp = (int *)(stage + OZ_STAGE_BYTES);         // np ints
  uint64_t *bars = (uint64_t *)(colexp + 128);           // [0] copy, [1] MMA
  uint32_t *tmem_slot = (uint32_t *)(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pass = blockIdx.y;
  const uint32_t copy_bar = smem_addr(&bars[0]), mma_bar = smem_addr(&bars[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(copy_bar));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mma_bar));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  const int64_t nchunks = r_begin < r_end ? (r_end - r_begin + kc - 1) / kc : 0;

  auto issue_copy = [&](int64_t row0) {
    const int rows = (int)imin64(kc, r_end - row0);
    const uint32_t bytes = (uint32_t)rows * (uint32_t)n * 8u;
    mbar_expect_tx(copy_bar, bytes);
    const uint8_t *src = (const uint8_t *)W + (size_t)row0 * (size_t)ldw * 8;
    for (uint32_t off = 0; off < bytes; off += 16384) {
      const uint32_t b = bytes - off < 16384 ? bytes - off : 16384;
      bulk_copy(smem_addr(stage) + off, src + off, b, copy_bar);
    }
  };
  if (bulk && tid == 0 && nchunks > 0) issue_copy(r_begin);

  // slicing role: column c, row pairs p = h + tpc i
  const int tpc = OZ_THREADS / np, c = tid % np, h = tid / np;
  const int npairs = kc / (2 * tpc);
  // flush role: TMEM lane L (tile row (q, j)), column half of this pass's 64
  const int L = 32 * (warp & 3) + lane, q = L / np, j = L % np, half = warp >> 2;
  const uint32_t lbo = 128, sbo = (uint32_t)(kc / 8) * 128;
  const uint32_t idesc = umma_idesc(128, 64);

  float ah[32], al[32], th[32], tl[32];  // chunk-sum pairs and second-level totals
#pragma unroll
  for (int k = 0; k < 32; ++k) { ah[k] = 0.f; al[k] = 0.f; th[k] = 0.f; tl[k] = 0.f; }

  bool ok = true;
  for (int64_t ci = 0; ci < nchunks && ok; ++ci) {
    const int64_t row0 = r_begin + ci * kc;
    const int rows = (int)imin64(kc, r_end - row0);
    const uint32_t parity = (uint32_t)(ci & 1);
    // ---- the chunk in shared memory
    if (tid < np) colexp[tid] = 0;
    if (bulk) {
      if (!__syncthreads_and(mbar_wait(copy_bar, parity, wait_bound(st, OZ_MAX_WAIT)))) {
        ok = false;
        if (tid == 0) status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
        mbar_wait(copy_bar, parity);  // second bounded wait for the copy in flight
        break;
      }
    } else {
      for (int e = tid; e < rows * n; e += OZ_THREADS) {
        const int r = e / n, cc = e - r * n;
        ((unsigned long long *)stage)[e] =
            ((const unsigned long long *)W)[(row0 + r) * ldw + cc];
      }
      __syncthreads();
    }
    // ---- column scales
    {
      int mx = 0;
      if (c < n)
        for (int i = 0; i < npairs; ++i) {
          const int r = 2 * (h + tpc * i);
          if (r < rows) mx = max(mx, expfield<IN_DF>(stage + ((size_t)r * n + c) * 8));
          if (r + 1 < rows) mx = max(mx, expfield<IN_DF>(stage + ((size_t)(r + 1) * n + c) * 8));
        }
      atomicMax(&colexp[c], mx);
    }
    __syncthreads();
    const int Ec = max(colexp[c] - 1023 + 1, -100);
    if (Ec > 100) status_fail(st, RANDQR_ERR_NONFINITE, 0, 0);
    // ---- slices into the A tiles (bf16 pairs along K)
    for (int i = 0; i < npairs; ++i) {
      const int k = 2 * (h + tpc * i);  // even K index within the chunk
      long long x[2];
#pragma unroll
      for (int u = 0; u < 2; ++u)
        x[u] = (c < n && k + u < rows) ? fixpt<IN_DF>(stage + ((size_t)(k + u) * n + c) * 8, Ec) : 0;
#pragma unroll
      for (int s = 0; s < OZ_S; ++s) {
        uint32_t bits[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const unsigned long long ax = (unsigned long long)(x[u] < 0 ? -x[u] : x[u]);
          int a = (int)((ax >> (49 - 7 * s)) & (s == 0 ? 255 : 127));
          bits[u] = int_to_bf16_bits(x[u] < 0 ? -a : a);
        }
        const int a_tile = s / sp, R = (s % sp) * np + c;
        const int off = ((R >> 3) * (kc >> 3) + (k >> 3)) * 64 + (R & 7) * 8 + (k & 7);
        *(uint32_t *)(A + a_tile * tile_bytes + (size_t)off * 2) = bits[0] | (bits[1] << 16);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n");
    __syncthreads();
    // ---- next chunk's copy, then the slice products
    if (tid == 0) {
      if (bulk && ci + 1 < nchunks) issue_copy(row0 + kc);
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t abase = smem_addr(A);
      for (int g = 0; g < OZ_S; ++g) {
        uint32_t accum = 0;
        for (int a = 0; a * sp <= g && a < nt; ++a) {
          const int t = g - a * sp;
          const int bt = t / sp, R0 = (t % sp) * np + 64 * pass;
          const uint64_t ad0 = umma_desc(abase + a * (uint32_t)tile_bytes, lbo, sbo);
          const uint64_t bd0 = umma_desc(abase + bt * (uint32_t)tile_bytes + (uint32_t)(R0 >> 3) * sbo, lbo, sbo);
          for (int kk = 0; kk < kc / 16; ++kk) {
            // +256 bytes per K step: 16 in the descriptor's address field
            umma_bf16(tmem + (uint32_t)(g * 64), ad0 + (uint64_t)(kk * 16), bd0 + (uint64_t)(kk * 16),
                      idesc, accum);
            accum = 1;
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          mma_bar));
    }
    if (!__syncthreads_and(mbar_wait(mma_bar, parity, wait_bound(st, OZ_MAX_WAIT)))) {
      ok = false;
      if (tid == 0) status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
      mbar_wait(mma_bar, parity);  // second bounded wait for the work in flight
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    // ---- flush: lane L, columns 32*half .. +31 of this pass, 8 at a time
    {
      const int Ej = max(colexp[j] - 1023 + 1, -100);
#pragma unroll
      for (int c8 = 0; c8 < 4; ++c8) {
        uint32_t v[OZ_S][8];
#pragma unroll
        for (int g = 0; g < OZ_S; ++g)
          tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(g * 64 + 32 * half + 8 * c8), v[g]);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float sh = 0.f, sl = 0.f;
#pragma unroll
          for (int g = 0; g < OZ_S; ++g) {  // exact terms, TwoSum into (sh, sl)
            const float tv = __uint_as_float(v[g][i]) * pow2f(-14 - 7 * (g + q));
            const float t = __fadd_rn(sh, tv);
            const float z = __fsub_rn(t, sh);
            sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(tv, z)));
            sh = t;
          }
          const int kk = 8 * c8 + i;
          const int k = 64 * pass + 32 * half + kk;
          const float sc = pow2f(Ej + max(colexp[k] - 1023 + 1, -100));
          df_add(ah[kk], al[kk], sh * sc, sl * sc);
        }
      }
      if ((ci & 7) == 7 || ci + 1 == nchunks) {
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
          df_add(th[kk], tl[kk], ah[kk], al[kk]);
          ah[kk] = 0.f;
          al[kk] = 0.f;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
  }
  // ---- results: G(j, k) for k >= j within this pass, one atomic each
  if (ok && j < n) {
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
      const int k = 64 * pass + 32 * half + kk;
      if (k >= j && k < n) atomicAdd(Gp + tri_idx(j, k), (double)th[kk] + (double)tl[kk]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(OZ_TMEM_COLS));
}

bool gram_oz_supported(int64_t n) { return n >= 1 && n <= 128; }

cudaError_t launch_gram_oz(const void *W, bool in_df, int64_t ldw, int64_t m, int64_t n,
                           double *Gpacked, bool acc_f64, int num_sms, DevStatus *st,
                           cudaStream_t s) {
  (void)acc_f64;  // both precisions accumulate chunk sums as pairs (see the file comment)
  const int np = n <= 64 ? 64 : 128;
  const int kc = np == 64 ? 128 : 64;  // kc * n * 8 <= 64 KB of staging
  const int sp = 128 / np, nt = OZ_S / sp;
  const size_t smem = (size_t)nt * 128 * kc * 2 + OZ_STAGE_BYTES + 128 * sizeof(int) + 32;
  const int passes = np / 64;
  int64_t ctas = std::min<int64_t>(ceil_div(m, kc), (int64_t)num_sms);
  const int64_t rows_per_cta = ceil_div(ceil_div(m, ctas), kc) * kc;
  ctas = ceil_div(m, rows_per_cta);
  const bool bulk = (ldw == n) && ((n * 8) % 16 == 0) && (((uintptr_t)W & 15) == 0);
  dim3 grid((unsigned)ctas, (unsigned)passes);
  cudaError_t e;
  if (in_df) {
    e = cudaFuncSetAttribute(k_gram_oz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_oz<true><<<grid, OZ_THREADS, smem, s>>>(W, ldw, m, (int)n, np, kc, rows_per_cta, bulk, Gpacked, st);
  } else {
    e = cudaFuncSetAttribute(k_gram_oz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_oz<false><<<grid, OZ_THREADS, smem, s>>>(W, ldw, m, (int)n, np, kc, rows_per_cta, bulk, Gpacked, st);
  }
  return cudaGetLastError();
}

}  // namespace rq
