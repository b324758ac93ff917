// sketch_tc.cu -- C += A B for a dense A (M x K, row-major) and B (K x n, row-major, n <= 64)
// from exact split products on the tensor cores: the Gaussian sketch Ws = S2 W1 of Sec. 3
// (S2 the s2 x s1 Gaussian or Rademacher matrix, W1 = S1 V the CountSketch output), and
// Ws = S2 V of the single-Gaussian sketch.
//
// K is cut into chunks of 64.  Within a chunk, row i of A gets a scale 2^E_i > max_k |a_ik| and
// column j of B a scale 2^F_j > max_k |b_kj|; a_ik = 2^(E_i - 54) X_ik up to truncation with the
// integer X_ik written in seven balanced byte digits d_s (tc.cuh; s = 0 the leading digit), and
// the same for b_kj with digits e_t.  The pairs s + t <= 7 are kept and gathered by g = s + t
// into eight regions of tensor memory,
//   D_g(i, j) = sum_{s + t = g} sum_{k in chunk} d_s(i, k) e_t(k, j),
// and the chunk adds 2^(E_i + F_j - 56) T_ij / 2^12 to c_ij, T_ij = sum_g 2^(8 (7 - g)) D_g(i, j).
// A chunk of 64 keeps every region within the bounds tc::recombine_b8 needs (at most 2^22 for
// g <= 4, below 2^23 above: a digit product is at most 2^14, at most 2^13 with a leading
// digit).  Truncation and the dropped pairs weigh about 2^-53 of 2^(E_i + F_j) per term, the
// size of an FP64 product's rounding relative to the chunk's largest entries of row i and
// column j.  With integer B and entries of A that are signed powers of two (+-1, the identity)
// every step is exact.
//
// One CTA per (128-row tile of A, run of consecutive chunks); all eight warps cut the chunk's A
// rows and B columns into digit slices in shared memory, one thread issues the chunk's 48 MMAs
// (per K-step of 16: A slice s times B slices t0 .. t0 + nt - 1 stacked along N, into regions
// s + t0 ..), and all warps read the regions back (warp w: TMEM lanes 32 (w & 3) .., columns
// 32 (w >> 2) ..), recombine, and keep the chunk sums in FP64 registers; the run's sums go to
// C with one FP64 atomic each (C zeroed by the caller).
#include "common.cuh"
#include "tc.cuh"

namespace rq {

namespace {
using namespace tc;

constexpr int SK_ROWS = 128, SK_K = 64, SK_NP = 64;
constexpr int SK_THREADS = 256;
constexpr uint32_t SK_TMEM_COLS = 512;
// A: K-major, no swizzle: slice s, 8-row group at 1024 bytes, K-step c (16 K) at 256, K-half at
// 128, row at 16, K pair at 4.
constexpr uint32_t SA_LBO = 128, SA_SBO = 1024, SA_SLICE = (SK_ROWS / 8) * SA_SBO;
// B: per K-step a block of 8 slices x 64 rows (columns of B), stacked along N (8-row groups
// 256 bytes apart), K-half at 128; slice 7 is zero and only pads the first product.
constexpr uint32_t SB_LBO = 128, SB_SBO = 256, SB_TSLICE = (SK_NP / 8) * SB_SBO, SB_KSTEP = 8 * SB_TSLICE;
constexpr size_t SOFF_A = 0;
constexpr size_t SOFF_B = SOFF_A + (size_t)NDIG8 * SA_SLICE;
constexpr size_t SOFF_ROWE = SOFF_B + 4 * (size_t)SB_KSTEP;
constexpr size_t SOFF_COLE = SOFF_ROWE + 2 * SK_ROWS * sizeof(int);
constexpr size_t SOFF_BAR = SOFF_COLE + 2 * SK_NP * sizeof(int);
constexpr size_t SOFF_MISC = SOFF_BAR + 8;  // tmem slot, failure flag
constexpr size_t SK_SMEM = SOFF_MISC + 16;
static_assert(SOFF_B % 1024 == 0 && SK_SMEM <= 232448, "layout");
// more than half of the shared memory: one CTA per SM, so the 512 tensor-memory columns are free
static_assert(SK_SMEM > 232448 / 2, "one CTA per SM");

// One K-step's products: A slice s times B slices t0 .. t0 + nt - 1 into regions s + t0 ...
__device__ __forceinline__ void sk_issue_kstep(uint32_t tmem, uint64_t ad, uint64_t bd, int c) {
  const uint64_t ac = ((uint64_t)c * 2 * SA_LBO) >> 4, bc = ((uint64_t)c * SB_KSTEP) >> 4;
#define SK_MMA(s, t0, nt, acc)                                                                             \
  umma_bf16(tmem + (uint32_t)(64 * ((s) + (t0))), ad + ac + (((uint64_t)(s) * SA_SLICE) >> 4),             \
            bd + bc + (((uint64_t)(t0) * SB_TSLICE) >> 4), umma_idesc_f16(SK_ROWS, 64 * (nt)), (acc))
  const uint32_t first = c == 0 ? 0u : 1u;  // the two slice-0 products open all eight regions
  SK_MMA(0, 0, 4, first);
  SK_MMA(0, 4, 4, first);
  SK_MMA(1, 0, 4, 1u);
  SK_MMA(1, 4, 3, 1u);
  SK_MMA(2, 0, 4, 1u);
  SK_MMA(2, 4, 2, 1u);
  SK_MMA(3, 0, 4, 1u);
  SK_MMA(3, 4, 1, 1u);
  SK_MMA(4, 0, 4, 1u);
  SK_MMA(5, 0, 3, 1u);
  SK_MMA(6, 0, 2, 1u);
#undef SK_MMA
}

}  // namespace

// RAD: A is the Rademacher sketch, generated here instead of read: entry (r, k) is -rad_scale
// when bit k mod 64 of splitmix64(rad_seed ^ splitmix64(r ceil(K / 64) + floor(k / 64))) is set,
// else +rad_scale (the same values a materialised Rademacher S2 holds, so the same products).
// A 64-long chunk of a row shares one 64-bit word: one generator call per row and chunk.
template <bool RAD>
__global__ void __launch_bounds__(SK_THREADS, 1)
    k_sketch_oz(const double *__restrict__ A, int64_t lda, const double *__restrict__ B, int64_t ldb, int M,
                int64_t K, int n, double *C, int64_t ldc, int64_t chunks_per_cta, int ctas_per_tile, uint64_t rad_seed,
                double rad_scale, DevStatus *st) {
  // one decision for the whole CTA (its threads meet at block barriers below)
  if (__syncthreads_or(threadIdx.x == 0 && status_failed(st))) return;
  extern __shared__ __align__(1024) uint8_t sk_smem[];
  uint8_t *As = sk_smem + SOFF_A;
  uint8_t *Bs = sk_smem + SOFF_B;
  int *rowE = (int *)(sk_smem + SOFF_ROWE);  // [2][128], by chunk parity
  int *colE = (int *)(sk_smem + SOFF_COLE);  // [2][64]
  const uint32_t bar = smem_addr(sk_smem + SOFF_BAR);
  uint32_t *tmem_slot = (uint32_t *)(sk_smem + SOFF_MISC);
  volatile int *failed = (volatile int *)(sk_smem + SOFF_MISC + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = lane & 7, pi = lane >> 3;

  const int tile = blockIdx.x / ctas_per_tile, part = blockIdx.x % ctas_per_tile;
  const int row0 = SK_ROWS * tile;
  const int64_t nchunks = (K + SK_K - 1) / SK_K;
  const int64_t c_begin = (int64_t)part * chunks_per_cta;
  const int64_t c_end = imin64(nchunks, c_begin + chunks_per_cta);

  if (tid == 0) {
    mbar_init_count(bar, 1);
    *failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // the zero slice 7 of every K-step block
  for (int e = tid; e < (int)(4 * SB_TSLICE / 16); e += SK_THREADS) {
    const int c = e / (SB_TSLICE / 16), o = e % (SB_TSLICE / 16);
    *(uint4 *)(Bs + (size_t)c * SB_KSTEP + 7 * SB_TSLICE + 16 * o) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (warp == 0) tmem_alloc(tmem_slot, SK_TMEM_COLS);
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  // read-back share: TMEM lanes (rows) 32 q .., columns 32 ch ..
  const int q = warp & 3, ch = warp >> 2;
  const bool reads = 32 * ch < n;
  double acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = 0.0;

  int it = 0;
  for (int64_t ci = c_begin; ci < c_end; ++ci, ++it) {
    const int64_t k0 = SK_K * ci;
    const int par = it & 1;
    // ---- A: rows 16 warp + 8 hh + r, K pairs 8 kg + 2 pi (+1)
    unsigned long long a[2][8][2];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int row = row0 + 16 * warp + 8 * hh + r;
      const double *ap = A + (int64_t)row * lda;
      uint64_t word = 0;
      if (RAD) word = splitmix64(rad_seed ^ splitmix64((uint64_t)row * (uint64_t)nchunks + (uint64_t)ci));
      const unsigned long long pos = (unsigned long long)__double_as_longlong(rad_scale);
#pragma unroll
      for (int kg = 0; kg < 8; ++kg)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int kk = 8 * kg + 2 * pi + e;
          const int64_t k = k0 + kk;
          if (RAD)
            a[hh][kg][e] = (row < M && k < K) ? (pos | (((word >> kk) & 1ULL) << 63)) : 0ULL;
          else
            a[hh][kg][e] = (row < M && k < K) ? (unsigned long long)__double_as_longlong(__ldg(ap + k)) : 0ULL;
        }
    }
    // ---- B: column 8 warp + r, K pairs 8 kg + 2 pi (+1)
    unsigned long long b[8][2];
    const int col = 8 * warp + r;
#pragma unroll
    for (int kg = 0; kg < 8; ++kg)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t k = k0 + 8 * kg + 2 * pi + e;
        b[kg][e] = (col < n && k < K) ? (unsigned long long)__double_as_longlong(__ldg(B + k * ldb + col)) : 0ULL;
      }
    // ---- scales: largest exponent field of each row of A and each column of B in the chunk
    int ea[2], eb = 0;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      int mx = 0;
#pragma unroll
      for (int kg = 0; kg < 8; ++kg)
        mx = max(mx, max((int)((a[hh][kg][0] >> 52) & 0x7ff), (int)((a[hh][kg][1] >> 52) & 0x7ff)));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
      ea[hh] = scale_exp(mx);
    }
#pragma unroll
    for (int kg = 0; kg < 8; ++kg) eb = max(eb, max((int)((b[kg][0] >> 52) & 0x7ff), (int)((b[kg][1] >> 52) & 0x7ff)));
    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 8));
    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 16));
    eb = scale_exp(eb);
    if (pi == 0) {
      rowE[par * SK_ROWS + 16 * warp + r] = ea[0];
      rowE[par * SK_ROWS + 16 * warp + 8 + r] = ea[1];
      colE[par * SK_NP + col] = eb;
    }
    // ---- digit slices (the previous chunk's products are complete: its read-back waited)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      uint8_t *dst = As + (size_t)(2 * warp + hh) * SA_SBO + (size_t)r * 16 + (size_t)pi * 4;
#pragma unroll
      for (int kg = 0; kg < 8; ++kg) {
        uint32_t w[NDIG8];
        digits8_biased(fix54_biased(a[hh][kg][0], ea[hh]), fix54_biased(a[hh][kg][1], ea[hh]), w);
        const size_t o = (size_t)(kg >> 1) * 2 * SA_LBO + (size_t)(kg & 1) * SA_LBO;
#pragma unroll
        for (int p = 0; p < NDIG8; ++p) *(uint32_t *)(dst + o + (size_t)(NDIG8 - 1 - p) * SA_SLICE) = w[p];
      }
    }
    {
      uint8_t *dst = Bs + (size_t)warp * SB_SBO + (size_t)r * 16 + (size_t)pi * 4;
#pragma unroll
      for (int kg = 0; kg < 8; ++kg) {
        uint32_t w[NDIG8];
        digits8_biased(fix54_biased(b[kg][0], eb), fix54_biased(b[kg][1], eb), w);
        const size_t o = (size_t)(kg >> 1) * SB_KSTEP + (size_t)(kg & 1) * SB_LBO;
#pragma unroll
        for (int p = 0; p < NDIG8; ++p) *(uint32_t *)(dst + o + (size_t)(NDIG8 - 1 - p) * SB_TSLICE) = w[p];
      }
    }
    fence_async_smem();
    __syncthreads();
    // ---- products (one thread), then every thread waits for them through thread 0
    if (tid == 0) {
      fence_after_sync();
      uint64_t ad = umma_desc(smem_addr(As), SA_LBO, SA_SBO), bd = umma_desc(smem_addr(Bs), SB_LBO, SB_SBO);
      asm volatile("" : "+l"(ad), "+l"(bd));
#pragma unroll 1
      for (int c = 0; c < 4; ++c) sk_issue_kstep(tmem, ad, bd, c);
      umma_commit(bar);
      if (!mbar_wait(bar, (uint32_t)par, wait_bound(st, MAX_WAIT))) *failed = 1;
    }
    __syncthreads();
    if (*failed) break;
    fence_after_sync();
    // ---- read-back: region values of 4 columns at a time, recombined and summed in FP64
    if (reads) {
      const int Er = rowE[par * SK_ROWS + 32 * q + lane];
      const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * ch);
#pragma unroll
      for (int cg = 0; cg < 8; ++cg) {
        if (32 * ch + 4 * cg >= n) break;
        uint32_t v[8][4];
#pragma unroll
        for (int g = 0; g < 8; ++g) tmem_ld4(tq + (uint32_t)(64 * g + 4 * cg), v[g]);
        tmem_wait_ld();
        tmem_regs_ready(v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = 32 * ch + 4 * cg + c;
          const long long t = recombine_b8(v[0][c], v[1][c], v[2][c], v[3][c], v[4][c], v[5][c], v[6][c], v[7][c]);
          // integer-pipe conversion: the FP64 pipe is left to the sums
          acc[4 * cg + c] += int_times_pow2(t, Er + colE[par * SK_NP + (j & 63)] - 56);
        }
      }
    }
    fence_before_sync();
  }

  if (*failed) {
    // the products may still run: wait for them once more (bounded) before tensor memory goes
    if (tid == 0) {
      status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
      mbar_wait(bar, (uint32_t)(it & 1));
    }
  } else if (reads) {
    const int row = row0 + 32 * q + lane;
    if (row < M) {
      double *cp = C + (int64_t)row * ldc;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int j = 32 * ch + c;
        if (j < n && it > 0) atomicAdd(cp + j, acc[c]);
      }
    }
  }
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_free(tmem, SK_TMEM_COLS);
}

bool sketch_oz_supported(int64_t n) { return n >= 1 && n <= 2 * SK_NP; }

namespace {
template <bool RAD>
cudaError_t launch_sketch_oz_t(const double *A, int64_t lda, const double *B, int64_t ldb, int64_t M, int64_t K,
                               int64_t n, double *C, int64_t ldc, uint64_t rad_seed, double rad_scale, int num_sms,
                               DevStatus *st, cudaStream_t s) {
  if (M <= 0 || K <= 0) return cudaSuccess;
  const int64_t tiles = ceil_div(M, SK_ROWS);
  const int64_t nchunks = ceil_div(K, SK_K);
  const int64_t per_tile = std::max<int64_t>(1, std::min<int64_t>(nchunks, (int64_t)num_sms / std::max<int64_t>(tiles, 1)));
  const int64_t chunks_per_cta = ceil_div(nchunks, per_tile);
  const int64_t ctas_per_tile = ceil_div(nchunks, chunks_per_cta);
  const int64_t grid = tiles * ctas_per_tile;
  if (grid >= ((int64_t)1 << 31) || M >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_sketch_oz<RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SK_SMEM);
  if (e != cudaSuccess) return e;
  k_sketch_oz<RAD><<<(unsigned)grid, SK_THREADS, SK_SMEM, s>>>(A, lda, B, ldb, (int)M, K, (int)n, C, ldc,
                                                               chunks_per_cta, (int)ctas_per_tile, rad_seed, rad_scale,
                                                               st);
  return cudaGetLastError();
}
}  // namespace

// n <= 128 as column blocks of at most 64 (the column scales are per column anyway)
cudaError_t launch_sketch_oz(const double *A, int64_t lda, const double *B, int64_t ldb, int64_t M, int64_t K,
                             int64_t n, double *C, int num_sms, DevStatus *st, cudaStream_t s) {
  for (int64_t c0 = 0; c0 < n; c0 += SK_NP) {
    cudaError_t e = launch_sketch_oz_t<false>(A, lda, B + c0, ldb, M, K, std::min<int64_t>(SK_NP, n - c0), C + c0, n, 0,
                                              0.0, num_sms, st, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_sketch_oz_rademacher(uint64_t seed, const double *B, int64_t ldb, int64_t M, int64_t K, int64_t n,
                                        double *C, int num_sms, DevStatus *st, cudaStream_t s) {
  for (int64_t c0 = 0; c0 < n; c0 += SK_NP) {
    cudaError_t e = launch_sketch_oz_t<true>(nullptr, 0, B + c0, ldb, M, K, std::min<int64_t>(SK_NP, n - c0), C + c0, n,
                                             seed, 1.0 / sqrt((double)M), num_sms, st, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace rq
