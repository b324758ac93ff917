// trsm_tc.cu -- Q = W R_c^{-1} (Algorithm 2 step 3 of rand_cholQR's second pass) as the product
// Q = W X with X = R_c^{-1}, from exact split products on the tensor cores.
//
// rand_cholQR's R_c is the Cholesky factor of the Gram of the preconditioned W, so
// kappa(R_c) = kappa(W) = O(1) (Sec. 4.1, Theorem 5.2): applying its explicit inverse is then
// as accurate as the row-wise solve (errors grow with kappa(R_c), not kappa(V)), and the
// solve becomes a dense contraction with K = n.  (The first solve, W = V R_s^{-1}, keeps the
// row-wise substitution: R_s inherits kappa(V).)
//
// Each row i of a 128-row tile gets its own scale 2^e_i and each column k of X its own scale
// 2^f_k (tc.cuh's eight 7-bit digits): Q_ik = 2^(e_i + f_k) sum_g 2^(-14 - 7 g) D_g(i, k),
// D_g = sum_{s + t = g} sum_j a_s(i, j) b_t(j, k), g <= 7.  Each D_g sums at most 8 x 64
// digit products (< 2^23): exact in the FP32 accumulators.  Region g of tensor memory (64
// columns) holds D_g; the K = 64 reduction runs in two halves of 32 so that one half of the
// row slices (64 KB) fits in shared memory beside X's slices and the row tile.
// n <= 64 (n padded to 64 with zeros).
#include "common.cuh"
#include "df.cuh"
#include "tc.cuh"

namespace rq {

namespace {
constexpr int TQ_THREADS = 256;
constexpr int TQ_ROWS = 128;
constexpr int TQ_NP = 64;
constexpr uint32_t TQ_TMEM_COLS = 512;
constexpr size_t TQ_B_BYTES = (size_t)tc::SLICES * TQ_NP * TQ_NP * 2;      // 64 KB
constexpr size_t TQ_A_BYTES = (size_t)tc::SLICES * TQ_ROWS * 32 * 2;       // 64 KB
constexpr size_t TQ_STAGE_BYTES = (size_t)TQ_ROWS * TQ_NP * 8;             // 64 KB
}  // namespace

template <bool IN_DF>
__global__ void __launch_bounds__(TQ_THREADS, 1)
    k_trsm_oz(const void *Win, int64_t ldw, double *Q, int64_t ldq, int64_t m, int n,
              const double *__restrict__ Xp, int64_t rows_per_cta, bool bulk, DevStatus *st) {
  using namespace tc;
  if (status_failed(st)) return;
  extern __shared__ __align__(1024) uint8_t tq_smem[];
  uint8_t *Bt = tq_smem;
  uint8_t *A = Bt + TQ_B_BYTES;
  uint8_t *stage = A + TQ_A_BYTES;
  int *rowexp = (int *)(stage + TQ_STAGE_BYTES);
  int *colexp = rowexp + TQ_ROWS;
  uint64_t *bars = (uint64_t *)(colexp + TQ_NP);
  uint32_t *tmem_slot = (uint32_t *)(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t copy_bar = smem_addr(&bars[0]), mma_bar = smem_addr(&bars[1]);

  if (warp == 0) tmem_alloc(tmem_slot, TQ_TMEM_COLS);
  if (tid == 0) {
    mbar_init(copy_bar);
    mbar_init(mma_bar);
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  if (tid < TQ_NP) colexp[tid] = 0;
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  // ---- X's slices (B operand): rows k (output column), K = j; X(j, k) = 0 for j > k
  for (int e = tid; e < TQ_NP * TQ_NP; e += TQ_THREADS) {
    const int k = e / TQ_NP, jj = e % TQ_NP;
    if (k < n && jj <= k) atomicMax(&colexp[k], expfield<false>(Xp + tri_idx(jj, k)));
  }
  __syncthreads();
  for (int e = tid; e < TQ_NP * TQ_NP / 2; e += TQ_THREADS) {
    const int k = e / (TQ_NP / 2), jj = 2 * (e % (TQ_NP / 2));
    const int f = scale_exp(colexp[k]);
    long long x[2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
      x[u] = (k < n && jj + u <= k) ? fixpt<false>(Xp + tri_idx(jj + u, k), f) : 0;
#pragma unroll
    for (int s = 0; s < SLICES; ++s)
      *(uint32_t *)(Bt + (size_t)s * TQ_NP * TQ_NP * 2 + (size_t)kmajor_off(k, jj, TQ_NP) * 2) =
          digit_bf16(x[0], s) | (digit_bf16(x[1], s) << 16);
  }

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  const uint32_t idesc = umma_idesc(TQ_ROWS, TQ_NP);
  const int L = 32 * (warp & 3) + lane, half = warp >> 2;  // flush: tile row L, 32 columns
  uint32_t copy_phase = 0, mma_phase = 0;
  bool ok = true;
  for (int64_t row0 = r_begin; row0 < r_end && ok; row0 += TQ_ROWS) {
    const int rows = (int)imin64(TQ_ROWS, r_end - row0);
    if (tid < TQ_ROWS) rowexp[tid] = 0;
    // ---- the row tile in shared memory (row-major, n entries of 8 bytes per row)
    if (bulk) {
      __syncthreads();
      if (tid == 0) {
        const uint32_t bytes = (uint32_t)rows * (uint32_t)n * 8u;
        mbar_expect_tx(copy_bar, bytes);
        const uint8_t *src = (const uint8_t *)Win + (size_t)row0 * (size_t)ldw * 8;
        for (uint32_t off = 0; off < bytes; off += 16384)
          bulk_load(smem_addr(stage) + off, src + off, bytes - off < 16384 ? bytes - off : 16384, copy_bar);
      }
      if (!__syncthreads_and(mbar_wait(copy_bar, copy_phase))) {
        ok = false;
        if (tid == 0) status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
        mbar_wait(copy_bar, copy_phase);
        break;
      }
      copy_phase ^= 1;
    } else {
      for (int e = tid; e < rows * n; e += TQ_THREADS) {
        const int r = e / n, c = e - r * n;
        ((unsigned long long *)stage)[e] = ((const unsigned long long *)Win)[(row0 + r) * ldw + c];
      }
      __syncthreads();
    }
    // ---- row scales
    {
      const int r = tid >> 1, c0 = 32 * (tid & 1);
      int mx = 0;
      if (r < rows)
        for (int c = c0; c < c0 + 32 && c < n; ++c) mx = max(mx, expfield<IN_DF>(stage + ((size_t)r * n + c) * 8));
      atomicMax(&rowexp[r], mx);
    }
    __syncthreads();
    // ---- two K halves: slice W's columns 32 hk .. +31, then their products
    for (int hk = 0; hk < 2 && ok; ++hk) {
      for (int e = tid; e < TQ_ROWS * 16; e += TQ_THREADS) {
        const int r = e / 16, jj = 2 * (e % 16), j = 32 * hk + jj;
        const int er = scale_exp(rowexp[r]);
        long long x[2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
          x[u] = (r < rows && j + u < n) ? fixpt<IN_DF>(stage + ((size_t)r * n + j + u) * 8, er) : 0;
#pragma unroll
        for (int s = 0; s < SLICES; ++s)
          *(uint32_t *)(A + (size_t)s * TQ_ROWS * 32 * 2 + (size_t)kmajor_off(r, jj, 32) * 2) =
              digit_bf16(x[0], s) | (digit_bf16(x[1], s) << 16);
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        fence_after_sync();
        const uint32_t abase = smem_addr(A), bbase = smem_addr(Bt);
        for (int g = 0; g < SLICES; ++g) {
          for (int s = 0; s <= g; ++s) {
            const int t = g - s;
            for (int kk = 0; kk < 2; ++kk) {
              const uint64_t ad = umma_desc(abase + (uint32_t)(s * TQ_ROWS * 32 * 2) + 256u * kk, 128, 512);
              const uint64_t bd = umma_desc(bbase + (uint32_t)(t * TQ_NP * TQ_NP * 2) + 128u * (4 * hk + 2 * kk),
                                            128, 1024);
              umma_bf16(tmem + (uint32_t)(g * 64), ad, bd, idesc, (hk | s | kk) ? 1u : 0u);
            }
          }
        }
        umma_commit(mma_bar);
      }
      if (!__syncthreads_and(mbar_wait(mma_bar, mma_phase))) {
        ok = false;
        if (tid == 0) status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
        mbar_wait(mma_bar, mma_phase);
        break;
      }
      mma_phase ^= 1;
      fence_after_sync();
    }
    if (!ok) break;
    // ---- flush: row L, columns 32 half .. +31 -> FP64 Q entries into the stage
    {
      const int er = scale_exp(rowexp[L]);
      double *qrow = (double *)stage + (size_t)L * n;
#pragma unroll
      for (int c8 = 0; c8 < 4; ++c8) {
        uint32_t v[SLICES][8];
#pragma unroll
        for (int g = 0; g < SLICES; ++g)
          tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(g * 64 + 32 * half + 8 * c8), v[g]);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float sh = 0.f, sl = 0.f;
#pragma unroll
          for (int g = 0; g < SLICES; ++g) {
            const float tv = __uint_as_float(v[g][i]) * pow2f(-14 - 7 * g);
            const float t = __fadd_rn(sh, tv);
            const float z = __fsub_rn(t, sh);
            sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(tv, z)));
            sh = t;
          }
          const int k = 32 * half + 8 * c8 + i;
          if (L < rows && k < n) qrow[k] = scale_pow2(df2d(sh, sl), er + scale_exp(colexp[k]));
        }
      }
    }
    fence_before_sync();
    fence_async_smem();
    __syncthreads();
    // ---- the tile back to Q (rows row0 .. row0 + rows - 1)
    if (bulk) {
      if (tid == 0) {
        const uint32_t bytes = (uint32_t)rows * (uint32_t)n * 8u;
        uint8_t *dst = (uint8_t *)Q + (size_t)row0 * (size_t)ldq * 8;
        for (uint32_t off = 0; off < bytes; off += 16384)
          bulk_store(dst + off, smem_addr(stage) + off, bytes - off < 16384 ? bytes - off : 16384);
        bulk_store_commit();
        bulk_store_wait();
      }
    } else {
      for (int e = tid; e < rows * n; e += TQ_THREADS) {
        const int r = e / n, c = e - r * n;
        Q[(row0 + r) * ldq + c] = ((const double *)stage)[e];
      }
    }
    __syncthreads();
  }
  if (bulk && tid == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");  // stores done
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, TQ_TMEM_COLS);
}

bool trsm_oz_supported(int64_t n) { return n >= 1 && n <= TQ_NP; }

cudaError_t launch_trsm_oz(const void *W, bool in_df, int64_t ldw, double *Q, int64_t ldq, int64_t m,
                           int64_t n, const double *Xpacked, int num_sms, DevStatus *st,
                           cudaStream_t s) {
  const size_t smem = TQ_B_BYTES + TQ_A_BYTES + TQ_STAGE_BYTES + (TQ_ROWS + TQ_NP) * sizeof(int) + 32;
  int64_t ctas = std::min<int64_t>(ceil_div(m, TQ_ROWS), (int64_t)num_sms);
  const int64_t rows_per_cta = ceil_div(ceil_div(m, ctas), TQ_ROWS) * TQ_ROWS;
  ctas = ceil_div(m, rows_per_cta);
  const bool bulk = ldw == n && ldq == n && ((n * 8) % 16 == 0) && (((uintptr_t)W & 15) == 0) &&
                    (((uintptr_t)Q & 15) == 0);
  cudaError_t e;
  if (in_df) {
    e = cudaFuncSetAttribute(k_trsm_oz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_trsm_oz<true><<<(unsigned)ctas, TQ_THREADS, smem, s>>>(W, ldw, Q, ldq, m, (int)n, Xpacked, rows_per_cta, bulk, st);
  } else {
    e = cudaFuncSetAttribute(k_trsm_oz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_trsm_oz<false><<<(unsigned)ctas, TQ_THREADS, smem, s>>>(W, ldw, Q, ldq, m, (int)n, Xpacked, rows_per_cta, bulk, st);
  }
  return cudaGetLastError();
}

}  // namespace rq
