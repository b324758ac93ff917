// trsm_tc.cu -- Y = X B for an upper-triangular B given by its packed FP64 entries (at most
// 64 x 64), from exact split products on the tensor cores.  rand_cholQR runs both of its
// triangular solves (W = V R_s^{-1} and Q = W R_c^{-1}, Algorithm 3) this way, as products with
// the explicit inverses; for 64 < n <= 128 the solves are blocked into such products (api.cu):
// X has nk <= 64 columns and Y nn <= 64 (B is nk x nn, entries j <= k), the columns of X and Y
// may be taken in reverse order (so that a strictly lower block becomes upper triangular), and
// the product may be added to a reference matrix instead of stored (Y = Ref + X B, formed as
// one integer sum and rounded once).
//
// Number format.  Row i of X gets a scale 2^E_i > max_j |x_ij| and column k of B a scale
// 2^F_k > max_j |b_jk|.  x_ij = 2^(E_i - 54) X_ij up to truncation, with the integer
// X_ij = trunc(x_ij 2^(54 - E_i)) written in seven balanced byte digits d_s (tc.cuh; slice
// s = 0 holds the leading digit), and the same for b_jk with digits e_t.  The product keeps the
// slice pairs s + t <= 7, gathered by g = s + t into eight regions of tensor memory:
//   D_g(i, k) = sum_{s + t = g} sum_j d_s(i, j) e_t(j, k),
//   y_ik = 2^(E_i + F_k - 56) T_ik / 2^12,   T_ik = sum_g 2^(8 (7 - g)) D_g(i, k).
// Every region is an exact FP32 integer (|D_g| < 2^23: at most 2^22 for g <= 4, where exactness
// of the conversion matters); tc::recombine_b8 turns them into T / 2^12 in 64-bit integer
// arithmetic, which is rounded once to FP64.  Truncation and the dropped pairs (s + t >= 8)
// weigh about 2^-54 of 2^(E_i + F_k) per term: a relative perturbation of each row of X, so the
// first solve's backward error in V stays at that level whatever kappa(V) is.
//
// Products.  A tcgen05.mma costs about as much for N = 16 as for N = 64 (the 128 x 16 A operand
// is read from shared memory each time) and reaches the tensor cores' full rate only from
// N = 128 on.  So the B slices are stacked along N: one MMA multiplies A slice s by the
// slices t = 0 .. 7 - s side by side and writes regions s .. 7 at once.  The output columns are
// taken in two halves of 32 (regions of one half occupy 8 x 32 tensor-memory columns): the
// half of columns 0-31 needs only the K-steps j < 32 of an upper-triangular B, and the read-back
// of one half overlaps the products of the other.  A tile of 128 rows takes 42 MMAs
// (7 per half and K-step) with N between 64 and 256.
//
// One CTA per SM, persistent over 128-row tiles; warps specialise:
//   warps 0-7 cut rows into digit slices (shared memory A: 7 slices x 128 rows x 64 K, f16);
//     warps 0-3 take sub-tiles 0 and 2 of each tile, 4-7 sub-tiles 1 and 3, one 8-row group each,
//   warps 8-15 read tensor memory back (TMEM lanes 32 (w & 3) .., 16 columns of each half),
//     recombine and store 64-byte row segments of Y,
//   warp 16 loads 32-row sub-tiles of X into a four-slot ring (slot q holds sub-tile q) with
//     16-byte asynchronous copies (one row per instruction; rows padded to 528 bytes in shared
//     memory, so the slicers' reads of eight rows at one column fall into eight different bank
//     groups) and prefetches the next tile towards L2,
//   warp 17 owns tensor memory and issues the MMAs,
// handing tiles over through mbarriers.  B's digit slices are built once per CTA.  A's K-block
// c (K-step c) is released to the next tile's slicers as soon as the last MMA that reads it has
// completed.  In place (Y == X) is safe: a tile's rows are read before any are written.
#include "common.cuh"
#include "gram_split_body.cuh"
#include "tc.cuh"

namespace rq {

namespace {
using namespace tc;

constexpr int TQ_ROWS = 128, TQ_NP = 64, TQ_SUB = 32, TQ_NSTAGE = 4;
constexpr int TQ_THREADS = 576;
constexpr int W_FLUSH0 = 8, W_LOAD = 16, W_MMA = 17;
constexpr uint32_t TQ_TMEM_COLS = 512;
// A: K-major, no swizzle.  A slicer lane (row r = lane & 7 of an 8-row group, pair pi =
// lane >> 3 of every K core matrix) stores 4 bytes at r * 16 + pi * 4 of a core matrix: one
// warp store covers one core matrix, all 32 banks.
constexpr uint32_t A_LBO = 128, A_SBO = 8 * A_LBO, A_SLICE = (TQ_ROWS / 8) * A_SBO;
// B: one block per (half h, K-step c) -- h = 0 needs c = 0, 1; h = 1 needs c = 0 .. 3 -- of
// 32 rows (output columns 32h ..) per slice t, slices stacked along N, 16 K, K-major with
// 8-row groups 256 bytes apart.  The blocks of K-step 0 carry an eighth, zero slice, so that
// the first MMA of a half (slice s = 0, N = 256) writes all eight regions.
constexpr uint32_t B_LBO = 128, B_SBO = 256, B_TSLICE = 32 * 32;
__host__ __device__ constexpr uint32_t b_block(int h, int c) {
  return h == 0 ? (c == 0 ? 0u : 8u * B_TSLICE) : (15u + (c == 0 ? 0u : 8u + 7u * (uint32_t)(c - 1))) * B_TSLICE;
}
constexpr uint32_t B_BYTES = b_block(1, 3) + 7 * B_TSLICE;
// A staged 32-row sub-tile holds its rows at a pitch of 528 bytes (64 FP64 values and 16
// bytes of padding): row r starts in bank group r mod 8, so eight rows read at one column
// touch eight different bank groups.
constexpr uint32_t STAGE_PITCH = TQ_NP * 8 + 16;
constexpr uint32_t STAGE_BYTES = TQ_SUB * STAGE_PITCH;
constexpr size_t OFF_B = 0;
constexpr size_t OFF_A = OFF_B + B_BYTES;
constexpr size_t OFF_STAGE = OFF_A + (size_t)NDIG8 * A_SLICE;
constexpr size_t OFF_ROWEXP = OFF_STAGE + (size_t)TQ_NSTAGE * STAGE_BYTES;
constexpr size_t OFF_COLEXP = OFF_ROWEXP + 3 * TQ_ROWS * sizeof(int);
constexpr size_t OFF_BARS = OFF_COLEXP + TQ_NP * sizeof(int);
// full[4], empty[4], a_full[4], kfree[4], h_done[2], t_empty[2], drain
constexpr int BAR_FULL = 0, BAR_EMPTY = 4, BAR_AFULL = 8, BAR_KFREE = 12, BAR_HDONE = 16, BAR_TEMPTY = 18,
              BAR_DRAIN = 20, NBARS = 21;
constexpr size_t OFF_MISC = OFF_BARS + NBARS * 8;  // tmem slot, abort flag
constexpr size_t TQ_SMEM = OFF_MISC + 16;
static_assert(OFF_A % 1024 == 0 && OFF_STAGE % 1024 == 0 && B_BYTES == 45056, "layout");
static_assert(TQ_SMEM <= 232448, "shared memory budget");

// LOAD_ASYNC: 16-byte asynchronous copies, one row per warp instruction (lane = 16-byte chunk);
// needs 16-byte aligned rows and an even column count.  LOAD_PLAIN: element loads.  Every loader
// lane arrives on the slot's barrier once per fill.
enum LoadMode { LOAD_ASYNC = 0, LOAD_PLAIN = 1 };

// Byte offset of element (row r, column col) of a staged sub-tile.
__device__ __forceinline__ uint32_t stage_off(int r, int col) { return (uint32_t)r * STAGE_PITCH + (uint32_t)col * 8u; }

__device__ __forceinline__ void set_abort(volatile int *abort_flag, DevStatus *st) {
  *abort_flag = 1;
  status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
}

// Descriptor offsets (16-byte units) of A slice s at K-step c, and of B's block (h, c).
__device__ __forceinline__ constexpr uint64_t a_off(int s, int c) { return ((uint64_t)s * A_SLICE + (uint64_t)c * 2 * A_LBO) >> 4; }
__device__ __forceinline__ constexpr uint64_t b_off(int h, int c) { return (uint64_t)b_block(h, c) >> 4; }

// One half's products for K-step C: A slice s times B slices 0 .. NR - 1 - s (at most 6) of block
// (H, C), into regions s .. NR - 1 of that half, NR = NDA + 1 regions for NDA digits of A (7: the
// pairs s + t <= 7; 6: s + t <= 6, a 46-bit product).  The first product of a half (C = 0, s = 0)
// covers every region (for NR = 8 with the zero eighth B slice) and overwrites them; every other
// accumulates.
template <int H, int C, int NDA>
__device__ __forceinline__ void issue_half_kstep(uint32_t tmem, uint64_t ad, uint64_t bd) {
  constexpr int NR = NDA + 1;
#pragma unroll
  for (int s = 0; s < NDA; ++s) {
    const int nt = (C == 0 && s == 0) ? NR : (NR - s < 7 ? NR - s : 7);
    umma_bf16(tmem + (uint32_t)(256 * H + 32 * s), ad + a_off(s, C), bd + b_off(H, C), umma_idesc_f16(TQ_ROWS, 32 * nt),
              (C == 0 && s == 0) ? 0u : 1u);
  }
}

}  // namespace

// ref + t 2^u0 (t the recombined product, |t| < 2^62) as one 64-bit integer sum, rounded once:
// the unit of the sum is 2^u0, or coarser when ref would not fit 2^61 units of it; ref is
// truncated to that unit (below 2^-59 of |ref|, an FP64 subtraction's rounding).
__device__ __forceinline__ double add_fixed(double ref, long long t, int u0) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(ref);
  const int ef = (int)((b >> 52) & 0x7ff);
  const int u1 = max(u0, ef - 1023 - 60);
  const int d = min(u1 - u0, 63);
  const long long ts = t >> d;
  const int sh = ef - 1075 - u1;  // ref = mant 2^(ef - 1075); at most 8 by the choice of u1
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
  long long rf = sh >= 0 ? (mant << sh) : (-sh < 63 ? (mant >> -sh) : 0);
  rf = ef == 0 ? 0 : rf;
  rf = (b >> 63) ? -rf : rf;
  return int_times_pow2_cvt(ts + rf, u1);
}

enum Epilogue { EPI_STORE = 0, EPI_ADDREF = 1, EPI_RESID = 2 };

// NH: column halves of 32 (1 when nk, nn <= 32: only K-blocks 0, 1 and tensor-memory half 0 are
// used).  NDA: digits of A (7, or 6 for the 46-bit products of RANDQR_F32X2).
// FULLN: nk == nn == 32 NH with 16-byte aligned rows of Y: no per-value column checks, and rows of a
// partly filled sub-tile are cut whatever their slot holds (their products are never stored).
// REV: X's columns are read as X J and Y's written as Y J (J the reversal of nk, nn columns).
// EPI_ADDREF: Y = Ref + X B (Ref may be Y itself, read in the same column order).
// EPI_RESID: instead of storing Y, accumulate sums[0] += sum (Ref - Y)^2 and sums[1] += sum Ref^2
// over the rows (the residual of a factorization V = Q R, with X = Q and B = R).
// SIG: after storing its rows of tile i, read-back warp f publishes i + 1 in the 32-bit word
// sig + 4 f of this CTA's shared memory (release at cluster scope), for a Gram CTA of the same
// cluster that reads the stored rows (k_solve_gram); PRODUCER_DONE there once it gives up.
template <bool FULLN, bool REV, int EPI, int NH, int NDA, bool SIG>
__device__ __forceinline__ void trsm_oz_cta(const double *__restrict__ X, int64_t ldx, double *Y, int64_t ldy,
                                            int64_t m, int nk, int nn, const double *__restrict__ Bp, int b_ld,
                                            int64_t rows_per_cta, int load_mode, bool vec_store, const double *Vref,
                                            int64_t ldvr, double *sums, DevStatus *st, int cta, uint32_t sig) {
  constexpr bool RESID = EPI == EPI_RESID;
  constexpr int NKB = 2 * NH;  // K-blocks of 16 columns
  const int lim = wait_bound(st, MAX_WAIT);
  extern __shared__ __align__(1024) uint8_t tq_smem[];
  uint8_t *Bs = tq_smem + OFF_B;
  uint8_t *As = tq_smem + OFF_A;
  uint8_t *stage = tq_smem + OFF_STAGE;
  int *rowexp = (int *)(tq_smem + OFF_ROWEXP);
  int *colexp = (int *)(tq_smem + OFF_COLEXP);
  uint64_t *bars = (uint64_t *)(tq_smem + OFF_BARS);
  uint32_t *tmem_slot = (uint32_t *)(tq_smem + OFF_MISC);
  volatile int *abort_flag = (volatile int *)(tq_smem + OFF_MISC + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar0 = smem_addr(&bars[0]);
  auto bar = [&](int b) { return bar0 + 8u * (uint32_t)b; };

  if (tid == 0) {
    for (int q = 0; q < TQ_NSTAGE; ++q) {
      mbar_init_count(bar(BAR_FULL + q), 32);
      mbar_init_count(bar(BAR_EMPTY + q), 4);
    }
    for (int c = 0; c < 4; ++c) {
      mbar_init_count(bar(BAR_AFULL + c), 8);
      mbar_init_count(bar(BAR_KFREE + c), 1);
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init_count(bar(BAR_HDONE + h), 1);
      mbar_init_count(bar(BAR_TEMPTY + h), 8);
    }
    mbar_init_count(bar(BAR_DRAIN), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (tid < TQ_NP) colexp[tid] = 0;
  if (warp == W_MMA) tmem_alloc(tmem_slot, TQ_TMEM_COLS);
  __syncthreads();

  // ---- B's digit slices (all threads, once): column scales, then the blocks
  // B entry (j, k): packed upper (b_ld == 0), or dense row-major with leading dimension b_ld; a
  // dense B contributes the rows j < 32 of its columns k < 32 only (the K-steps the first column
  // half takes), its other rows there being left to another product
  auto b_used = [&](int j, int k) { return k < nn && j < nk && (b_ld ? (k >= 32 || j < 32) : j <= k); };
  auto b_at = [&](int j, int k) { return b_ld ? Bp + (int64_t)j * b_ld + k : Bp + tri_idx(j, k); };
  for (int e = tid; e < TQ_NP * TQ_NP; e += TQ_THREADS) {
    const int k = e >> 6, j = e & 63;
    if (b_used(j, k)) atomicMax(&colexp[k], expfield<false>(b_at(j, k)));
  }
  for (int e = tid; e < (int)(B_TSLICE / 4); e += TQ_THREADS) {  // the zero eighth slices
    *(uint32_t *)(Bs + b_block(0, 0) + 7 * B_TSLICE + 4 * e) = 0u;
    *(uint32_t *)(Bs + b_block(1, 0) + 7 * B_TSLICE + 4 * e) = 0u;
  }
  __syncthreads();
  // 6 blocks x 32 columns x 8 K pairs; block index bb: (h, c) = (0, 0), (0, 1), (1, 0) .. (1, 3)
  for (int e = tid; e < 6 * 32 * 8; e += TQ_THREADS) {
    const int bb = e >> 8, kp = (e >> 3) & 31, jp = e & 7;
    const int h = bb < 2 ? 0 : 1, c = bb < 2 ? bb : bb - 2;
    const int k = 32 * h + kp, j = 16 * c + 2 * jp;
    const int F = scale_exp(colexp[k]);
    const long long za = b_used(j, k) ? fix54(*b_at(j, k), F) : 0;
    const long long zb = b_used(j + 1, k) ? fix54(*b_at(j + 1, k), F) : 0;
    uint32_t w[NDIG8];
    digits8(za, zb, w);
    const uint32_t off = b_block(h, c) + (uint32_t)(kp >> 3) * B_SBO + (uint32_t)(jp >> 2) * B_LBO +
                         (uint32_t)(kp & 7) * 16 + (uint32_t)(jp & 3) * 4;
#pragma unroll
    for (int p = 0; p < NDIG8; ++p) *(uint32_t *)(Bs + off + (uint32_t)(NDIG8 - 1 - p) * B_TSLICE) = w[p];
  }
  fence_async_smem();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int64_t r_begin = (int64_t)cta * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  const int ntiles = r_end > r_begin ? (int)((r_end - r_begin + TQ_ROWS - 1) / TQ_ROWS) : 0;
  auto sub_rows = [&](int i, int q) -> int {
    const int64_t r0 = r_begin + (int64_t)i * TQ_ROWS + TQ_SUB * q;
    return r0 < r_end ? (int)imin64(TQ_SUB, r_end - r0) : 0;
  };

  if (warp == W_LOAD) {
    // ------------------------------------------------------------------ loader
    // Slot q holds sub-tile q of every tile; its only consumers are the four slicer warps of
    // group q & 1, so the phase of slot q in tile i is i & 1.
    int last_i[TQ_NSTAGE];  // last tile whose sub-tile q was loaded into slot q
#pragma unroll
    for (int q = 0; q < TQ_NSTAGE; ++q) last_i[q] = -1;
    for (int i = 0; i < ntiles && !*abort_flag; ++i) {
      bool ok = true;
      // the next tile's rows towards L2 while this tile's slots free up (contiguous rows only)
      if (lane == 0 && load_mode != LOAD_PLAIN && ldx == nk && i + 1 < ntiles) {
        const int64_t p0 = r_begin + (int64_t)(i + 1) * TQ_ROWS;
        const int64_t prow = imin64(TQ_ROWS, r_end - p0);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(X + p0 * ldx),
                     "r"((uint32_t)(prow * nk * 8)) : "memory");
      }
      // the reference rows this tile's read-back adds to (EPI_ADDREF), towards L2 a tile ahead
      // of their use: one prefetch per 128-byte line of each row's nn values
      if (EPI == EPI_ADDREF) {
        const int64_t t0 = r_begin + (int64_t)i * TQ_ROWS;
        for (int r = lane; r < TQ_ROWS && t0 + r < r_end; r += 32) {
          const double *row = Vref + (t0 + r) * ldvr;
          for (int c = 0; c < nn + 16; c += 16)  // every line the row's nn values touch
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(row + min(c, nn - 1)) : "memory");
        }
      }
      for (int q = 0; q < TQ_NSTAGE; ++q) {
        if (!mbar_wait_or_abort(bar(BAR_EMPTY + q), (uint32_t)((i & 1) ^ 1), abort_flag, lim)) {
          if (lane == 0 && !*abort_flag) set_abort(abort_flag, st);
          ok = false;
          break;
        }
        const int64_t r0 = r_begin + (int64_t)i * TQ_ROWS + TQ_SUB * q;
        const int cnt = sub_rows(i, q);
        uint8_t *dst = stage + (size_t)q * STAGE_BYTES;
        const uint32_t fb = bar(BAR_FULL + q);
        // the cnt rows of the sub-tile (rows past cnt keep what the slot held; the slicers mask them)
        if (load_mode == LOAD_ASYNC) {
          const int chunks = nk >> 1;  // 16-byte chunks per row
          if (lane < chunks)
            for (int r = 0; r < cnt; ++r)
              cp_async16(smem_addr(dst + (size_t)r * STAGE_PITCH + 16u * lane), X + (r0 + r) * ldx + 2 * lane);
          cp_async_arrive(fb);
        } else {
          for (int e = lane; e < cnt * nk; e += 32) {
            const int r = e / nk, cc = e - r * nk;
            *(double *)(dst + stage_off(r, cc)) = X[(r0 + r) * ldx + cc];
          }
          __syncwarp();
          mbar_arrive(fb);
        }
        last_i[q] = i;
      }
      if (!ok) break;

    }
    // copies still in flight (only after an abort) land before the CTA leaves
    if (lane == 0)
      for (int q = 0; q < TQ_NSTAGE; ++q)
        if (last_i[q] >= 0) mbar_wait(bar(BAR_FULL + q), (uint32_t)(last_i[q] & 1));
  } else if (warp == W_MMA) {
    // ------------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint64_t ad0 = umma_desc(smem_addr(As), A_LBO, A_SBO), bd0 = umma_desc(smem_addr(Bs), B_LBO, B_SBO);
      for (int i = 0; i < ntiles; ++i) {
        const uint32_t ph = (uint32_t)(i & 1);
        // half 0: K-steps 0 and 1 (A's K-blocks 0, 1), once the previous tile's half 0 is read
        if (!mbar_wait_or_abort(bar(BAR_TEMPTY + 0), ph ^ 1, abort_flag, lim) ||
            !mbar_wait_or_abort(bar(BAR_AFULL + 0), ph, abort_flag, lim) ||
            !mbar_wait_or_abort(bar(BAR_AFULL + 1), ph, abort_flag, lim)) {
          if (!*abort_flag) set_abort(abort_flag, st);
          break;
        }
        fence_after_sync();
        // opaque per tile: keeps the compiler from hoisting all descriptor sums into registers
        uint64_t ad = ad0, bd = bd0;
        asm volatile("" : "+l"(ad), "+l"(bd));
        issue_half_kstep<0, 0, NDA>(tmem, ad, bd);
        issue_half_kstep<0, 1, NDA>(tmem, ad, bd);
        umma_commit(bar(BAR_HDONE + 0));
        if (NH == 1) {  // no second half: A's K-blocks 0 and 1 are free once these complete
          umma_commit(bar(BAR_KFREE + 0));
          umma_commit(bar(BAR_KFREE + 1));
          continue;
        }
        // half 1: all four K-steps; after K-step c no MMA of this tile reads A's K-block c
        if (!mbar_wait_or_abort(bar(BAR_TEMPTY + 1), ph ^ 1, abort_flag, lim) ||
            !mbar_wait_or_abort(bar(BAR_AFULL + 2), ph, abort_flag, lim) ||
            !mbar_wait_or_abort(bar(BAR_AFULL + 3), ph, abort_flag, lim)) {
          if (!*abort_flag) set_abort(abort_flag, st);
          break;
        }
        fence_after_sync();
        issue_half_kstep<1, 0, NDA>(tmem, ad, bd);
        umma_commit(bar(BAR_KFREE + 0));
        issue_half_kstep<1, 1, NDA>(tmem, ad, bd);
        umma_commit(bar(BAR_KFREE + 1));
        issue_half_kstep<1, 2, NDA>(tmem, ad, bd);
        umma_commit(bar(BAR_KFREE + 2));
        issue_half_kstep<1, 3, NDA>(tmem, ad, bd);
        umma_commit(bar(BAR_KFREE + 3));
        umma_commit(bar(BAR_HDONE + 1));
      }
      // every MMA issued so far completes before tensor memory is released
      umma_commit(bar(BAR_DRAIN));
      mbar_wait(bar(BAR_DRAIN), 0);
    }
    __syncwarp();
  } else if (warp < W_FLUSH0) {
    // ------------------------------------------------------------------ slicers
    // Each warp takes one 8-row group in sub-tiles grp and grp + 2.  Lane (r, kk, qq) holds
    // row r of the group in sub-tile grp + 2 qq, K groups kg = 2c + kk (8 columns each) for the
    // four K-blocks c: it reads them into registers (freeing the stage slots at once), then, as
    // the previous tile's K-steps release A's blocks, writes one 16-byte core-matrix row per
    // slice and K-block.  A warp's store covers four whole core matrices.
    const int grp = warp >> 2, sg = warp & 3;
    const int r = lane & 7, kk = (lane >> 3) & 1, qq = lane >> 4;
    const int q = grp + 2 * qq, row = TQ_SUB * q + 8 * sg + r;
    uint8_t *const arow = As + (size_t)(row >> 3) * A_SBO + (size_t)(row & 7) * 16;
    bool ok = true;
    for (int i = 0; i < ntiles && ok; ++i) {
      unsigned long long e[NKB][8];
      for (int u = 0; u < 2; ++u)
        if (!mbar_wait_or_abort(bar(BAR_FULL + grp + 2 * u), (uint32_t)(i & 1), abort_flag, lim)) ok = false;
      if (!ok) break;
      const int rr = 8 * sg + r;  // row within the sub-tile
      const bool live = rr < sub_rows(i, q);
      const uint8_t *src = stage + (size_t)q * STAGE_BYTES;
      uint32_t mxh = 0;  // largest high word without its sign: bits 20-30 are the exponent field
#pragma unroll
      for (int c = 0; c < NKB; ++c) {
        const int kg = 2 * c + kk;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c0 = 8 * kg + 2 * u;
          // REV: K indices c0, c0 + 1 are columns nk - 1 - c0, nk - 2 - c0 (nk even: one aligned pair)
          const int sc = REV ? max(nk - 2 - c0, 0) : c0;
          const ulonglong2 raw = *(const ulonglong2 *)(src + stage_off(rr, sc));
          const unsigned long long v0 = REV ? raw.y : raw.x, v1 = REV ? raw.x : raw.y;
          if (FULLN) {
            e[c][2 * u] = v0;
            e[c][2 * u + 1] = v1;
          } else {
            e[c][2 * u] = (live && c0 < nk) ? v0 : 0ULL;
            e[c][2 * u + 1] = (live && c0 + 1 < nk) ? v1 : 0ULL;
          }
          mxh = max(mxh, max((uint32_t)(e[c][2 * u] >> 32) & 0x7fffffffu, (uint32_t)(e[c][2 * u + 1] >> 32) & 0x7fffffffu));
        }
      }
      int mx = (int)(mxh >> 20);
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bar(BAR_EMPTY + grp));
        mbar_arrive(bar(BAR_EMPTY + grp + 2));
      }
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 8));  // the other half of the row
      const int E = scale_exp(mx);
#pragma unroll
      for (int c = 0; c < NKB; ++c) {
        if (i > 0 && !mbar_wait_or_abort(bar(BAR_KFREE + c), (uint32_t)((i - 1) & 1), abort_flag, lim)) {
          ok = false;
          break;
        }
        // rowexp[i % 3] was last read by the flushers of tile i - 3, which finished before
        // the previous tile's half 1 (and so its K-block 0) could start
        if (c == 0 && kk == 0) rowexp[(i % 3) * TQ_ROWS + row] = E;
        uint32_t w[4][NDIG8];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          digits8_biased(fix54_biased(e[c][2 * u], E), fix54_biased(e[c][2 * u + 1], E), w[u]);
        uint8_t *dst = arow + (size_t)(2 * c + kk) * A_LBO;
#pragma unroll
        for (int p = NDIG8 - NDA; p < NDIG8; ++p)  // slices s = NDIG8 - 1 - p < NDA
          *(uint4 *)(dst + (size_t)(NDIG8 - 1 - p) * A_SLICE) = make_uint4(w[0][p], w[1][p], w[2][p], w[3][p]);
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(BAR_AFULL + c));
      }
    }
    if (!ok && lane == 0 && !*abort_flag) set_abort(abort_flag, st);
  } else {
    // ------------------------------------------------------------------ recombination
    // Half h is final once its MMAs are done.  Each warp reads 16 of the half's 32 columns for
    // its 32 TMEM lanes (rows) with 16-lane x 8-column loads: thread t gets rows t / 4 and
    // t / 4 + 8 of a 16-row group, columns 2 (t % 4) and 2 (t % 4) + 1, so that four threads
    // store one row's 64-byte segment.  One 16-row group (16 columns, all eight regions) per wait.
    const int f = warp - W_FLUSH0, quad = f & 3, cq = f >> 2;  // warp % 4 == quad: lanes 32 quad ..
    const int tr = lane >> 2, tc2 = 2 * (lane & 3);
    double res2 = 0.0, ref2 = 0.0;  // RESID sums of this thread
    bool ok = true;
    for (int i = 0; i < ntiles && ok; ++i) {
      const int64_t row0 = r_begin + (int64_t)i * TQ_ROWS + 32 * quad;
      int er[2][2];
#pragma unroll 1
      for (int h = 0; h < NH; ++h) {
        if (!mbar_wait_or_abort(bar(BAR_HDONE + h), (uint32_t)(i & 1), abort_flag, lim)) {
          ok = false;
          break;
        }
        fence_after_sync();
        if (h == 0)
#pragma unroll
          for (int rg = 0; rg < 2; ++rg)
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) er[rg][hr] = rowexp[(i % 3) * TQ_ROWS + 32 * quad + 16 * rg + 8 * hr + tr];
#pragma unroll 1
        for (int rg = 0; rg < 2; ++rg) {  // 16-row group
          const uint32_t ta = tmem + ((uint32_t)(32 * quad + 16 * rg) << 16) + (uint32_t)(256 * h + 16 * cq);
          // EPI_ADDREF: this group's reference pairs are requested before the tensor-memory loads,
          // so their latency overlaps the read-back (pairs that are not whole are read below)
          double2 rvh[2][2];
          if (EPI == EPI_ADDREF) {
#pragma unroll
            for (int cc = 0; cc < 2; ++cc)
#pragma unroll
              for (int hr = 0; hr < 2; ++hr) {
                const int64_t grow = row0 + 16 * rg + 8 * hr + tr;
                const int k0 = 32 * h + 16 * cq + 8 * cc + tc2;
                const bool whole = grow < r_end && k0 + 1 < nn && (REV || FULLN || vec_store);
                const int64_t col = REV ? (int64_t)nn - 2 - k0 : (int64_t)k0;
                rvh[cc][hr] = whole ? *(const double2 *)(Vref + grow * ldvr + col) : make_double2(0.0, 0.0);
              }
          }
          // NCC of the two 8-column chunks per tensor-memory wait: both (more loads in flight), or
          // one at a time where the add-to-reference epilogue's live values would not fit the
          // registers otherwise
          constexpr int NCC = EPI == EPI_ADDREF ? 1 : 2;
#pragma unroll
          for (int c2 = 0; c2 < 2 / NCC; ++c2) {
          uint32_t v[NCC][8][4];
#pragma unroll
          for (int li = 0; li < NCC; ++li)
#pragma unroll
            for (int g = 0; g < 8; ++g) {
              if (g < NDA + 1) {
                tmem_ld16x256(ta + (uint32_t)(32 * g + 8 * (c2 * NCC + li)), v[li][g]);
              } else {  // six-digit products: region 7 holds nothing
                v[li][g][0] = v[li][g][1] = v[li][g][2] = v[li][g][3] = 0u;
              }
            }
          tmem_wait_ld();
#pragma unroll
          for (int li = 0; li < NCC; ++li) tmem_regs_ready(v[li]);
          if (rg == 1 && c2 == 2 / NCC - 1) {  // this half read: the next tile's MMAs of the half may start
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(BAR_TEMPTY + h));
          }
#pragma unroll
          for (int li = 0; li < NCC; ++li) {
            const int cc = c2 * NCC + li;
            const int k0 = 32 * h + 16 * cq + 8 * cc + tc2;
            const int e0 = scale_exp(colexp[k0]) - 56, e1 = scale_exp(colexp[k0 + 1]) - 56;
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
              const int64_t grow = row0 + 16 * rg + 8 * hr + tr;
              const long long t0 = recombine_b8(v[li][0][2 * hr], v[li][1][2 * hr], v[li][2][2 * hr], v[li][3][2 * hr],
                                                v[li][4][2 * hr], v[li][5][2 * hr], v[li][6][2 * hr], v[li][7][2 * hr]);
              const long long t1 = recombine_b8(v[li][0][2 * hr + 1], v[li][1][2 * hr + 1], v[li][2][2 * hr + 1],
                                                v[li][3][2 * hr + 1], v[li][4][2 * hr + 1], v[li][5][2 * hr + 1],
                                                v[li][6][2 * hr + 1], v[li][7][2 * hr + 1]);
              // T / 2^12 (|.| < 2^63) times 2^(E_i + F_k - 56)
              const double y0 = int_times_pow2_cvt(t0, er[rg][hr] + e0);
              const double y1 = int_times_pow2_cvt(t1, er[rg][hr] + e1);
              if (grow < r_end) {
                if (RESID) {
                  const double *vp = Vref + grow * ldvr + k0;
                  if (k0 < nn) {
                    const double v = vp[0], d = v - y0;
                    res2 = fma(d, d, res2);
                    ref2 = fma(v, v, ref2);
                  }
                  if (k0 + 1 < nn) {
                    const double v = vp[1], d = v - y1;
                    res2 = fma(d, d, res2);
                    ref2 = fma(v, v, ref2);
                  }
                } else if (REV) {
                  // columns nn - 1 - k0 (y0) and nn - 2 - k0 (y1): one aligned pair (nn even)
                  const int64_t cpos = (int64_t)nn - 2 - k0;
                  if (k0 + 1 < nn) {
                    double a1 = y1, a0 = y0;
                    if (EPI == EPI_ADDREF) {
                      const double2 rv = rvh[cc][hr];
                      a1 = add_fixed(rv.x, t1, er[rg][hr] + e1);
                      a0 = add_fixed(rv.y, t0, er[rg][hr] + e0);
                    }
                    *(double2 *)(Y + grow * ldy + cpos) = make_double2(a1, a0);
                  }
                } else {
                  double *yp = Y + grow * ldy + k0;
                  double a0 = y0, a1 = y1;
                  if (FULLN || (vec_store && k0 + 1 < nn)) {
                    if (EPI == EPI_ADDREF) {
                      const double2 rv = rvh[cc][hr];
                      a0 = add_fixed(rv.x, t0, er[rg][hr] + e0);
                      a1 = add_fixed(rv.y, t1, er[rg][hr] + e1);
                    }
                    *(double2 *)yp = make_double2(a0, a1);
                  } else {
                    const double *rp = Vref + grow * ldvr + k0;
                    if (k0 < nn) yp[0] = EPI == EPI_ADDREF ? add_fixed(rp[0], t0, er[rg][hr] + e0) : a0;
                    if (k0 + 1 < nn) yp[1] = EPI == EPI_ADDREF ? add_fixed(rp[1], t1, er[rg][hr] + e1) : a1;
                  }
                }
              }
            }
          }
          }  // c2
        }
      }
      if (SIG && ok) {  // this warp's rows of tile i are stored
        __syncwarp();
        if (lane == 0) st_release_cluster_u32(sig + 4u * (uint32_t)f, (uint32_t)(i + 1));
      }
    }
    if (!ok && lane == 0 && !*abort_flag) set_abort(abort_flag, st);
    if (SIG && !ok && lane == 0) st_release_cluster_u32(sig + 4u * (uint32_t)f, PRODUCER_DONE);
    if (RESID) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        res2 += __shfl_xor_sync(0xffffffffu, res2, o);
        ref2 += __shfl_xor_sync(0xffffffffu, ref2, o);
      }
      if (lane == 0) {
        atomicAdd(&sums[0], res2);
        atomicAdd(&sums[1], ref2);
      }
    }
  }

  __syncthreads();
  fence_after_sync();
  if (warp == W_MMA) tmem_free(tmem, TQ_TMEM_COLS);
}

template <bool FULLN, bool REV, int EPI, int NH, int NDA>
__global__ void __launch_bounds__(TQ_THREADS, 1)
    k_trsm_oz(const double *__restrict__ X, int64_t ldx, double *Y, int64_t ldy, int64_t m, int nk, int nn,
              const double *__restrict__ Bp, int b_ld, int64_t rows_per_cta, int load_mode, bool vec_store,
              const double *Vref, int64_t ldvr, double *sums, DevStatus *st) {
  if (status_failed(st)) return;
  trsm_oz_cta<FULLN, REV, EPI, NH, NDA, false>(X, ldx, Y, ldy, m, nk, nn, Bp, b_ld, rows_per_cta, load_mode, vec_store,
                                               Vref, ldvr, sums, st, (int)blockIdx.x, 0u);
}

bool trsm_oz_supported(int64_t n) { return n >= 1 && n <= TQ_NP; }

template <bool REV, int EPI, int NDA>
cudaError_t launch_trsm_oz_t(const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t m, int64_t nk, int64_t nn,
                             const double *Bpacked, const double *Vref, int64_t ldvr, double *sums, int num_sms,
                             DevStatus *st, cudaStream_t s, int b_ld = 0) {
  if (m <= 0) return cudaSuccess;
  int64_t ctas = std::min<int64_t>(ceil_div(m, TQ_ROWS), (int64_t)num_sms);
  const int64_t rows_per_cta = ceil_div(ceil_div(m, ctas), TQ_ROWS) * TQ_ROWS;
  ctas = ceil_div(m, rows_per_cta);
  // bulk copies need 16-byte aligned rows of a multiple of 16 bytes
  const int load_mode =
      (((uintptr_t)X & 15) == 0 && (ldx * 8) % 16 == 0 && (nk * 8) % 16 == 0) ? LOAD_ASYNC : LOAD_PLAIN;
  const bool vec_store = ((uintptr_t)Y & 15) == 0 && (ldy % 2) == 0 &&
                         (EPI != EPI_ADDREF || (((uintptr_t)Vref & 15) == 0 && (ldvr % 2) == 0));
  if (REV && (!vec_store || (nk % 2) != 0 || (nn % 2) != 0)) return cudaErrorInvalidValue;
  // one column half when both widths fit in 32 (B then needs K < 32 only)
  const bool half = nk <= 32 && nn <= 32 && !REV && EPI != EPI_RESID;
  // the full-width form stores 16-byte pairs unconditionally: only with aligned rows of Y
  const int64_t width = half ? 32 : TQ_NP;
  const bool full = nk == width && nn == width && vec_store && EPI != EPI_RESID;
  decltype(&k_trsm_oz<false, REV, EPI, 2, NDA>) kern;
  if (half)
    kern = full ? k_trsm_oz<true, false, EPI == EPI_RESID ? EPI_STORE : EPI, 1, NDA>
                : k_trsm_oz<false, false, EPI == EPI_RESID ? EPI_STORE : EPI, 1, NDA>;
  else
    kern = full ? k_trsm_oz<true, REV, EPI, 2, NDA> : k_trsm_oz<false, REV, EPI, 2, NDA>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TQ_SMEM);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)ctas, TQ_THREADS, TQ_SMEM, s>>>(X, ldx, Y, ldy, m, (int)nk, (int)nn, Bpacked, b_ld, rows_per_cta,
                                                   load_mode, vec_store, Vref, ldvr, sums, st);
  return cudaGetLastError();
}

cudaError_t launch_trsm_oz(const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t m, int64_t n,
                           const double *Bpacked, int num_sms, DevStatus *st, cudaStream_t s, int digits) {
  if (digits == 6)
    return launch_trsm_oz_t<false, EPI_STORE, 6>(X, ldx, Y, ldy, m, n, n, Bpacked, nullptr, 0, nullptr, num_sms, st, s);
  return launch_trsm_oz_t<false, EPI_STORE, 7>(X, ldx, Y, ldy, m, n, n, Bpacked, nullptr, 0, nullptr, num_sms, st, s);
}

cudaError_t launch_trsm_oz_block(const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t m, int64_t nk,
                                 int64_t nn, const double *Bpacked, bool reverse, const double *Ref, int64_t ldref,
                                 int num_sms, DevStatus *st, cudaStream_t s, int b_ld) {
  if (b_ld && (reverse || b_ld < nn)) return cudaErrorInvalidValue;
  if (!Ref) {
    if (reverse) return cudaErrorInvalidValue;
    return launch_trsm_oz_t<false, EPI_STORE, 7>(X, ldx, Y, ldy, m, nk, nn, Bpacked, nullptr, 0, nullptr, num_sms, st, s,
                                                 b_ld);
  }
  if (reverse)
    return launch_trsm_oz_t<true, EPI_ADDREF, 7>(X, ldx, Y, ldy, m, nk, nn, Bpacked, Ref, ldref, nullptr, num_sms, st, s);
  return launch_trsm_oz_t<false, EPI_ADDREF, 7>(X, ldx, Y, ldy, m, nk, nn, Bpacked, Ref, ldref, nullptr, num_sms, st, s,
                                                b_ld);
}

cudaError_t launch_trsm_oz_resid(const double *Q, int64_t ldq, const double *V, int64_t ldv, int64_t m, int64_t n,
                                 const double *Rpacked, double *sums, int num_sms, DevStatus *st, cudaStream_t s) {
  return launch_trsm_oz_t<false, EPI_RESID, 7>(Q, ldq, nullptr, 0, m, n, n, Rpacked, V, ldv, sums, num_sms, st, s);
}

// ---------------------------------------------------------------------------------------------
// The first row pass of rand_cholQR in one launch (Algorithm 3: W = V R_s^{-1}, then the Gram
// G = W^T W of the Cholesky pass, Algorithm 2 step 1), on pairs of CTAs of one cluster over one
// row range each: the solver runs the solve above (full width, n = 64) and stores W; after each
// 128-row tile its eight read-back warps publish their progress in the solver's shared memory,
// and its partner runs the Gram of those rows (gram_split_body.cuh), each group once the tile
// that holds it is stored, so W reaches the Gram from L2 a few tiles behind the solve instead
// of from a second pass over HBM.  V is read once and W written once; G is accumulated as by
// k_gram_split.  Each role is bound by its own instruction issue, not by HBM, and runs on half
// the SMs, so the launch takes about as long as the two separate passes together or longer.
namespace {
constexpr size_t SG_BODY = TQ_SMEM > GsCfg<TQ_NP>::SMEM ? TQ_SMEM : GsCfg<TQ_NP>::SMEM;
constexpr size_t SG_OFF_SIG = (SG_BODY + 15) / 16 * 16;
constexpr size_t SG_SMEM = SG_OFF_SIG + 4 * PRODUCER_WARPS;
static_assert(SG_SMEM <= 232448, "shared memory budget");
static_assert(GS_THREADS <= TQ_THREADS && TQ_ROWS == TQ_PRODUCER_ROWS, "paired roles");
// CTAs per cluster (SG_CL / 2 pairs) and the rank bit that tells the roles apart: rank r solves
// when r & SG_ROLE is 0, and its Gram partner is rank r ^ SG_ROLE.  Clusters of four with the
// solves on ranks 0, 1 and the Grams on ranks 2, 3, so that two SMs sharing a TPC run the same
// role.  One launch at m = 2^23, n = 64: 4.93 ms this way (36 clusters, 144 SMs); 7.65 ms with
// the roles alternating (ranks 0, 2 solve) and 7.33 ms with clusters of two (76 clusters) --
// an SM slows down sharply when its TPC neighbour runs the other role's code.  Each role alone
// at the same size (its partner idle): the solve 4.23 ms, the Gram 4.43 ms.
constexpr int SG_CL = 4, SG_ROLE = 2;
}  // namespace

template <int NDA, int CL, int ROLE>
__global__ void __launch_bounds__(TQ_THREADS, 1)
    k_solve_gram(const double *__restrict__ V, int64_t ldv, double *W, int64_t m, const double *__restrict__ Bp,
                 double *Gp, int64_t rows_per_pair, DevStatus *st) {
  extern __shared__ __align__(1024) uint8_t sg_smem[];
  const uint32_t rank = cluster_rank();
  const bool solver = (rank & (uint32_t)ROLE) == 0;
  // pair index: the cluster's pairs in order of the rank bits other than the role bit
  const uint32_t in_cl = (rank & (uint32_t)(ROLE - 1)) | ((rank >> 1) & ~(uint32_t)(ROLE - 1));
  const int pair = (int)((blockIdx.x / CL) * (CL / 2) + in_cl);
  const bool skip = status_failed(st);
  const uint32_t sig = smem_addr(sg_smem + SG_OFF_SIG);
  if (solver && threadIdx.x < PRODUCER_WARPS)
    ((volatile uint32_t *)(sg_smem + SG_OFF_SIG))[threadIdx.x] = skip ? PRODUCER_DONE : 0u;
  __syncwarp();
  cluster_sync_all();  // the progress words are set before the Gram CTAs read them
  if (!skip) {
    if (solver)
      trsm_oz_cta<true, false, EPI_STORE, 2, NDA, true>(V, ldv, W, TQ_NP, m, TQ_NP, TQ_NP, Bp, 0, rows_per_pair,
                                                       LOAD_ASYNC, true, nullptr, 0, nullptr, st, pair, sig);
    else
      gram_split_cta<TQ_NP, false, true>(W, TQ_NP, m, TQ_NP, Gp, rows_per_pair, GLOAD_ASYNC16, st, pair,
                                         map_shared_rank(sig, rank ^ (uint32_t)ROLE));
  }
  __syncwarp();
  cluster_sync_all();  // neither CTA leaves while the other may still read its shared memory
}

namespace {
template <int NDA>
cudaLaunchConfig_t solve_gram_config(cudaLaunchAttribute *attr, unsigned ctas, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(TQ_THREADS);
  cfg.dynamicSmemBytes = SG_SMEM;
  cfg.stream = s;
  attr->id = cudaLaunchAttributeClusterDimension;
  attr->val.clusterDim.x = SG_CL;
  attr->val.clusterDim.y = 1;
  attr->val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Solve/Gram pairs of the paired kernel that fit on the device at once (0 when none does), per
// device: the clusters that fit times the pairs of a cluster.
template <int NDA>
int solve_gram_pairs(int num_sms, cudaStream_t s) {
  constexpr int MAX_DEV = 64;
  static int cached[MAX_DEV];  // 0: not asked yet; -1: none fits; else the count
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return 0;
  if (cached[dev] == 0) {
    int clusters = 0;
    cudaLaunchAttribute attr;
    const cudaLaunchConfig_t cfg = solve_gram_config<NDA>(&attr, (unsigned)(SG_CL * (num_sms / SG_CL)), s);
    if (cudaFuncSetAttribute(k_solve_gram<NDA, SG_CL, SG_ROLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SG_SMEM) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveClusters(&clusters, k_solve_gram<NDA, SG_CL, SG_ROLE>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;  // not cached: asked again next time
    }
    cached[dev] = clusters > 0 ? clusters * (SG_CL / 2) : -1;
  }
  return cached[dev] > 0 ? cached[dev] : 0;
}

template <int NDA>
cudaError_t launch_solve_gram_t(const double *V, int64_t ldv, double *W, int64_t m, const double *Bpacked,
                                double *Gpacked, int num_sms, DevStatus *st, cudaStream_t s) {
  const int max_pairs = solve_gram_pairs<NDA>(num_sms, s);
  if (max_pairs <= 0) return cudaErrorInvalidConfiguration;
  int64_t pairs = std::min<int64_t>(ceil_div(m, TQ_ROWS), (int64_t)max_pairs);
  const int64_t rows_per_pair = ceil_div(ceil_div(m, pairs), TQ_ROWS) * TQ_ROWS;
  pairs = ceil_div(ceil_div(m, rows_per_pair), SG_CL / 2) * (SG_CL / 2);  // whole clusters (a pair past m idles)
  cudaError_t e = cudaFuncSetAttribute(k_solve_gram<NDA, SG_CL, SG_ROLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SG_SMEM);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr;
  const cudaLaunchConfig_t cfg = solve_gram_config<NDA>(&attr, (unsigned)(2 * pairs), s);
  return cudaLaunchKernelEx(&cfg, k_solve_gram<NDA, SG_CL, SG_ROLE>, V, ldv, W, m, Bpacked, Gpacked, rows_per_pair, st);
}
}  // namespace

bool solve_gram_supported(int64_t n, const double *V, int64_t ldv, const double *W, int64_t ldw, int num_sms) {
  return n == TQ_NP && ldv == TQ_NP && ldw == TQ_NP && ((uintptr_t)V & 15) == 0 && ((uintptr_t)W & 15) == 0 &&
         solve_gram_pairs<7>(num_sms, nullptr) > 0;
}

cudaError_t launch_solve_gram(const double *V, int64_t ldv, double *W, int64_t ldw, int64_t m, int64_t n,
                              const double *Bpacked, double *Gpacked, int num_sms, DevStatus *st, cudaStream_t s,
                              int digits) {
  if (m <= 0) return cudaSuccess;
  if (!solve_gram_supported(n, V, ldv, W, ldw, num_sms)) return cudaErrorInvalidValue;
  return digits == 6 ? launch_solve_gram_t<6>(V, ldv, W, m, Bpacked, Gpacked, num_sms, st, s)
                     : launch_solve_gram_t<7>(V, ldv, W, m, Bpacked, Gpacked, num_sms, st, s);
}

}  // namespace rq
