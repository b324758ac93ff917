// trsm_tc.cu -- Y = X B for an n x n upper-triangular B given by its packed FP64 entries
// (n <= 64), from exact split products on the tensor cores.  rand_cholQR runs both of its
// triangular solves (W = V R_s^{-1} and Q = W R_c^{-1}, Algorithm 3) this way, as products with
// the explicit inverses.
//
// Number format.  Row i of X gets a scale 2^E_i > max_j |x_ij| and column k of B a scale
// 2^F_k > max_j |b_jk|.  x_ij = 2^(E_i - 54) X_ij up to truncation, with the integer
// X_ij = trunc(x_ij 2^(54 - E_i)) written in eight balanced 7-bit digits (tc.cuh), and the
// same for b_jk with digits e.  With slice s = 7 - p (s = 0 the leading digit) the product keeps
// the slice pairs s + t <= 8, gathered by g = s + t into regions of tensor memory:
//   D_g(i, k) = sum_{s + t = g} sum_j d_s(i, j) e_t(j, k),   |D_g| <= 8 * 64 * 2^12 = 2^21,
//   y_ik = 2^(E_i + F_k - 59) T_ik,   T_ik = sum_g 2^(7 (7 - g)) D_g(i, k).
// Regions 0-6 hold exact FP32 integers.  Region 8 is summed first in region 7's columns and
// folded in at weight 2^-7 by the first region-7 MMA (scale-input-d), so that region holds
// D_7 + 2^-7 D_8 rounded to FP32, an error far below T's last unit.  The recombination turns
// the regions into integers, forms T / 8 in 64-bit integer arithmetic and rounds once to FP64.
// Truncation and the dropped pairs (s + t >= 9) weigh about 2^-54 of 2^(E_i + F_k) per term: a
// relative perturbation of each row of X, so the first solve's backward error in V stays at
// that level whatever kappa(V) is.
//
// One CTA per SM, persistent over 128-row tiles; warps specialise:
//   warps 0-7 cut rows into digit slices (shared memory A: 8 slices x 128 rows x 64 K, f16);
//     warps 0-3 take the even 32-row sub-tiles, 4-7 the odd ones, one 8-row group each,
//   warps 8-15 read tensor memory back (TMEM lanes 32 (w & 3) .., 32 columns each),
//     recombine and store rows of Y,
//   warp 16 loads 32-row sub-tiles of X into a three-slot ring with per-row bulk copies,
//   warp 17 owns tensor memory and issues the MMAs,
// handing tiles over through mbarriers.  B's digit slices are built once per CTA.  B is upper
// triangular, so the K-step j in [16c, 16c + 16) meets only columns k >= 16c and its MMAs run
// with N = 64 - 16c.  In place (Y == X) is safe: a tile's rows are read before any are written.
#include "common.cuh"
#include "tc.cuh"

namespace rq {

namespace {
using namespace tc;

constexpr int TQ_ROWS = 128, TQ_NP = 64, TQ_SUB = 32, TQ_NSTAGE = 3;
constexpr int TQ_THREADS = 576;
constexpr int W_FLUSH0 = 8, W_LOAD = 16, W_MMA = 17;
constexpr uint32_t TQ_TMEM_COLS = 512;
// A: K-major, no swizzle.  A slicer lane (row r = lane & 7 of an 8-row group, pair pi =
// lane >> 3 of every K core matrix) stores 4 bytes at r * 16 + pi * 4 of a core matrix: one
// warp store covers one core matrix, all 32 banks.
constexpr uint32_t A_LBO = 128, A_SBO = 8 * A_LBO, A_SLICE = (TQ_ROWS / 8) * A_SBO;
// B: per K-step c a block of (64 - 16c) rows (output column k) x 16 K, 32 bytes per row.
constexpr uint32_t B_SLICE = 160 * 32;
// Staged rows are 528 bytes apart (512 + 16): the slicers' 16-byte reads of eight rows at one
// K offset then fall into eight different bank groups.
constexpr uint32_t STAGE_PITCH = 528;
constexpr uint32_t STAGE_BYTES = TQ_SUB * STAGE_PITCH;
constexpr size_t OFF_B = 0;
constexpr size_t OFF_A = OFF_B + (size_t)NDIG * B_SLICE;
constexpr size_t OFF_STAGE = OFF_A + (size_t)NDIG * A_SLICE;
constexpr size_t OFF_ROWEXP = OFF_STAGE + (size_t)TQ_NSTAGE * STAGE_BYTES;
constexpr size_t OFF_COLEXP = OFF_ROWEXP + 3 * TQ_ROWS * sizeof(int);
constexpr size_t OFF_BARS = OFF_COLEXP + TQ_NP * sizeof(int);
constexpr int NBARS = 2 * TQ_NSTAGE + 7;  // full[3], empty[3], a_full, kdone[4], t_empty, drain
constexpr size_t OFF_MISC = OFF_BARS + NBARS * 8;  // tmem slot, abort flag, slot tags[3]
constexpr size_t TQ_SMEM = OFF_MISC + 32;
static_assert(TQ_SMEM <= 232448, "shared memory budget");

enum LoadMode { LOAD_ROWS = 0, LOAD_PLAIN = 1 };

__device__ __forceinline__ uint32_t b_row0(int c) { return c == 0 ? 0u : c == 1 ? 64u : c == 2 ? 112u : 144u; }

__device__ __forceinline__ void set_abort(volatile int *abort_flag, DevStatus *st) {
  *abort_flag = 1;
  status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
}

// Exponent field of one 8-byte element (FP64, or the leading float of a pair, rebased).
template <bool IN_DF>
__device__ __forceinline__ int elem_expfield(unsigned long long bits) {
  if (IN_DF) {
    const int ef = (int)(((uint32_t)bits >> 23) & 0xff);
    return ef ? ef - 127 + 1023 : 0;
  }
  return (int)((bits >> 52) & 0x7ff);
}

template <bool IN_DF>
__device__ __forceinline__ long long elem_fix(unsigned long long bits, int E) {
  if (IN_DF)
    return fix54(__uint_as_float((uint32_t)bits), E) + fix54(__uint_as_float((uint32_t)(bits >> 32)), E);
  return fix54(__longlong_as_double((long long)bits), E);
}

// Descriptor offsets (16-byte units) of slice s / K-step c in A and slice t / K-step c in B.
__device__ __forceinline__ constexpr uint64_t a_off(int s, int c) { return ((uint64_t)s * A_SLICE + (uint64_t)c * 2 * A_LBO) >> 4; }
__device__ __forceinline__ constexpr uint64_t b_off(int t, int c) {
  return ((uint64_t)t * B_SLICE + (uint64_t)(c == 0 ? 0 : c == 1 ? 64 : c == 2 ? 112 : 144) * 32) >> 4;
}

// A tile's MMAs, fully unrolled so that every descriptor is a base plus a constant (a single
// issuing thread otherwise spends more time forming descriptors than the tensor core spends on
// the products).  Region 8 goes first, into region 7's columns, for every K-step; then the main
// products K-step by K-step.  After main K-step c nothing reads A's K-block c again and no
// later product touches columns < 16 (c + 1), so a commit there releases that block of A to
// the next tile's slicers and columns 16c .. 16c + 15 of every region to the read-back.
__device__ __forceinline__ void issue_region8(uint32_t tmem, uint64_t ad0, uint64_t bd0) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint32_t idesc = umma_idesc_f16(TQ_ROWS, TQ_NP - 16 * c);
#pragma unroll
    for (int s = 1; s < NDIG; ++s)
      umma_bf16(tmem + (uint32_t)(7 * 64 + 16 * c), ad0 + a_off(s, c), bd0 + b_off(8 - s, c), idesc,
                (c | (s - 1)) ? 1u : 0u);
  }
}

template <int C>
__device__ __forceinline__ void issue_kstep(uint32_t tmem, uint64_t ad0, uint64_t bd0) {
  const uint32_t idesc = umma_idesc_f16(TQ_ROWS, TQ_NP - 16 * C);
#pragma unroll
  for (int s = 0; s < NDIG; ++s)
#pragma unroll
    for (int t = 0; t < NDIG - s; ++t) {
      const uint32_t d = tmem + (uint32_t)((s + t) * 64 + 16 * C);
      if (C == 0 && s == 0 && t == NDIG - 1)
        umma_scaled7(d, ad0 + a_off(s, C), bd0 + b_off(t, C), idesc);  // D_8 (every K-step) x 2^-7
      else
        umma_bf16(d, ad0 + a_off(s, C), bd0 + b_off(t, C), idesc, (C | s) ? 1u : 0u);
    }
}

}  // namespace

template <bool IN_DF>
__global__ void __launch_bounds__(TQ_THREADS, 1)
    k_trsm_oz(const void *Xin, int64_t ldx, double *Y, int64_t ldy, int64_t m, int n,
              const double *__restrict__ Bp, int64_t rows_per_cta, int load_mode, bool vec_store,
              DevStatus *st) {
  if (status_failed(st)) return;
  extern __shared__ __align__(1024) uint8_t tq_smem[];
  uint8_t *Bs = tq_smem + OFF_B;
  uint8_t *As = tq_smem + OFF_A;
  uint8_t *stage = tq_smem + OFF_STAGE;
  int *rowexp = (int *)(tq_smem + OFF_ROWEXP);
  int *colexp = (int *)(tq_smem + OFF_COLEXP);
  uint64_t *bars = (uint64_t *)(tq_smem + OFF_BARS);
  uint32_t *tmem_slot = (uint32_t *)(tq_smem + OFF_MISC);
  volatile int *abort_flag = (volatile int *)(tq_smem + OFF_MISC + 4);
  // slot_tag[q]: the sub-tile the loader has assigned to stage slot q.  Two slicer groups take
  // alternate sub-tiles, so a group can reach a slot's next use while the other group's load
  // into it is still in flight; waiting for the tag first keeps the full barrier's parity
  // unambiguous (the wait then always targets the phase in progress).
  volatile int *slot_tag = (volatile int *)(tq_smem + OFF_MISC + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full0 = smem_addr(&bars[0]), empty0 = smem_addr(&bars[TQ_NSTAGE]);
  const uint32_t a_full = smem_addr(&bars[2 * TQ_NSTAGE]);
  const uint32_t kdone0 = smem_addr(&bars[2 * TQ_NSTAGE + 1]);  // kdone[c] at kdone0 + 8c
  const uint32_t t_empty = smem_addr(&bars[2 * TQ_NSTAGE + 5]), drain = smem_addr(&bars[2 * TQ_NSTAGE + 6]);

  if (tid == 0) {
    for (int q = 0; q < TQ_NSTAGE; ++q) {
      mbar_init_count(full0 + 8 * q, 1);
      mbar_init_count(empty0 + 8 * q, 4);
    }
    mbar_init_count(a_full, 8);
    for (int c = 0; c < 4; ++c) mbar_init_count(kdone0 + 8 * c, 1);
    mbar_init_count(t_empty, 8);
    mbar_init_count(drain, 1);
    *abort_flag = 0;
    for (int q = 0; q < TQ_NSTAGE; ++q) slot_tag[q] = -1;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (tid < TQ_NP) colexp[tid] = 0;
  if (warp == W_MMA) tmem_alloc(tmem_slot, TQ_TMEM_COLS);
  __syncthreads();

  // ---- B's digit slices (all threads, once)
  for (int e = tid; e < TQ_NP * TQ_NP; e += TQ_THREADS) {
    const int k = e >> 6, j = e & 63;
    if (k < n && j <= k) atomicMax(&colexp[k], expfield<false>(Bp + tri_idx(j, k)));
  }
  __syncthreads();
  for (int e = tid; e < TQ_NP * TQ_NP / 2; e += TQ_THREADS) {
    const int k = e >> 5, j = 2 * (e & 31), c = j >> 4;
    if (k < 16 * c) continue;  // block c holds rows k >= 16c only
    const int F = scale_exp(colexp[k]);
    const long long za = (k < n && j <= k) ? fix54(Bp[tri_idx(j, k)], F) : 0;
    const long long zb = (k < n && j + 1 <= k) ? fix54(Bp[tri_idx(j + 1, k)], F) : 0;
    uint32_t w[NDIG];
    digits2(za, zb, w);
    const int kk = k - 16 * c, jj = j & 15;
    const uint32_t off = b_row0(c) * 32 + (kk >> 3) * 256 + (jj >> 3) * 128 + (kk & 7) * 16 + (jj & 7) * 2;
#pragma unroll
    for (int p = 0; p < NDIG; ++p) *(uint32_t *)(Bs + (NDIG - 1 - p) * B_SLICE + off) = w[p];
  }
  fence_async_smem();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  const int ntiles = r_end > r_begin ? (int)((r_end - r_begin + TQ_ROWS - 1) / TQ_ROWS) : 0;
  auto sub_rows = [&](int i, int q) -> int {
    const int64_t r0 = r_begin + (int64_t)i * TQ_ROWS + TQ_SUB * q;
    return r0 < r_end ? (int)imin64(TQ_SUB, r_end - r0) : 0;
  };

  if (warp == W_LOAD) {
    // ------------------------------------------------------------------ loader
    int last_u[TQ_NSTAGE];
#pragma unroll
    for (int q = 0; q < TQ_NSTAGE; ++q) last_u[q] = -1;
    for (int i = 0; i < ntiles && !*abort_flag; ++i) {
      bool ok = true;
      for (int q = 0; q < 4; ++q) {
        const int u = 4 * i + q, slot = u % TQ_NSTAGE;
        if (!mbar_wait_or_abort(empty0 + 8 * slot, ((u / TQ_NSTAGE) & 1) ^ 1, abort_flag)) {
          if (lane == 0 && !*abort_flag) set_abort(abort_flag, st);
          ok = false;
          break;
        }
        const int64_t r0 = r_begin + (int64_t)i * TQ_ROWS + TQ_SUB * q;
        const int cnt = sub_rows(i, q);
        uint8_t *dst = stage + (size_t)slot * STAGE_BYTES;
        const uint32_t fb = full0 + 8 * slot;
        if (lane == 0) slot_tag[slot] = u;
        if (cnt > 0 && load_mode == LOAD_ROWS) {
          if (lane == 0) mbar_expect_tx(fb, (uint32_t)cnt * (uint32_t)n * 8u);
          __syncwarp();
          for (int r = lane; r < cnt; r += 32)
            bulk_load(smem_addr(dst + r * STAGE_PITCH), (const uint8_t *)Xin + (size_t)(r0 + r) * (size_t)ldx * 8,
                      (uint32_t)n * 8u, fb);
        } else {
          const unsigned long long *src = (const unsigned long long *)Xin;
          for (int e = lane; e < cnt * n; e += 32) {
            const int r = e / n, cc = e - r * n;
            *(unsigned long long *)(dst + r * STAGE_PITCH + 8 * cc) = src[(r0 + r) * ldx + cc];
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(fb);
        }
        last_u[slot] = u;
      }
      if (!ok) break;
    }
    // copies still in flight (only after an abort) land before the CTA leaves
    if (lane == 0)
      for (int q = 0; q < TQ_NSTAGE; ++q)
        if (last_u[q] >= 0) mbar_wait(full0 + 8 * q, (last_u[q] / TQ_NSTAGE) & 1);
  } else if (warp == W_MMA) {
    // ------------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint64_t ad0 = umma_desc(smem_addr(As), A_LBO, A_SBO), bd0 = umma_desc(smem_addr(Bs), 128, 256);
      for (int i = 0; i < ntiles; ++i) {
        if (!mbar_wait_or_abort(a_full, i & 1, abort_flag) ||
            !mbar_wait_or_abort(t_empty, (i & 1) ^ 1, abort_flag)) {
          if (!*abort_flag) set_abort(abort_flag, st);
          break;
        }
        fence_after_sync();
        // opaque per tile: keeps the compiler from hoisting all 172 descriptor sums into registers
        uint64_t ad = ad0, bd = bd0;
        asm volatile("" : "+l"(ad), "+l"(bd));
        issue_region8(tmem, ad, bd);
        issue_kstep<0>(tmem, ad, bd);
        umma_commit(kdone0);
        issue_kstep<1>(tmem, ad, bd);
        umma_commit(kdone0 + 8);
        issue_kstep<2>(tmem, ad, bd);
        umma_commit(kdone0 + 16);
        issue_kstep<3>(tmem, ad, bd);
        umma_commit(kdone0 + 24);
      }
      // every MMA issued so far completes before tensor memory is released
      umma_commit(drain);
      mbar_wait(drain, 0);
    }
    __syncwarp();
  } else if (warp < W_FLUSH0) {
    // ------------------------------------------------------------------ slicers
    // Each warp takes one 8-row group in sub-tiles grp and grp + 2, reads both into registers
    // (freeing the stage slots at once), then writes A block by block as the previous tile's
    // K-steps release them.
    const int grp = warp >> 2, sg = warp & 3;
    const int r = 8 * sg + (lane & 7), pi = lane >> 3;  // pi: column pair within each K core matrix
    bool ok = true;
    for (int i = 0; i < ntiles && ok; ++i) {
      unsigned long long ea[2][8], eb[2][8];
      int E[2];
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int q = grp + 2 * qq, u = 4 * i + q, slot = u % TQ_NSTAGE;
        bool tagged = false;
        for (int it = 0; it < MAX_WAIT && !tagged && !*abort_flag; ++it) tagged = slot_tag[slot] == u;
        if (!tagged || !mbar_wait_or_abort(full0 + 8 * slot, (u / TQ_NSTAGE) & 1, abort_flag)) {
          ok = false;
          break;
        }
        const int cnt = sub_rows(i, q);
        const uint8_t *src = stage + (size_t)slot * STAGE_BYTES + r * STAGE_PITCH + 16 * pi;
        int mx = 0;
#pragma unroll
        for (int kg = 0; kg < 8; ++kg) {  // columns 8 kg + 2 pi, 8 kg + 2 pi + 1 of row r
          const ulonglong2 raw = *(const ulonglong2 *)(src + 64 * kg);
          const int c0 = 8 * kg + 2 * pi;
          ea[qq][kg] = (r < cnt && c0 < n) ? raw.x : 0ULL;
          eb[qq][kg] = (r < cnt && c0 + 1 < n) ? raw.y : 0ULL;
          mx = max(mx, max(elem_expfield<IN_DF>(ea[qq][kg]), elem_expfield<IN_DF>(eb[qq][kg])));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * slot);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
        E[qq] = scale_exp(mx);
        if (pi == 0) rowexp[(i % 3) * TQ_ROWS + TQ_SUB * q + r] = E[qq];
      }
      if (!ok) break;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (i > 0 && !mbar_wait_or_abort(kdone0 + 8 * c, (i - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
          const int row = TQ_SUB * (grp + 2 * qq) + r;
          uint8_t *dst = As + (size_t)(row >> 3) * A_SBO + (row & 7) * 16 + pi * 4;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const int kg = 2 * c + kk;
            uint32_t w[NDIG];
            digits2(elem_fix<IN_DF>(ea[qq][kg], E[qq]), elem_fix<IN_DF>(eb[qq][kg], E[qq]), w);
#pragma unroll
            for (int p = 0; p < NDIG; ++p) *(uint32_t *)(dst + (size_t)(NDIG - 1 - p) * A_SLICE + kg * A_LBO) = w[p];
          }
        }
      }
      if (!ok) break;
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(a_full);
    }
    if (!ok && lane == 0 && !*abort_flag) set_abort(abort_flag, st);
  } else {
    // ------------------------------------------------------------------ recombination
    // Column block b (16 columns) of every region is final once K-step b is done; each warp
    // reads 8 of its columns for its 32 TMEM lanes.
    const int f = warp - W_FLUSH0, quad = f & 3, half = f >> 2;  // warp % 4 == quad: lanes 32 quad ..
    const int L = 32 * quad + lane;
    const uint32_t tq = tmem + ((uint32_t)(32 * quad) << 16);
    bool ok = true;
    for (int i = 0; i < ntiles && ok; ++i) {
      const int64_t grow = r_begin + (int64_t)i * TQ_ROWS + L;
      double *yrow = Y + grow * ldy;
      int er = 0;
#pragma unroll 1
      for (int b = 0; b < 4; ++b) {
        if (!mbar_wait_or_abort(kdone0 + 8 * b, i & 1, abort_flag)) {
          ok = false;
          break;
        }
        fence_after_sync();
        if (b == 0) er = rowexp[(i % 3) * TQ_ROWS + L];
        // both 4-column groups of this warp's 8 columns are loaded before one wait
        uint32_t v[2][NDIG][4];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
          for (int g = 0; g < NDIG; ++g) tmem_ld4(tq + (uint32_t)(g * 64 + 16 * b + 8 * half + 4 * hh), v[hh][g]);
        tmem_wait_ld();
        tmem_regs_ready(v[0]);
        tmem_regs_ready(v[1]);
        if (b == 3) {  // every region read: the next tile's MMAs may start
          fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(t_empty);
        }
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int k0 = 16 * b + 8 * half + 4 * hh;
          double y[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const long long t = recombine8<3>(v[hh][0][c], v[hh][1][c], v[hh][2][c], v[hh][3][c], v[hh][4][c],
                                              v[hh][5][c], v[hh][6][c], v[hh][7][c]);
            y[c] = int_times_pow2_cvt(t, er + scale_exp(colexp[k0 + c]) - 56);  // T / 8 (|T| < 2^65)
          }
          if (grow < r_end) {
            if (vec_store && k0 + 3 < n) {
              *(double2 *)(yrow + k0) = make_double2(y[0], y[1]);
              *(double2 *)(yrow + k0 + 2) = make_double2(y[2], y[3]);
            } else {
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (k0 + c < n) yrow[k0 + c] = y[c];
            }
          }
        }
      }
    }
    if (!ok && lane == 0 && !*abort_flag) set_abort(abort_flag, st);
  }

  __syncthreads();
  fence_after_sync();
  if (warp == W_MMA) tmem_free(tmem, TQ_TMEM_COLS);
}

bool trsm_oz_supported(int64_t n) { return n >= 1 && n <= TQ_NP; }

cudaError_t launch_trsm_oz(const void *W, bool in_df, int64_t ldw, double *Q, int64_t ldq, int64_t m,
                           int64_t n, const double *Xpacked, int num_sms, DevStatus *st,
                           cudaStream_t s) {
  int64_t ctas = std::min<int64_t>(ceil_div(m, TQ_ROWS), (int64_t)num_sms);
  const int64_t rows_per_cta = ceil_div(ceil_div(m, ctas), TQ_ROWS) * TQ_ROWS;
  ctas = ceil_div(m, rows_per_cta);
  const bool aligned = ((uintptr_t)W & 15) == 0;
  const int load_mode = (aligned && (n * 8) % 16 == 0 && (ldw * 8) % 16 == 0) ? LOAD_ROWS : LOAD_PLAIN;
  const bool vec_store = ((uintptr_t)Q & 15) == 0 && (ldq % 2) == 0;
  cudaError_t e;
  if (in_df) {
    e = cudaFuncSetAttribute(k_trsm_oz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TQ_SMEM);
    if (e != cudaSuccess) return e;
    k_trsm_oz<true><<<(unsigned)ctas, TQ_THREADS, TQ_SMEM, s>>>(W, ldw, Q, ldq, m, (int)n, Xpacked, rows_per_cta,
                                                                load_mode, vec_store, st);
  } else {
    e = cudaFuncSetAttribute(k_trsm_oz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TQ_SMEM);
    if (e != cudaSuccess) return e;
    k_trsm_oz<false><<<(unsigned)ctas, TQ_THREADS, TQ_SMEM, s>>>(W, ldw, Q, ldq, m, (int)n, Xpacked, rows_per_cta,
                                                                 load_mode, vec_store, st);
  }
  return cudaGetLastError();
}

}  // namespace rq
