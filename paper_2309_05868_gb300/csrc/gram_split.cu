// gram_split.cu -- G = W^T W (Algorithm 2 step 1, the Gram of each Cholesky pass) for n <= 64
// from exact split products on the tensor cores.
//
// Rows are taken in groups of 64.  Column j of a group gets a scale 2^E_j > max_r |w_rj| and
// w_rj = 2^(E_j - 54) X_rj up to truncation, with X_rj = trunc(w_rj 2^(54 - E_j)) written in
// eight balanced 7-bit digits d_p (tc.cuh; slice s = 7 - p).  Slices s = 2a and 2a + 1 of all
// 64 columns stack into the 128 rows of A-tile a (TMEM lane 64 * (s & 1) + j); slices t of the
// same buffer are the B operand, several stacked along N, so one MMA covers up to four
// regions.  Region g' (64 columns of tensor memory) gathers the pairs (a, t) with 2a + t = g':
// lanes 0-63 then hold D_g for g = g', lanes 64-127 hold g = g' + 1 (odd s).
//
// Groups form events: the first group of an event takes its column maxima plus one bit of
// headroom as scales, and the following groups keep those scales unless one of their columns
// outgrew them, up to 16 groups.  An event's groups accumulate in the same regions (at most 1024
// rows), so every D is a sum of at most 4 x 1024 digit products of at most 2^12, |D| <= 2^24,
// exact in FP32.  With
//   T_p(j, k) = sum_g' 2^(7 (7 - g')) D_g'(64p + j, k),
// the event's contribution is 2^(E_j + E_k - 59 - 7p) T_p; pairs with g >= 9 (and half of g = 8)
// are dropped, below 2^-54 of 2^(E_j + E_k) per row.  T_p / 256 is formed in 64-bit integers
// (tc::recombine_g7w), converted on the FP64 pipe and added to per-thread FP64 sums; one FP64
// atomic per entry (j <= k) and parity at the end.  Longer events mean fewer read-backs, and the
// next event's products wait for a read-back to finish (tensor memory holds one event).
//
// One CTA per SM, persistent over its row range; warps specialise:
//   warps 0-3 find each group's column scales (first pass over the staged rows) and cut the
//     group into digit slices (second pass; two 64 KB slice buffers, alternating groups),
//   warps 4-11 read the regions back (warp w: TMEM lanes 32 (w & 3) .., columns k in
//     [32 h, 32 h + 32) with h = (w - 4) / 4) and keep the FP64 sums,
//   warp 12 loads 32-row sub-tiles into a four-slot ring with bulk copies (two groups in
//     flight, so a group's rows arrive while the previous one is cut),
//   warp 13 owns tensor memory and issues the MMAs (24 per group), closing an event
//     (commit to the recombination warps) when the next group starts a new one.
#include "common.cuh"
#include "tc.cuh"

namespace rq {

namespace {
using namespace tc;

constexpr int GS_SUB = 32, GS_NP = 64, GS_GROUP = 64;
// Groups per tensor-memory accumulation: 1024 rows keep every region within 4 x 1024 digit
// products of at most 2^12, |D| <= 2^24, exact in FP32.
constexpr int GS_EV_GROUPS = 16;
constexpr int GS_THREADS = 448;
constexpr int GW_LOAD = 12, GW_MMA = 13;
constexpr uint32_t GS_TMEM_COLS = 512;
constexpr uint32_t GS_SLICE = 8192;                 // 64 columns x 64 rows of f16 digits
constexpr uint32_t GS_BUF = NDIG * GS_SLICE;        // one 64-row tile's slices
constexpr uint32_t GS_STAGE = GS_SUB * GS_NP * 8;   // 16 KB sub-tile
constexpr size_t GOFF_SL = 0;
constexpr size_t GOFF_STAGE = GOFF_SL + 2 * (size_t)GS_BUF;
constexpr size_t GOFF_COLE = GOFF_STAGE + 4 * (size_t)GS_STAGE;
constexpr size_t GOFF_EVT = GOFF_COLE + 4 * GS_NP * sizeof(int);  // merge[3], grow[3], ev_grp[4]
constexpr size_t GOFF_BARS = GOFF_EVT + 16 * sizeof(int);
constexpr int GS_NBARS = 17;  // full[4], empty[4], sl_full[2], sl_empty[2], t_full, t_empty, drain,
                              // scale_bar, ev_bar
constexpr size_t GOFF_MISC = GOFF_BARS + GS_NBARS * 8;
constexpr size_t GS_SMEM = GOFF_MISC + 16;
static_assert(GS_SMEM <= 232448, "shared memory budget");

enum GLoadMode { GLOAD_BLOCK = 0, GLOAD_ROWS = 1, GLOAD_PLAIN = 2 };

template <bool IN_DF>
__device__ __forceinline__ int g_expfield(unsigned long long bits) {
  if (IN_DF) {
    const int ef = (int)(((uint32_t)bits >> 23) & 0xff);
    return ef ? ef - 127 + 1023 : 0;
  }
  return (int)((bits >> 52) & 0x7ff);
}

template <bool IN_DF>
__device__ __forceinline__ long long g_fix(unsigned long long bits, int E) {
  if (IN_DF)
    return fix54(__uint_as_float((uint32_t)bits), E) + fix54(__uint_as_float((uint32_t)(bits >> 32)), E);
  return fix54(__longlong_as_double((long long)bits), E);
}

// One 64-row tile's MMAs (K = 64 in four steps): A-tile a = slices 2a, 2a + 1; B = slices t0 ..
// t0 + nt - 1 stacked along N; D = regions 2a + t0 ...
__device__ __forceinline__ void gram_issue_tile(uint32_t tmem, uint64_t d0, bool first) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint64_t kc = (uint64_t)(256 * c) >> 4;
#define GS_MMA(a, t0, nt)                                                                              \
  umma_bf16(tmem + (uint32_t)((2 * (a) + (t0)) * 64), d0 + kc + ((uint64_t)(2 * (a)) * GS_SLICE >> 4), \
            d0 + kc + ((uint64_t)(t0) * GS_SLICE >> 4), umma_idesc_f16(128, 64 * (nt)),                 \
            (first && c == 0 && (a) == 0) ? 0u : 1u)
    GS_MMA(0, 0, 4);
    GS_MMA(0, 4, 4);
    GS_MMA(1, 0, 4);
    GS_MMA(1, 4, 2);
    GS_MMA(2, 0, 4);
    GS_MMA(3, 0, 2);
#undef GS_MMA
  }
}

}  // namespace

template <bool IN_DF>
__global__ void __launch_bounds__(GS_THREADS, 1)
    k_gram_split(const void *Win, int64_t ldw, int64_t m, int n, double *Gp, int64_t rows_per_cta,
                 int load_mode, DevStatus *st) {
  if (status_failed(st)) return;
  const int lim = wait_bound(st, MAX_WAIT);
  extern __shared__ __align__(1024) uint8_t gs_smem[];
  uint8_t *slices = gs_smem + GOFF_SL;
  uint8_t *stage = gs_smem + GOFF_STAGE;
  int *colE = (int *)(gs_smem + GOFF_COLE);
  volatile int *evt = (volatile int *)(gs_smem + GOFF_EVT);
  uint64_t *bars = (uint64_t *)(gs_smem + GOFF_BARS);
  uint32_t *tmem_slot = (uint32_t *)(gs_smem + GOFF_MISC);
  volatile int *abort_flag = (volatile int *)(gs_smem + GOFF_MISC + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full0 = smem_addr(&bars[0]), empty0 = smem_addr(&bars[4]);
  const uint32_t slf0 = smem_addr(&bars[8]), sle0 = smem_addr(&bars[10]);
  const uint32_t t_full = smem_addr(&bars[12]), t_empty = smem_addr(&bars[13]), drain = smem_addr(&bars[14]);
  const uint32_t scale_bar = smem_addr(&bars[15]), ev_bar = smem_addr(&bars[16]);

  if (tid == 0) {
    for (int q = 0; q < 4; ++q) {
      mbar_init_count(full0 + 8 * q, 1);
      mbar_init_count(empty0 + 8 * q, 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init_count(slf0 + 8 * b, 4);
      mbar_init_count(sle0 + 8 * b, 1);
    }
    mbar_init_count(t_full, 1);
    mbar_init_count(t_empty, 8);
    mbar_init_count(drain, 1);
    mbar_init_count(scale_bar, 4);
    mbar_init_count(ev_bar, 1);
    *abort_flag = 0;
    for (int e = 0; e < 16; ++e) evt[e] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == GW_MMA) tmem_alloc(tmem_slot, GS_TMEM_COLS);
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  const int ngroups = r_end > r_begin ? (int)((r_end - r_begin + GS_GROUP - 1) / GS_GROUP) : 0;
  auto sub_rows = [&](int g, int q) -> int {
    const int64_t r0 = r_begin + (int64_t)g * GS_GROUP + GS_SUB * q;
    return r0 < r_end ? (int)imin64(GS_SUB, r_end - r0) : 0;
  };

  if (warp == GW_LOAD) {
    // ------------------------------------------------------------------ loader
    // group g uses slots 2 (g & 1) and 2 (g & 1) + 1: two groups in flight
    int last_g[4] = {-1, -1, -1, -1};
    for (int g = 0; g < ngroups && !*abort_flag; ++g) {
      bool ok = true;
      for (int qq = 0; qq < 2; ++qq) {
        const int q = 2 * (g & 1) + qq;
        if (!mbar_wait_or_abort(empty0 + 8 * q, ((g >> 1) & 1) ^ 1, abort_flag, lim)) {
          if (lane == 0 && !*abort_flag) {
            *abort_flag = 1;
            status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
          }
          ok = false;
          break;
        }
        const int64_t r0 = r_begin + (int64_t)g * GS_GROUP + GS_SUB * qq;
        const int cnt = sub_rows(g, qq);
        uint8_t *dst = stage + (size_t)q * GS_STAGE;
        const uint32_t fb = full0 + 8 * q;
        if (cnt > 0 && load_mode == GLOAD_BLOCK) {
          if (lane == 0) {
            mbar_expect_tx(fb, (uint32_t)cnt * 512u);
            bulk_load(smem_addr(dst), (const uint8_t *)Win + (size_t)r0 * 512, (uint32_t)cnt * 512u, fb);
          }
        } else if (cnt > 0 && load_mode == GLOAD_ROWS) {
          if (lane == 0) mbar_expect_tx(fb, (uint32_t)cnt * (uint32_t)n * 8u);
          __syncwarp();
          for (int r = lane; r < cnt; r += 32)
            bulk_load(smem_addr(dst + r * 512), (const uint8_t *)Win + (size_t)(r0 + r) * (size_t)ldw * 8,
                      (uint32_t)n * 8u, fb);
        } else {
          const unsigned long long *src = (const unsigned long long *)Win;
          for (int e = lane; e < cnt * n; e += 32) {
            const int r = e / n, cc = e - r * n;
            ((unsigned long long *)dst)[r * GS_NP + cc] = src[(r0 + r) * ldw + cc];
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(fb);
        }
        last_g[q] = g;
      }
      if (!ok) break;
    }
    if (lane == 0)
      for (int q = 0; q < 4; ++q)
        if (last_g[q] >= 0) mbar_wait(full0 + 8 * q, (last_g[q] >> 1) & 1);
  } else if (warp == GW_MMA) {
    // ------------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint64_t dA = umma_desc(smem_addr(slices), 128, 1024);
      const uint64_t dB = umma_desc(smem_addr(slices + GS_BUF), 128, 1024);
      // Events: one tensor-memory accumulation = one group, or up to GS_EV_GROUPS consecutive
      // groups with common scales.  evt[8 + (ev & 3)] names the event's last group (whose scale
      // slot the recombination reads).
      int ev = 0, pending_g = -1, last_g = -1;
      bool ok = true;
      auto close_event = [&]() {
        evt[8 + (ev & 3)] = last_g;
        umma_commit(t_full);
        mbar_arrive(ev_bar);
        ++ev;
        pending_g = -1;
      };
      for (int g = 0; g < ngroups && ok; ++g) {
        const int b = g & 1;  // slice buffer
        if (!mbar_wait_or_abort(slf0 + 8 * b, (g >> 1) & 1, abort_flag, lim)) {
          ok = false;
          break;
        }
        const bool merge = evt[g % 3] != 0;
        if (!merge) {
          if (pending_g >= 0) close_event();
          if (!mbar_wait_or_abort(t_empty, (ev & 1) ^ 1, abort_flag, lim)) {  // previous event read back
            ok = false;
            break;
          }
          pending_g = g;
        }
        fence_after_sync();
        uint64_t d = b ? dB : dA;
        asm volatile("" : "+l"(d));
        gram_issue_tile(tmem, d, !merge);
        last_g = g;
        umma_commit(sle0 + 8 * b);
      }
      if (ok && pending_g >= 0) close_event();
      if (ok && mbar_wait_or_abort(t_empty, (ev & 1) ^ 1, abort_flag, lim)) {
        evt[8 + (ev & 3)] = -1;  // no more events
        mbar_arrive(ev_bar);
      } else if (!*abort_flag) {
        *abort_flag = 1;
        status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
      }
      umma_commit(drain);
      mbar_wait(drain, 0);
    }
    __syncwarp();
  } else if (warp < 4) {
    // ------------------------------------------------------------------ scales and slices
    const int j = 16 * warp + (lane & 15), h = lane >> 4;
    const bool cj = j < n;
    int ev_len = 0, n_scale_syncs = 0;  // the same in every slicer thread
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1, q = 2 * b + h;  // slice buffer, this lane's staged sub-tile
      bool ok = true;
      for (int qq = 0; qq < 2 && ok; ++qq) ok = mbar_wait_or_abort(full0 + 8 * (2 * b + qq), (g >> 1) & 1, abort_flag, lim);
      if (!ok) {
        if (lane == 0 && !*abort_flag) {
          *abort_flag = 1;
          status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
        }
        break;
      }
      // Scales.  The first group of an event takes its column maxima (a first pass over the staged
      // rows) plus one bit of headroom; a later group is cut with the event's scales straight
      // away and keeps them unless one of its values reached 2^E, in which case it is cut
      // again with its own maxima and starts a new event (up to GS_EV_GROUPS groups per event).
      const int cnt = sub_rows(g, h);
      const uint8_t *src = stage + (size_t)q * GS_STAGE + 8 * j;
      const bool spec = g > 0 && ev_len < GS_EV_GROUPS;
      int E;
      if (spec) {
        E = colE[((g - 1) & 3) * GS_NP + j];
      } else {
        int mx = 0;
#pragma unroll 8
        for (int r = 0; r < GS_SUB; ++r) {
          const unsigned long long bits = (cj && r < cnt) ? *(const unsigned long long *)(src + r * 512) : 0ULL;
          mx = max(mx, g_expfield<IN_DF>(bits));
        }
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
        E = scale_exp(mx) + 1;
      }
      if (!mbar_wait_or_abort(sle0 + 8 * b, ((g >> 1) & 1) ^ 1, abort_flag, lim)) {
        ok = false;
      } else {
        uint8_t *buf = slices + (size_t)b * GS_BUF + (size_t)(j >> 3) * 1024 + (j & 7) * 16;
        bool merge = false;
        for (int attempt = 0; attempt < 2; ++attempt) {
          // pass 2: the group's 64 rows into slice buffer b (and this lane's largest exponent)
          int mxe = 0;
#pragma unroll 1
          for (int r0 = 0; r0 < GS_SUB; r0 += 8) {
            uint32_t w[4][NDIG];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int ra = r0 + 2 * u, rb = ra + 1;
              const unsigned long long ba = (cj && ra < cnt) ? *(const unsigned long long *)(src + ra * 512) : 0ULL;
              const unsigned long long bb = (cj && rb < cnt) ? *(const unsigned long long *)(src + rb * 512) : 0ULL;
              mxe = max(mxe, max(g_expfield<IN_DF>(ba), g_expfield<IN_DF>(bb)));
              if (IN_DF)
                digits2(g_fix<IN_DF>(ba, E), g_fix<IN_DF>(bb, E), w[u]);
              else
                digits2_biased(fix54_biased<DIG_BIAS>(ba, E), fix54_biased<DIG_BIAS>(bb, E), w[u]);
            }
            const int kg = (GS_SUB * h + r0) >> 3;  // K-group of rows r0 .. r0 + 7 within the tile
#pragma unroll
            for (int p = 0; p < NDIG; ++p)
              *(uint4 *)(buf + (size_t)(NDIG - 1 - p) * GS_SLICE + kg * 128) = make_uint4(w[0][p], w[1][p], w[2][p], w[3][p]);
          }
          if (!spec || attempt == 1) break;
          // did any value of the group reach the event's scale?  (the four slicer warps meet)
          const bool over = __any_sync(0xffffffffu, cj && mxe >= E + 1023);
          if (lane == 0 && over) atomicMax((int *)&evt[3 + g % 3], g + 1);
          __syncwarp();
          if (lane == 0) mbar_arrive(scale_bar);
          if (!mbar_wait_or_abort(scale_bar, (uint32_t)(n_scale_syncs & 1), abort_flag, lim)) {
            ok = false;
            break;
          }
          ++n_scale_syncs;
          merge = evt[3 + g % 3] != g + 1;
          if (merge) break;
          mxe = max(mxe, __shfl_xor_sync(0xffffffffu, mxe, 16));
          E = scale_exp(mxe) + 1;  // cut again with the group's own scales
        }
        if (ok) {
          ev_len = merge ? ev_len + 1 : 1;
          // four scale slots: an event's read-back uses the slot of its last group, and the
          // slicers cannot get further than three groups past that group before it is done
          if (h == 0) colE[(g & 3) * GS_NP + j] = E;
          if (warp == 0 && lane == 0) evt[g % 3] = merge;  // g continues the event of g - 1
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(empty0 + 8 * (2 * b));
            mbar_arrive(empty0 + 8 * (2 * b + 1));
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(slf0 + 8 * b);
        }
      }
      if (!ok) {
        if (lane == 0 && !*abort_flag) {
          *abort_flag = 1;
          status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
        }
        break;
      }
    }
  } else {
    // ------------------------------------------------------------------ recombination and sums
    const int quad = warp & 3, kh = (warp - 4) >> 2;
    const int L = 32 * quad + lane, par = L >> 6, j = L & 63;
    const int jlo = 32 * (quad & 1);  // smallest j of this warp
    const uint32_t tq = tmem + ((uint32_t)(32 * quad) << 16);
    double S[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) S[c] = 0.0;
    const bool active = 32 * kh + 31 >= jlo;  // some k >= j in this warp's block
    for (int ev = 0;; ++ev) {
      if (!mbar_wait_or_abort(ev_bar, ev & 1, abort_flag, lim)) {
        if (lane == 0 && !*abort_flag) {
          *abort_flag = 1;
          status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
        }
        break;
      }
      const int g = evt[8 + (ev & 3)];
      if (g < 0) break;
      if (!mbar_wait_or_abort(t_full, ev & 1, abort_flag, lim)) {
        if (lane == 0 && !*abort_flag) {
          *abort_flag = 1;
          status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
        }
        break;
      }
      fence_after_sync();
      if (active) {
        const int *ce = colE + (g & 3) * GS_NP;
        const int ebase = ce[j] - 51 - 7 * par;
#pragma unroll
        for (int h4 = 0; h4 < 8; ++h4) {
          const int k0 = 32 * kh + 4 * h4;
          if (k0 + 3 < jlo) continue;  // the whole 4-column group lies below this warp's diagonal
          uint32_t v[NDIG][4];
#pragma unroll
          for (int gg = 0; gg < NDIG; ++gg) tmem_ld4(tq + (uint32_t)(gg * 64 + k0), v[gg]);
          tmem_wait_ld();
          tmem_regs_ready(v);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const long long t = recombine_g7w(v[0][c], v[1][c], v[2][c], v[3][c], v[4][c], v[5][c], v[6][c], v[7][c]);
            const double y = int_times_pow2_cvt(t, ebase + ce[k0 + c]);  // T / 256 (|T| < 2^71)
            S[4 * h4 + c] += y;
          }
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(t_empty);
    }
    if (active && j < n) {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int k = 32 * kh + c;
        if (k >= j && k < n) atomicAdd(&Gp[tri_idx(j, k)], S[c]);
      }
    }
  }

  __syncthreads();
  fence_after_sync();
  if (warp == GW_MMA) tmem_free(tmem, GS_TMEM_COLS);
}

bool gram_split_supported(int64_t n) { return n >= 1 && n <= GS_NP; }

cudaError_t launch_gram_split(const void *W, bool in_df, int64_t ldw, int64_t m, int64_t n, double *Gpacked,
                              int num_sms, DevStatus *st, cudaStream_t s) {
  int64_t ctas = std::min<int64_t>(ceil_div(m, GS_GROUP), (int64_t)num_sms);
  const int64_t rows_per_cta = ceil_div(ceil_div(m, ctas), GS_GROUP) * GS_GROUP;
  ctas = ceil_div(m, rows_per_cta);
  const bool aligned = ((uintptr_t)W & 15) == 0;
  const int load_mode = (aligned && n == GS_NP && ldw == GS_NP) ? GLOAD_BLOCK
                        : (aligned && (n * 8) % 16 == 0 && (ldw * 8) % 16 == 0) ? GLOAD_ROWS
                                                                                 : GLOAD_PLAIN;
  cudaError_t e;
  if (in_df) {
    e = cudaFuncSetAttribute(k_gram_split<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GS_SMEM);
    if (e != cudaSuccess) return e;
    k_gram_split<true><<<(unsigned)ctas, GS_THREADS, GS_SMEM, s>>>(W, ldw, m, (int)n, Gpacked, rows_per_cta,
                                                                   load_mode, st);
  } else {
    e = cudaFuncSetAttribute(k_gram_split<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GS_SMEM);
    if (e != cudaSuccess) return e;
    k_gram_split<false><<<(unsigned)ctas, GS_THREADS, GS_SMEM, s>>>(W, ldw, m, (int)n, Gpacked, rows_per_cta,
                                                                    load_mode, st);
  }
  return cudaGetLastError();
}

}  // namespace rq
