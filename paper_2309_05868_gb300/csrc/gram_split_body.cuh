// gram_split_body.cuh -- the CTA body of G = W^T W (Algorithm 2 step 1, the Gram of each Cholesky pass) for n <= 64
// from exact split products on the tensor cores.
//
// Rows are taken in groups (64 64 / NP rows for the instance of width NP, below).  Column j of a
// group gets a scale 2^E_j > max_r |w_rj| and
// w_rj = 2^(E_j - 54) X_rj up to truncation, with X_rj = trunc(w_rj 2^(54 - E_j)) written in
// eight balanced 7-bit digits d_p (tc.cuh; slice s = 7 - p).  The kernel comes in three widths
// NP = 64, 32, 16 (n padded to NP): a slice holds NP columns, and SPA = 128 / NP consecutive
// slices stack into the 128 rows of an A-tile (TMEM lane L <-> slice SPA a + L / NP, column
// L % NP).  Slices t of the same buffer are the B operand, up to 256 / NP of them stacked along
// N per MMA.  A-tile a times slice t lands in region c = SPA a + t (NP tensor-memory columns),
// so region c of lane L gathers the pairs (s, t) with s + t = c + L / NP: lanes with p = L / NP
// hold D_g for g = c + p.  A-tile a needs the slices t <= 7 - SPA a; per K-step of 16 rows
// NP = 64 issues 6 MMAs (N from 128 to 256), NP = 32 two, NP = 16 one.  A group of 64 64 / NP
// rows (64, 128, 256) keeps the work per group, 4096 values and 64 KB of slices, the same.
//
// Groups form events: the first group of an event takes its column maxima plus one bit of
// headroom as scales, and the following groups keep those scales unless one of their columns
// outgrew them, up to 1024 rows.  An event's groups accumulate in the same regions, so every D
// is a sum of at most 4 x 1024 digit products of at most 2^12, |D| <= 2^24,
// exact in FP32 (NP = 32: two pairs per region, NP = 16: one).  With
//   T_p(j, k) = sum_c 2^(7 (7 - c)) D_c(SPA-row p, j, k),
// the event's contribution is 2^(E_j + E_k - 59 - 7p) T_p; pairs with g >= 9 (and half of g = 8)
// are dropped, below 2^-54 of 2^(E_j + E_k) per row.  T_p / 256 is formed in 64-bit integers
// (tc::recombine_g7w), converted on the FP64 pipe and added to per-thread FP64 sums; one FP64
// atomic per entry (j <= k) and lane row p at the end.  Longer events mean fewer read-backs, and
// the next event's products wait for a read-back to finish (tensor memory holds one event).
//
// One CTA per SM, persistent over its row range; warps specialise:
//   warps 0 .. GS_NSW - 1 find each group's column scales (first pass over the staged rows) and
//     cut the group into digit slices (second pass; two slice buffers, alternating groups); a
//     warp owns NP / GS_NSW columns, and the lanes of one column split the group's rows,
//   the next 8 warps read the regions back (warp w: TMEM lanes 32 (w & 3) .., one half of the
//     NP columns k) and keep the FP64 sums,
//   the next warp loads 32-row sub-tiles into a ring with bulk copies (two groups in flight, so
//     a group's rows arrive while the previous one is cut),
//   the last warp owns tensor memory and issues the MMAs, closing an event (commit to the
//     recombination warps) when the next group starts a new one.
#pragma once
#include "common.cuh"
#include "tc.cuh"

namespace rq {

namespace {
using namespace tc;

constexpr int GS_SUB = 32;
// Rows per tensor-memory accumulation: 1024 keep every region within 4 x 1024 digit products of
// at most 2^12, |D| <= 2^24, exact in FP32.
constexpr int GS_EV_ROWS = 1024;
constexpr int GS_NSW = 4;                       // slicer warps (0 .. GS_NSW - 1)
constexpr int GW_READ0 = GS_NSW;                 // 8 recombination warps (a multiple of 4 first)
constexpr int GW_LOAD = GS_NSW + 8, GW_MMA = GS_NSW + 9;
constexpr int GS_THREADS = 32 * (GS_NSW + 10);
constexpr int GS_NBARS_MAX = 2 * 16 + 9;  // full[NQ], empty[NQ], sl_full[2], sl_empty[2], t_full,
                                          // t_empty, drain, scale_bar, ev_bar

// Shared-memory plan of the width-NP instance.  A group has 64 * 64 / NP rows, so that every
// instance cuts 4096 values per group (32 rows per slicer lane) into 64 KB of slices.
template <int NP>
struct GsCfg {
  static constexpr int GROUP = 64 * 64 / NP;           // rows per group (K of its products)
  static constexpr int KSTEPS = GROUP / 16;            // MMA K-steps per group
  static constexpr int EV_GROUPS = GS_EV_ROWS / GROUP; // groups per event at most
  static constexpr int SPA = 128 / NP;                 // slices per A-tile
  static constexpr int SPB = 256 / NP;                 // slices per MMA's B (N <= 256)
  static constexpr int NAT = 8 / SPA;                  // A-tiles
  static constexpr int NSUB = GROUP / GS_SUB;          // staged 32-row sub-tiles per group
  static constexpr int NQ = 2 * NSUB;                  // stage slots: two groups in flight
  static constexpr int CPW = NP / GS_NSW;              // columns per slicer warp
  static constexpr int RP = 32 / CPW;                  // lanes per column
  static constexpr int RPT = GROUP / RP;               // rows of a group per slicer lane
  static constexpr uint32_t SBO = GROUP * 16;          // 8-column core-matrix groups
  static constexpr uint32_t SLICE = NP * GROUP * 2;    // one slice of one group (f16 digits)
  static constexpr uint32_t BUF = NDIG * SLICE;
  static constexpr uint32_t PITCH = NP * 8;            // staged row
  static constexpr uint32_t STAGE = GS_SUB * PITCH;    // one 32-row sub-tile
  static constexpr uint32_t TMEM_COLS = 8 * NP;
  static constexpr size_t OFF_SL = 0;
  static constexpr size_t OFF_STAGE = OFF_SL + 2 * (size_t)BUF;
  static constexpr size_t OFF_COLE = OFF_STAGE + (size_t)NQ * STAGE;
  static constexpr size_t OFF_EVT = OFF_COLE + 4 * NP * sizeof(int);  // merge[3], grow[3], ev_grp[4]
  static constexpr size_t OFF_BARS = OFF_EVT + 16 * sizeof(int);
  static constexpr int NBARS = 2 * NQ + 9;
  static constexpr size_t OFF_MISC = OFF_BARS + NBARS * 8;
  static constexpr size_t SMEM = OFF_MISC + 16;
  static_assert(SMEM <= 232448, "shared memory budget");
  static_assert(RPT % 8 == 0 && GS_SUB % RPT == 0, "a slicer lane cuts whole K-groups of one sub-tile");
  static_assert(NBARS <= GS_NBARS_MAX, "barrier count");
};

// GLOAD_BLOCK: one bulk copy per sub-tile (contiguous rows of NP values); GLOAD_ROWS: one bulk
// copy per row; GLOAD_PLAIN: element loads; GLOAD_ASYNC16: 16-byte asynchronous copies, one row
// per warp instruction (rows of exactly 64 values at a 16-byte aligned address), which read
// global memory as ordinary loads do -- for rows another CTA has just written.
enum GLoadMode { GLOAD_BLOCK = 0, GLOAD_ROWS = 1, GLOAD_PLAIN = 2, GLOAD_ASYNC16 = 3 };

// Producer progress published by the eight read-back warps of a paired solve CTA (trsm_tc.cu):
// word f of the producer's shared memory holds how many of its tiles (TQ_PRODUCER_ROWS rows each)
// warp f has stored.  PRODUCER_DONE releases every wait (the producer skipped or gave up).
constexpr int TQ_PRODUCER_ROWS = 128, PRODUCER_WARPS = 8;
constexpr uint32_t PRODUCER_DONE = 0x7fffffffu;

// Waits until every producer warp has stored `need` tiles (words at the cluster address
// `producer`); `seen` keeps the smallest count seen at the last successful poll, so that most
// calls return without touching the producer.  The eight words are read together (relaxed) and
// one acquire fence follows a poll that found them high enough.  Bounded: false after `limit`
// polls, on the local abort flag, or once the status word reports a failure.
__device__ __forceinline__ bool wait_producer(uint32_t producer, uint32_t need, uint32_t &seen, int limit,
                                              volatile int *abort, const DevStatus *st) {
  if (seen >= need) return true;
  for (int it = 0;; ++it) {
    uint32_t mn = 0xffffffffu;
#pragma unroll
    for (int f = 0; f < PRODUCER_WARPS; ++f) mn = min(mn, ld_relaxed_cluster_u32(producer + 4u * (uint32_t)f));
    if (mn >= need) {
      fence_acquire_cluster();
      seen = mn;
      return true;
    }
    if (it >= limit || *abort || ((it & 255) == 255 && status_failed(st))) return false;
    __nanosleep(64);
  }
}

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

// One group's MMAs (K = GROUP in steps of 16): A-tile a (slices SPA a ..) times the slices
// t = 0 .. 7 - SPA a, SPB of them stacked per MMA, into regions SPA a + t.  The first A-tile's
// products at K-step 0 of an event's first group open every region.
template <int NP>
__device__ __forceinline__ void gram_issue_tile(uint32_t tmem, uint64_t d0, bool first) {
  using C = GsCfg<NP>;
#pragma unroll
  for (int c = 0; c < C::KSTEPS; ++c) {
    const uint64_t kc = (uint64_t)(256 * c) >> 4;
#pragma unroll
    for (int a = 0; a < C::NAT; ++a) {
      const int tmax = 8 - C::SPA * a;  // slices t = 0 .. tmax - 1
#pragma unroll
      for (int t0 = 0; t0 < tmax; t0 += C::SPB) {
        const int nt = (tmax - t0) < C::SPB ? (tmax - t0) : C::SPB;
        umma_bf16(tmem + (uint32_t)((C::SPA * a + t0) * NP),
                  d0 + kc + (((uint64_t)(C::SPA * a) * C::SLICE) >> 4),
                  d0 + kc + (((uint64_t)t0 * C::SLICE) >> 4), umma_idesc_f16(128, NP * nt),
                  (first && c == 0 && a == 0) ? 0u : 1u);
      }
    }
  }
}


template <int NP, bool IN_DF, bool WAIT>
__device__ __forceinline__ void gram_split_cta(const void *Win, int64_t ldw, int64_t m, int n, double *Gp,
                                               int64_t rows_per_cta, int load_mode, DevStatus *st, int cta,
                                               uint32_t producer) {
  using C = GsCfg<NP>;
  const int lim = wait_bound(st, MAX_WAIT);
  extern __shared__ __align__(1024) uint8_t gs_smem[];
  uint8_t *slices = gs_smem + C::OFF_SL;
  uint8_t *stage = gs_smem + C::OFF_STAGE;
  int *colE = (int *)(gs_smem + C::OFF_COLE);
  volatile int *evt = (volatile int *)(gs_smem + C::OFF_EVT);
  uint64_t *bars = (uint64_t *)(gs_smem + C::OFF_BARS);
  uint32_t *tmem_slot = (uint32_t *)(gs_smem + C::OFF_MISC);
  volatile int *abort_flag = (volatile int *)(gs_smem + C::OFF_MISC + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full0 = smem_addr(&bars[0]), empty0 = smem_addr(&bars[C::NQ]);
  const uint32_t slf0 = smem_addr(&bars[2 * C::NQ]), sle0 = smem_addr(&bars[2 * C::NQ + 2]);
  const uint32_t t_full = smem_addr(&bars[2 * C::NQ + 4]), t_empty = smem_addr(&bars[2 * C::NQ + 5]);
  const uint32_t drain = smem_addr(&bars[2 * C::NQ + 6]);
  const uint32_t scale_bar = smem_addr(&bars[2 * C::NQ + 7]), ev_bar = smem_addr(&bars[2 * C::NQ + 8]);
  auto fail = [&]() {
    if (!*abort_flag) {
      *abort_flag = 1;
      status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
    }
  };

  if (tid == 0) {
    for (int q = 0; q < C::NQ; ++q) {
      mbar_init_count(full0 + 8 * q, load_mode == GLOAD_ASYNC16 ? 32 : 1);
      mbar_init_count(empty0 + 8 * q, GS_NSW);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init_count(slf0 + 8 * b, GS_NSW);
      mbar_init_count(sle0 + 8 * b, 1);
    }
    mbar_init_count(t_full, 1);
    mbar_init_count(t_empty, 8);
    mbar_init_count(drain, 1);
    mbar_init_count(scale_bar, GS_NSW);
    mbar_init_count(ev_bar, 1);
    *abort_flag = 0;
    for (int e = 0; e < 16; ++e) evt[e] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == GW_MMA) tmem_alloc(tmem_slot, C::TMEM_COLS);
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int64_t r_begin = (int64_t)cta * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  const int ngroups = r_end > r_begin ? (int)((r_end - r_begin + C::GROUP - 1) / C::GROUP) : 0;
  auto sub_rows = [&](int g, int q) -> int {
    const int64_t r0 = r_begin + (int64_t)g * C::GROUP + GS_SUB * q;
    return r0 < r_end ? (int)imin64(GS_SUB, r_end - r0) : 0;
  };

  if (warp == GW_LOAD) {
    // ------------------------------------------------------------------ loader
    // group g uses slots NSUB (g & 1) .. NSUB (g & 1) + NSUB - 1, on their (g >> 1)-th use
    int last_use[C::NQ];
#pragma unroll
    for (int q = 0; q < C::NQ; ++q) last_use[q] = -1;
    uint32_t seen = 0;  // WAIT: producer tiles known to be stored
    for (int g = 0; g < ngroups && !*abort_flag; ++g) {
      bool ok = true;
      const int use = g >> 1;
      if (WAIT) {
        // every row of the group stored by the producer (the tiles that hold them)
        const int64_t rows_in = imin64((int64_t)(g + 1) * C::GROUP, r_end - r_begin);
        const uint32_t need = (uint32_t)((rows_in + TQ_PRODUCER_ROWS - 1) / TQ_PRODUCER_ROWS);
        int got = 1;
        if (lane == 0) got = wait_producer(producer, need, seen, lim, abort_flag, st);
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();  // the other lanes' copies are ordered after lane 0's acquire
        if (!got) {
          if (lane == 0) fail();
          break;
        }
      }
      for (int qq = 0; qq < C::NSUB; ++qq) {
        const int q = C::NSUB * (g & 1) + qq;
        if (!mbar_wait_or_abort(empty0 + 8 * q, (uint32_t)((use & 1) ^ 1), abort_flag, lim)) {
          if (lane == 0) fail();
          ok = false;
          break;
        }
        const int64_t r0 = r_begin + (int64_t)g * C::GROUP + GS_SUB * qq;
        const int cnt = sub_rows(g, qq);
        uint8_t *dst = stage + (size_t)q * C::STAGE;
        const uint32_t fb = full0 + 8 * q;
        if (NP == 64 && load_mode == GLOAD_ASYNC16) {
          // lane = 16-byte chunk of a 512-byte row; every lane arrives once its copies have landed
          for (int r = 0; r < cnt; ++r)
            cp_async16(smem_addr(dst + r * C::PITCH + 16 * lane), (const double *)Win + (r0 + r) * ldw + 2 * lane);
          cp_async_arrive(fb);
        } else if (cnt > 0 && load_mode == GLOAD_BLOCK) {
          if (lane == 0) {
            mbar_expect_tx(fb, (uint32_t)cnt * C::PITCH);
            bulk_load(smem_addr(dst), (const uint8_t *)Win + (size_t)r0 * C::PITCH, (uint32_t)cnt * C::PITCH, fb);
          }
        } else if (cnt > 0 && load_mode == GLOAD_ROWS) {
          if (lane == 0) mbar_expect_tx(fb, (uint32_t)cnt * (uint32_t)n * 8u);
          __syncwarp();
          for (int r = lane; r < cnt; r += 32)
            bulk_load(smem_addr(dst + r * C::PITCH), (const uint8_t *)Win + (size_t)(r0 + r) * (size_t)ldw * 8,
                      (uint32_t)n * 8u, fb);
        } else {
          const unsigned long long *src = (const unsigned long long *)Win;
          for (int e = lane; e < cnt * n; e += 32) {
            const int r = e / n, cc = e - r * n;
            ((unsigned long long *)dst)[r * NP + cc] = src[(r0 + r) * ldw + cc];
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(fb);
        }
        last_use[q] = use;
      }
      if (!ok) break;
    }
    if (lane == 0)
      for (int q = 0; q < C::NQ; ++q)
        if (last_use[q] >= 0) mbar_wait(full0 + 8 * q, (uint32_t)(last_use[q] & 1));
  } else if (warp == GW_MMA) {
    // ------------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint64_t dA = umma_desc(smem_addr(slices), 128, C::SBO);
      const uint64_t dB = umma_desc(smem_addr(slices + C::BUF), 128, C::SBO);
      // Events: one tensor-memory accumulation = one group, or up to EV_GROUPS consecutive
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
        if (!mbar_wait_or_abort(slf0 + 8 * b, (uint32_t)((g >> 1) & 1), abort_flag, lim)) {
          ok = false;
          break;
        }
        const bool merge = evt[g % 3] != 0;
        if (!merge) {
          if (pending_g >= 0) close_event();
          if (!mbar_wait_or_abort(t_empty, (uint32_t)((ev & 1) ^ 1), abort_flag, lim)) {  // previous event read back
            ok = false;
            break;
          }
          pending_g = g;
        }
        fence_after_sync();
        uint64_t d = b ? dB : dA;
        asm volatile("" : "+l"(d));
        gram_issue_tile<NP>(tmem, d, !merge);
        last_g = g;
        umma_commit(sle0 + 8 * b);
      }
      if (ok && pending_g >= 0) close_event();
      if (ok && mbar_wait_or_abort(t_empty, (uint32_t)((ev & 1) ^ 1), abort_flag, lim)) {
        evt[8 + (ev & 3)] = -1;  // no more events
        mbar_arrive(ev_bar);
      } else {
        fail();
      }
      umma_commit(drain);
      mbar_wait(drain, 0);
    }
    __syncwarp();
  } else if (warp < GS_NSW) {
    // ------------------------------------------------------------------ scales and slices
    // Lane: column j = CPW warp + (lane % CPW); the RPT rows from rp RPT (rp = lane / CPW) of
    // the group, inside sub-tile hq.
    const int j = C::CPW * warp + (lane % C::CPW), rp = lane / C::CPW;
    const int row0 = rp * C::RPT, hq = row0 / GS_SUB, rin = row0 % GS_SUB;
    const bool cj = j < n;
    int ev_len = 0, n_scale_syncs = 0;  // the same in every slicer thread
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1, use = g >> 1;
      const int q = C::NSUB * b + hq;  // this lane's staged sub-tile
      bool ok = true;
      for (int qq = 0; qq < C::NSUB && ok; ++qq)
        ok = mbar_wait_or_abort(full0 + 8 * (C::NSUB * b + qq), (uint32_t)(use & 1), abort_flag, lim);
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      // Scales.  The first group of an event takes its column maxima (a first pass over the staged
      // rows) plus one bit of headroom; a later group is cut with the event's scales straight
      // away and keeps them unless one of its values reached 2^E, in which case it is cut
      // again with its own maxima and starts a new event (up to EV_GROUPS groups per event).
      const int cnt = sub_rows(g, hq) - rin;  // rows of this lane's range that exist
      const uint8_t *src = stage + (size_t)q * C::STAGE + (size_t)rin * C::PITCH + 8 * j;
      const bool spec = g > 0 && ev_len < C::EV_GROUPS;
      int E;
      if (spec) {
        E = colE[((g - 1) & 3) * NP + j];
      } else {
        int mx = 0;
#pragma unroll 8
        for (int r = 0; r < C::RPT; ++r) {
          const unsigned long long bits = (cj && r < cnt) ? *(const unsigned long long *)(src + r * C::PITCH) : 0ULL;
          mx = max(mx, g_expfield<IN_DF>(bits));
        }
#pragma unroll
        for (int o = C::CPW; o < 32; o <<= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        E = scale_exp(mx) + 1;
      }
      if (!mbar_wait_or_abort(sle0 + 8 * b, (uint32_t)(((g >> 1) & 1) ^ 1), abort_flag, lim)) {
        ok = false;
      } else {
        uint8_t *buf = slices + (size_t)b * C::BUF + (size_t)(j >> 3) * C::SBO + (j & 7) * 16;
        bool merge = false;
        for (int attempt = 0; attempt < 2; ++attempt) {
          // pass 2: this lane's rows into slice buffer b (and its largest exponent)
          int mxe = 0;
#pragma unroll (NP == 64 ? 2 : 1)  // NP = 64: two 8-row K-groups per iteration (2.053 -> 2.028 ms at m = 2^23)
          for (int r0 = 0; r0 < C::RPT; r0 += 8) {
            uint32_t w[4][NDIG];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int ra = r0 + 2 * u, rb = ra + 1;
              const unsigned long long ba = (cj && ra < cnt) ? *(const unsigned long long *)(src + ra * C::PITCH) : 0ULL;
              const unsigned long long bb = (cj && rb < cnt) ? *(const unsigned long long *)(src + rb * C::PITCH) : 0ULL;
              mxe = max(mxe, max(g_expfield<IN_DF>(ba), g_expfield<IN_DF>(bb)));
              if (IN_DF)
                digits2(g_fix<IN_DF>(ba, E), g_fix<IN_DF>(bb, E), w[u]);
              else
                digits2_biased(fix54_biased<DIG_BIAS>(ba, E), fix54_biased<DIG_BIAS>(bb, E), w[u]);
            }
            const int kg = (row0 + r0) >> 3;  // K-group of rows row0 + r0 .. + 7 within the group
#pragma unroll
            for (int p = 0; p < NDIG; ++p)
              *(uint4 *)(buf + (size_t)(NDIG - 1 - p) * C::SLICE + kg * 128) = make_uint4(w[0][p], w[1][p], w[2][p], w[3][p]);
          }
          if (!spec || attempt == 1) break;
          // did any value of the group reach the event's scale?  (the slicer warps meet)
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
#pragma unroll
          for (int o = C::CPW; o < 32; o <<= 1) mxe = max(mxe, __shfl_xor_sync(0xffffffffu, mxe, o));
          E = scale_exp(mxe) + 1;  // cut again with the group's own scales
        }
        if (ok) {
          ev_len = merge ? ev_len + 1 : 1;
          // four scale slots: an event's read-back uses the slot of its last group, and the
          // slicers cannot get further than three groups past that group before it is done
          if (rp == 0) colE[(g & 3) * NP + j] = E;
          if (warp == 0 && lane == 0) evt[g % 3] = merge;  // g continues the event of g - 1
          __syncwarp();
          if (lane == 0)
            for (int qq = 0; qq < C::NSUB; ++qq) mbar_arrive(empty0 + 8 * (C::NSUB * b + qq));
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(slf0 + 8 * b);
        }
      }
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
    }
  } else if (warp < GW_READ0 + 8) {  // (warps past the kernel's own idle in a paired launch)
    // ------------------------------------------------------------------ recombination and sums
    // Warp: TMEM lanes 32 quad .. 32 quad + 31 (lane L: slice row p = L / NP of the A-tiles,
    // column j = L % NP), columns k in [KH kh, KH kh + KH).
    constexpr int KH = NP / 2;
    const int quad = warp & 3, kh = (warp - GW_READ0) >> 2;
    const int L = 32 * quad + lane, par = L / NP, j = L % NP;
    const int jlo = (32 * quad) % NP;  // smallest j of this warp
    const uint32_t tq = tmem + ((uint32_t)(32 * quad) << 16);
    double S[KH];
#pragma unroll
    for (int c = 0; c < KH; ++c) S[c] = 0.0;
    const bool active = KH * kh + KH - 1 >= jlo;  // some k >= j in this warp's block
    for (int ev = 0;; ++ev) {
      if (!mbar_wait_or_abort(ev_bar, (uint32_t)(ev & 1), abort_flag, lim)) {
        if (lane == 0) fail();
        break;
      }
      const int g = evt[8 + (ev & 3)];
      if (g < 0) break;
      if (!mbar_wait_or_abort(t_full, (uint32_t)(ev & 1), abort_flag, lim)) {
        if (lane == 0) fail();
        break;
      }
      fence_after_sync();
      if (active) {
        const int *ce = colE + (g & 3) * NP;
        const int ebase = ce[j] - 51 - 7 * par;
#pragma unroll
        for (int h4 = 0; h4 < KH / 4; ++h4) {
          const int k0 = KH * kh + 4 * h4;
          if (k0 + 3 < jlo) continue;  // the whole 4-column group lies below this warp's diagonal
          uint32_t v[NDIG][4];
#pragma unroll
          for (int gg = 0; gg < NDIG; ++gg) tmem_ld4(tq + (uint32_t)(gg * NP + k0), v[gg]);
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
      for (int c = 0; c < KH; ++c) {
        const int k = KH * kh + c;
        if (k >= j && k < n) atomicAdd(&Gp[tri_idx(j, k)], S[c]);
      }
    }
  }

  __syncthreads();
  fence_after_sync();
  if (warp == GW_MMA) tmem_free(tmem, C::TMEM_COLS);
}

}  // namespace
}  // namespace rq
