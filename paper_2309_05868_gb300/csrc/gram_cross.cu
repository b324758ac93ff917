// gram_cross.cu -- the last n - 64 columns of G = W^T W (Algorithm 2 step 1) for 64 < n <= 128,
// from exact split products on the tensor cores: G[:, 64:n] = W^T W[:, 64:n], all n rows at once.
// Together with the Gram of W's first 64 columns (gram_split.cu) that is the whole upper
// triangle of G.
//
// Number format as in gram_split.cu: per 32-row group, column J of W gets a scale 2^E_J and
// eight balanced 7-bit digits (slice s = 0 the leading one).  Here an A operand is ONE slice of
// all 128 (padded) columns -- M = 128, TMEM lane i <-> column J(i) -- and B is slices t of the
// block of columns 64 .. 127 stacked along N, so region g = s + t (64 tensor-memory columns)
// gathers every pair (s, t) with s + t = g, g = 0 .. 7, in all 128 lanes, and
//   sum_rows w_J w_{64 + k} = 2^(E_J + E_{64+k} - 51) T / 256,  T = sum_g 2^(7 (7 - g)) D_g(J, k).
// A region holds up to eight digit-pair sums of at most 2^12 each per row, so an event (groups
// accumulated before one read-back) spans at most 512 rows: |D| <= 2^24, exact in FP32.
//
// Slice layout (K-major core matrices of 8 columns x 8 rows, no swizzle): slice s at 8 KB s, and
// within it the 8-column group c of column block b at 512 B (2 c + b).  So one slice's 16
// row-groups are 512 B apart (A: M = 128, lane i <-> column 64 ((i >> 3) & 1) + 8 (i >> 4) + (i & 7)),
// and block 1's groups are 1 KB apart through consecutive slices (B: N = 64 per slice, stacked).
//
// One CTA per SM, persistent over its rows; warps: 0-3 cut each 32-row group (two columns and
// 16 rows per lane), 4-11 read the regions back and keep FP64 sums, 12 loads the groups' rows
// (two groups in flight), 13 owns tensor memory and issues the MMAs.  Two slice buffers of
// 64 KB: a group is cut while the previous group's products run.
#include "common.cuh"
#include "tc.cuh"

namespace rq {

namespace {
using namespace tc;

constexpr int GC_SUB = 32, GC_COLS = 128, GC_GROUP = 32;
constexpr int GC_EV_GROUPS = 512 / GC_GROUP;  // 512 rows per event
constexpr int GC_THREADS = 448;
constexpr int GCW_LOAD = 12, GCW_MMA = 13;
constexpr uint32_t GC_TMEM_COLS = 512;
constexpr uint32_t GC_SBO = GC_GROUP * 16;       // 8-column core-matrix groups: 512 B
constexpr uint32_t GC_SLICE = 16 * GC_SBO;       // 128 columns x 32 rows of f16 digits: 8 KB
constexpr uint32_t GC_BUF = NDIG * GC_SLICE;     // 64 KB
constexpr uint32_t GC_ROW = GC_COLS * 8;         // staged row: 1 KB
constexpr uint32_t GC_STAGE = GC_SUB * GC_ROW;   // 32 KB sub-tile
constexpr size_t COFF_SL = 0;
constexpr size_t COFF_STAGE = COFF_SL + 2 * (size_t)GC_BUF;
constexpr size_t COFF_COLE = COFF_STAGE + 2 * (size_t)GC_STAGE;
constexpr size_t COFF_EVT = COFF_COLE + 4 * GC_COLS * sizeof(int);
constexpr size_t COFF_BARS = COFF_EVT + 16 * sizeof(int);
// full[2], empty[2], sl_full[2], sl_empty[2], t_full, t_empty, drain, scale, ev
constexpr int GC_NBARS = 13;
constexpr size_t COFF_MISC = COFF_BARS + GC_NBARS * 8;
constexpr size_t GC_SMEM = COFF_MISC + 16;
static_assert(GC_SMEM <= 232448, "shared memory budget");

enum GcLoad { GC_LOAD_BLOCK = 0, GC_LOAD_ROWS = 1, GC_LOAD_PLAIN = 2 };

// Byte offset, within a slice, of column J's core-matrix row (K-group 0).
__device__ __forceinline__ uint32_t gc_col_off(int J) {
  return (uint32_t)(2 * ((J & 63) >> 3) + (J >> 6)) * GC_SBO + (uint32_t)(J & 7) * 16u;
}

// One 32-row group's products (K = 32 in two steps): A slice s (all columns) times B slices t
// of block 1 stacked along N (at most four per MMA), into regions s + t.  The two slice-0
// products of an event's first group open all eight regions.
__device__ __forceinline__ void gc_issue_group(uint32_t tmem, uint64_t dA, uint64_t dB, bool first) {
#pragma unroll
  for (int c = 0; c < GC_GROUP / 16; ++c) {
    const uint64_t kc = (uint64_t)(256 * c) >> 4;
#pragma unroll
    for (int s = 0; s < NDIG; ++s) {
#pragma unroll
      for (int t0 = 0; t0 < NDIG - s; t0 += 4) {
        const int nt = (NDIG - s - t0) < 4 ? (NDIG - s - t0) : 4;
        umma_bf16(tmem + (uint32_t)(64 * (s + t0)), dA + kc + (((uint64_t)s * GC_SLICE) >> 4),
                  dB + kc + (((uint64_t)t0 * GC_SLICE) >> 4), umma_idesc_f16(128, 64 * nt),
                  (first && c == 0 && s == 0) ? 0u : 1u);
      }
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(GC_THREADS, 1)
    k_gram_cross(const double *__restrict__ W, int64_t ldw, int64_t m, int n, double *Gp, int64_t rows_per_cta,
                 int load_mode, DevStatus *st) {
  if (status_failed(st)) return;
  const int lim = wait_bound(st, MAX_WAIT);
  extern __shared__ __align__(1024) uint8_t gc_smem[];
  uint8_t *slices = gc_smem + COFF_SL;
  uint8_t *stage = gc_smem + COFF_STAGE;
  int *colE = (int *)(gc_smem + COFF_COLE);
  volatile int *evt = (volatile int *)(gc_smem + COFF_EVT);
  uint64_t *bars = (uint64_t *)(gc_smem + COFF_BARS);
  uint32_t *tmem_slot = (uint32_t *)(gc_smem + COFF_MISC);
  volatile int *abort_flag = (volatile int *)(gc_smem + COFF_MISC + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full0 = smem_addr(&bars[0]), empty0 = smem_addr(&bars[2]);
  const uint32_t slf0 = smem_addr(&bars[4]), sle0 = smem_addr(&bars[6]);
  const uint32_t t_full = smem_addr(&bars[8]), t_empty = smem_addr(&bars[9]), drain = smem_addr(&bars[10]);
  const uint32_t scale_bar = smem_addr(&bars[11]), ev_bar = smem_addr(&bars[12]);
  auto fail = [&]() {
    if (!*abort_flag) {
      *abort_flag = 1;
      status_fail(st, RANDQR_ERR_TIMEOUT, 0, 0);
    }
  };

  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      mbar_init_count(full0 + 8 * q, 1);
      mbar_init_count(empty0 + 8 * q, 4);
      mbar_init_count(slf0 + 8 * q, 4);
      mbar_init_count(sle0 + 8 * q, 1);
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
  if (warp == GCW_MMA) tmem_alloc(tmem_slot, GC_TMEM_COLS);
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = imin64(m, r_begin + rows_per_cta);
  const int ngroups = r_end > r_begin ? (int)((r_end - r_begin + GC_GROUP - 1) / GC_GROUP) : 0;
  auto sub_rows = [&](int g, int q) -> int {
    const int64_t r0 = r_begin + (int64_t)g * GC_GROUP + GC_SUB * q;
    return r0 < r_end ? (int)imin64(GC_SUB, r_end - r0) : 0;
  };

  if (warp == GCW_LOAD) {
    // ------------------------------------------------------------------ loader
    // group g (one 32-row sub-tile) goes to slot g & 1, on the slot's (g >> 1)-th use
    int last_g[2] = {-1, -1};
    for (int g = 0; g < ngroups && !*abort_flag; ++g) {
      bool ok = true;
      {
        const int q = g & 1;
        if (!mbar_wait_or_abort(empty0 + 8 * q, (uint32_t)(((g >> 1) & 1) ^ 1), abort_flag, lim)) {
          if (lane == 0) fail();
          ok = false;
          break;
        }
        const int64_t r0 = r_begin + (int64_t)g * GC_GROUP;
        const int cnt = sub_rows(g, 0);
        uint8_t *dst = stage + (size_t)q * GC_STAGE;
        const uint32_t fb = full0 + 8 * q;
        if (cnt > 0 && load_mode == GC_LOAD_BLOCK) {
          if (lane == 0) {
            mbar_expect_tx(fb, (uint32_t)cnt * GC_ROW);
            bulk_load(smem_addr(dst), W + r0 * ldw, (uint32_t)cnt * GC_ROW, fb);
          }
        } else if (cnt > 0 && load_mode == GC_LOAD_ROWS) {
          if (lane == 0) mbar_expect_tx(fb, (uint32_t)cnt * (uint32_t)n * 8u);
          __syncwarp();
          if (lane < cnt) bulk_load(smem_addr(dst + (size_t)lane * GC_ROW), W + (r0 + lane) * ldw, (uint32_t)n * 8u, fb);
        } else {
          for (int e = lane; e < cnt * n; e += 32) {
            const int r = e / n, cc = e - r * n;
            *(double *)(dst + (size_t)r * GC_ROW + 8 * cc) = W[(r0 + r) * ldw + cc];
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(fb);
        }
        last_g[q] = g;
      }
      if (!ok) break;
    }
    if (lane == 0)
      for (int q = 0; q < 2; ++q)
        if (last_g[q] >= 0) mbar_wait(full0 + 8 * q, (uint32_t)((last_g[q] >> 1) & 1));
  } else if (warp == GCW_MMA) {
    // ------------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint64_t dA0 = umma_desc(smem_addr(slices), 128, GC_SBO);
      const uint64_t dB0 = umma_desc(smem_addr(slices) + GC_SBO, 128, 2 * GC_SBO);
      const uint64_t dA1 = umma_desc(smem_addr(slices + GC_BUF), 128, GC_SBO);
      const uint64_t dB1 = umma_desc(smem_addr(slices + GC_BUF) + GC_SBO, 128, 2 * GC_SBO);
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
          if (!mbar_wait_or_abort(t_empty, (uint32_t)((ev & 1) ^ 1), abort_flag, lim)) {
            ok = false;
            break;
          }
          pending_g = g;
        }
        fence_after_sync();
        uint64_t da = b ? dA1 : dA0, db = b ? dB1 : dB0;
        asm volatile("" : "+l"(da), "+l"(db));
        gc_issue_group(tmem, da, db, !merge);
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
  } else if (warp < 4) {
    // ------------------------------------------------------------------ scales and slices
    // Lane: columns J0 = 16 warp + (lane & 15) and J1 = J0 + 64, rows 16 h .. 16 h + 15 of the
    // group (h = lane >> 4).
    const int h = lane >> 4;
    constexpr int RPT = GC_GROUP / 2;
    int Jc[2], E[2], mxe[2];
    Jc[0] = 16 * warp + (lane & 15);
    Jc[1] = Jc[0] + 64;
    int ev_len = 0, n_scale_syncs = 0;
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1;  // stage slot and slice buffer of the group
      bool ok = mbar_wait_or_abort(full0 + 8 * b, (uint32_t)((g >> 1) & 1), abort_flag, lim);
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      const int cnt = sub_rows(g, 0) - RPT * h;  // rows of this lane's range that exist
      const uint8_t *srow = stage + (size_t)b * GC_STAGE + (size_t)(RPT * h) * GC_ROW;
      const bool spec = g > 0 && ev_len < GC_EV_GROUPS;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int J = Jc[cc];
        const bool cj = J < n;
        if (spec) {
          E[cc] = colE[((g - 1) & 3) * GC_COLS + J];
        } else {
          int mx = 0;
#pragma unroll 8
          for (int r = 0; r < RPT; ++r) {
            const unsigned long long bits = (cj && r < cnt) ? *(const unsigned long long *)(srow + r * GC_ROW + 8 * J) : 0ULL;
            mx = max(mx, (int)((bits >> 52) & 0x7ff));
          }
          mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
          E[cc] = scale_exp(mx) + 1;
        }
      }
      // the products of group g - 2 have read slice buffer b
      if (!mbar_wait_or_abort(sle0 + 8 * b, (uint32_t)(((g >> 1) & 1) ^ 1), abort_flag, lim)) {
        if (lane == 0) fail();
        break;
      }
      bool merge = false;
      for (int attempt = 0; attempt < 2; ++attempt) {
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int J = Jc[cc];
          const bool cj = J < n;
          uint8_t *buf = slices + (size_t)b * GC_BUF + gc_col_off(J);
          int mxl = 0;
#pragma unroll 1
          for (int r0 = 0; r0 < RPT; r0 += 8) {
            uint32_t w[4][NDIG];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int ra = r0 + 2 * u, rb = ra + 1;
              const unsigned long long ba = (cj && ra < cnt) ? *(const unsigned long long *)(srow + ra * GC_ROW + 8 * J) : 0ULL;
              const unsigned long long bb = (cj && rb < cnt) ? *(const unsigned long long *)(srow + rb * GC_ROW + 8 * J) : 0ULL;
              mxl = max(mxl, max((int)((ba >> 52) & 0x7ff), (int)((bb >> 52) & 0x7ff)));
              digits2_biased(fix54_biased<DIG_BIAS>(ba, E[cc]), fix54_biased<DIG_BIAS>(bb, E[cc]), w[u]);
            }
            const int kg = (RPT * h + r0) >> 3;  // K-group of rows r0 .. r0 + 7 within the group
#pragma unroll
            for (int p = 0; p < NDIG; ++p)
              *(uint4 *)(buf + (size_t)(NDIG - 1 - p) * GC_SLICE + kg * 128) = make_uint4(w[0][p], w[1][p], w[2][p], w[3][p]);
          }
          mxe[cc] = mxl;
        }
        if (!spec || attempt == 1) break;
        // did any value of the group reach the event's scale?  (the four slicer warps meet)
        const bool over = __any_sync(0xffffffffu, (Jc[0] < n && mxe[0] >= E[0] + 1023) ||
                                                       (Jc[1] < n && mxe[1] >= E[1] + 1023));
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
        for (int cc = 0; cc < 2; ++cc) {
          const int mm = max(mxe[cc], __shfl_xor_sync(0xffffffffu, mxe[cc], 16));
          E[cc] = scale_exp(mm) + 1;  // cut again with the group's own scales
        }
      }
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      ev_len = merge ? ev_len + 1 : 1;
      // four scale slots: an event's read-back uses its last group's slot, and the slicers cannot
      // get further than three groups past that group before the read-back is done
      if (h == 0) {
        colE[(g & 3) * GC_COLS + Jc[0]] = E[0];
        colE[(g & 3) * GC_COLS + Jc[1]] = E[1];
      }
      if (warp == 0 && lane == 0) evt[g % 3] = merge;
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * b);
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(slf0 + 8 * b);
    }
  } else {
    // ------------------------------------------------------------------ recombination and sums
    // Warp w: TMEM lanes 32 (w & 3) .. (columns J of W), B columns 32 kh .. 32 kh + 31.
    const int quad = warp & 3, kh = (warp - 4) >> 2;
    const int L = 32 * quad + lane;
    const int J = 64 * ((L >> 3) & 1) + 8 * (L >> 4) + (L & 7);
    const uint32_t tq = tmem + ((uint32_t)(32 * quad) << 16);
    double S[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) S[c] = 0.0;
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
      const int *ce = colE + (g & 3) * GC_COLS;
      const int ebase = ce[J] - 51;
#pragma unroll
      for (int h4 = 0; h4 < 8; ++h4) {
        const int k0 = 32 * kh + 4 * h4;
        uint32_t v[NDIG][4];
#pragma unroll
        for (int gg = 0; gg < NDIG; ++gg) tmem_ld4(tq + (uint32_t)(gg * 64 + k0), v[gg]);
        tmem_wait_ld();
        tmem_regs_ready(v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const long long t = recombine_g7w(v[0][c], v[1][c], v[2][c], v[3][c], v[4][c], v[5][c], v[6][c], v[7][c]);
          S[4 * h4 + c] += int_times_pow2_cvt(t, ebase + ce[64 + k0 + c]);  // T / 256
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(t_empty);
    }
    if (J < n) {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int k = 64 + 32 * kh + c;  // column of G
        if (k < n && J <= k) atomicAdd(&Gp[tri_idx(J, k)], S[c]);
      }
    }
  }

  __syncthreads();
  fence_after_sync();
  if (warp == GCW_MMA) tmem_free(tmem, GC_TMEM_COLS);
}

cudaError_t launch_gram_cross(const double *W, int64_t ldw, int64_t m, int64_t n, double *Gpacked, int num_sms,
                              DevStatus *st, cudaStream_t s) {
  if (n <= 64 || n > GC_COLS) return cudaErrorInvalidValue;
  int64_t ctas = std::min<int64_t>(ceil_div(m, GC_GROUP), (int64_t)num_sms);
  const int64_t rows_per_cta = ceil_div(ceil_div(m, ctas), GC_GROUP) * GC_GROUP;
  ctas = ceil_div(m, rows_per_cta);
  const bool aligned = ((uintptr_t)W & 15) == 0;
  const int load_mode = (aligned && n == GC_COLS && ldw == GC_COLS) ? GC_LOAD_BLOCK
                        : (aligned && (n * 8) % 16 == 0 && (ldw * 8) % 16 == 0) ? GC_LOAD_ROWS
                                                                                 : GC_LOAD_PLAIN;
  cudaError_t e = cudaFuncSetAttribute(k_gram_cross, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GC_SMEM);
  if (e != cudaSuccess) return e;
  k_gram_cross<<<(unsigned)ctas, GC_THREADS, GC_SMEM, s>>>(W, ldw, m, (int)n, Gpacked, rows_per_cta, load_mode, st);
  return cudaGetLastError();
}

}  // namespace rq
