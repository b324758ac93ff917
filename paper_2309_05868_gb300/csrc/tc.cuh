// tc.cuh -- fifth-generation tensor core (tcgen05) and bulk-copy primitives, and the exact
// integer splitting of FP64 / pair values, shared by the split-product kernels.
//
// Splitting: a value w with scale 2^E > |w| becomes the 56-bit fixed point
// X = trunc(|w| 2^(56 - E)), cut into eight 7-bit digits a_s = (X >> (49 - 7 s)) & 127
// (the top digit may reach 128 for pair inputs), each carrying the sign of w:
// w = 2^(E - 56) sum_s a_s 2^(49 - 7 s) up to 2^(E - 56).  bf16 holds every digit exactly and
// the tensor cores accumulate digit products exactly in FP32 while the sums stay below 2^24.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace rq {
namespace tc {

constexpr int SLICES = 8;
constexpr int MAX_WAIT = 1 << 24;  // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major, no swizzle: lbo = byte step between core matrices
// (8 rows x 16 bytes) along K, sbo = byte step between 8-row groups.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: kind::f16 with bf16 A and B (both K-major), FP32 D, M x N.
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

// D = A B + 2^-7 D (scale-input-d): folds the sums already in D in at a 2^-7 lower weight.
__device__ __forceinline__ void umma_scaled7(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, 1, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p, 7;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar));
}

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar));
}

// Poll an mbarrier phase, at most `limit` times; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit = MAX_WAIT) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
  return done != 0;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}

// Bulk asynchronous copy global -> shared (TMA engine), completion counted in bytes on mbar.
// Addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// Bulk asynchronous copy shared -> global; bulk_store_wait() returns once the shared source
// has been read (it may then be overwritten).
__device__ __forceinline__ void bulk_store(void *dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_store_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_store_wait() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }

// 16-byte asynchronous copy global -> shared (through L2, not L1); an ordinary load as far as
// memory ordering goes.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
// arrives on mbar once this thread's earlier cp.async copies have landed (no extra pending count)
__device__ __forceinline__ void cp_async_arrive(uint32_t mbar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(mbar) : "memory");
}

// Thread-block clusters: this CTA's rank, a barrier over every thread of the cluster, the
// address of a shared-memory location in CTA `rank`, and release/acquire on 32-bit words.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ uint32_t map_shared_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t ld_acquire_cluster_u32(uint32_t cluster_addr) {
  uint32_t v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];\n" : "=r"(v) : "r"(cluster_addr) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_cluster_u32(uint32_t cluster_addr) {
  uint32_t v;
  asm volatile("ld.relaxed.cluster.shared::cluster.u32 %0, [%1];\n" : "=r"(v) : "r"(cluster_addr) : "memory");
  return v;
}
// after relaxed loads that saw values written by releases: makes the writes before those
// releases visible to this thread's later accesses
__device__ __forceinline__ void fence_acquire_cluster() { asm volatile("fence.acq_rel.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void st_release_cluster_u32(uint32_t local_addr, uint32_t v) {
  asm volatile("st.release.cluster.shared::cta.u32 [%0], %1;\n" ::"r"(local_addr), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

// Tensor memory, allocated by one whole warp; the address lands in *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(slot)),
               "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(cols));
}

// 8 consecutive columns of this warp's 32 tensor-memory lanes (thread = lane).
__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(addr));
}
// 4 consecutive columns of this warp's 32 tensor-memory lanes (thread = lane).
__device__ __forceinline__ void tmem_ld4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
// 16 tensor-memory lanes x 8 consecutive columns: thread t gets lanes t / 4 and t / 4 + 8 of the
// 16, columns 2 (t % 4) and 2 (t % 4) + 1: r = {(t/4, 2(t%4)), (t/4, 2(t%4)+1), (t/4+8, 2(t%4)),
// (t/4+8, 2(t%4)+1)}.
__device__ __forceinline__ void tmem_ld16x256(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Orders uses of tcgen05.ld destination registers after the tcgen05.wait::ld that completes
// them: the compiler does not know the loads are asynchronous.
template <int R, int C>
__device__ __forceinline__ void tmem_regs_ready(uint32_t (&v)[R][C]) {
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < C; ++c) asm volatile("" : "+r"(v[r][c]));
}

// Exponent field of an element rebased to the FP64 bias; 0 for zero / subnormal.
template <bool IN_DF>
__device__ __forceinline__ int expfield(const void *p) {
  if (IN_DF) {
    const int ef = (__float_as_uint(((const float2 *)p)->x) >> 23) & 0xff;
    return ef ? ef - 127 + 1023 : 0;
  }
  return (int)(((unsigned long long)__double_as_longlong(*(const double *)p) >> 52) & 0x7ff);
}

// Scale exponent E (|w| < 2^E) from the largest exponent field of a set; tiny sets clamp.
__device__ __forceinline__ int scale_exp(int expfield_max) { return max(expfield_max - 1023 + 1, -100); }

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

// Digit s of a fixed-point value, as bf16 bits.
__device__ __forceinline__ uint32_t digit_bf16(long long x, int s) {
  const unsigned long long ax = (unsigned long long)(x < 0 ? -x : x);
  const int a = (int)((ax >> (49 - 7 * s)) & (s == 0 ? 255 : 127));
  return int_to_bf16_bits(x < 0 ? -a : a);
}

__device__ __forceinline__ float pow2f(int e) {  // 2^e, e clamped to [-126, 127]
  e = max(min(e, 127), -126);
  return __uint_as_float((uint32_t)(e + 127) << 23);
}

// Element offset (bf16 units) of (row, k) in a K-major, unswizzled tile with kdim columns.
__device__ __forceinline__ int kmajor_off(int row, int k, int kdim) {
  return ((row >> 3) * (kdim >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

}  // namespace tc
}  // namespace rq

namespace rq {
namespace tc {

// ---------------------------------------------------------------------------------------
// Balanced 7-bit digits (f16 operands).  An integer X with |X| < 2^54 is written as
// X = sum_{p=0}^{7} d_p 2^(7p) with d_p in [-64, 63]: the bytes-of-seven of X + DIG_BIAS,
// DIG_BIAS = sum_p 64 * 2^(7p), are d_p + 64.  Each d_p is an exact f16, and a product of
// two digits is at most 2^12 in magnitude.
// ---------------------------------------------------------------------------------------
constexpr int NDIG = 8;
constexpr unsigned long long DIG_BIAS = 0x81020408102040ULL;

// Instruction descriptor: kind::f16 with f16 A and B (both K-major), FP32 D, M x N.
__device__ __forceinline__ uint32_t umma_idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init_count(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

// Poll an mbarrier phase at most `limit` times, giving up early once *abort is set.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t mbar, uint32_t parity, volatile int *abort,
                                                   int limit = MAX_WAIT) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort) return false;
  }
  return false;
}

// trunc(x 2^(54 - E)) for |x| < 2^E, as a signed integer (|.| < 2^54).
__device__ __forceinline__ long long fix54(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7ff);
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
  const int sh = ef - 1021 - E;  // x = mant 2^(ef - 1075)
  long long v = sh >= 0 ? (mant << (sh & 1)) : (-sh < 63 ? (mant >> -sh) : 0);
  v = ef == 0 ? 0 : v;
  return (b >> 63) ? -v : v;
}
__device__ __forceinline__ long long fix54(float f, int E) {
  const uint32_t b = __float_as_uint(f);
  const int ef = (int)((b >> 23) & 0xff);
  const long long mant = (long long)((b & 0x7fffff) | 0x800000);
  const int sh = ef - 96 - E;  // f = mant 2^(ef - 150)
  long long v = sh >= 0 ? (sh < 31 ? (mant << sh) : 0) : (-sh < 63 ? (mant >> -sh) : 0);
  v = ef == 0 ? 0 : v;
  return (b >> 31) ? -v : v;
}

__device__ __forceinline__ uint32_t hsub2_bits(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Digit words of two fixed-point values already offset by DIG_BIAS (ya = xa + DIG_BIAS):
// w[p] = f16(d_p(xa)) | f16(d_p(xb)) << 16.
__device__ __forceinline__ void digits2_biased(unsigned long long ya, unsigned long long yb, uint32_t (&w)[NDIG]) {
  const uint32_t la = (uint32_t)ya, ha = (uint32_t)(ya >> 32);
  const uint32_t lb = (uint32_t)yb, hb = (uint32_t)(yb >> 32);
  uint32_t win[4];  // window q: bits 14q .. 14q + 13 of each value, one per 16-bit half
  win[0] = __byte_perm(la, lb, 0x5410);
  win[1] = __byte_perm(la >> 14, lb >> 14, 0x5410);
  win[2] = __byte_perm(__funnelshift_r(la, ha, 28), __funnelshift_r(lb, hb, 28), 0x5410);
  win[3] = __byte_perm(ha >> 10, hb >> 10, 0x5410);
  // f16(1024 + y) = 0x6400 | y for y < 1024; subtracting f16(1088) leaves y - 64 exactly.
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    w[2 * q] = hsub2_bits((win[q] & 0x007F007Fu) | 0x64006400u, 0x64406440u);
    w[2 * q + 1] = hsub2_bits(((win[q] >> 7) & 0x007F007Fu) | 0x64006400u, 0x64406440u);
  }
}
__device__ __forceinline__ void digits2(long long xa, long long xb, uint32_t (&w)[NDIG]) {
  digits2_biased((unsigned long long)xa + DIG_BIAS, (unsigned long long)xb + DIG_BIAS, w);
}

// The integer value of an FP32 accumulator that holds an exact integer of magnitude < 2^22.
__device__ __forceinline__ int acc_to_int(uint32_t bits) {
  return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}

// ---------------------------------------------------------------------------------------
// Recombination of eight region accumulators (exact FP32 integers, |D_g| <= 2^22) into
//   T = sum_g 2^(7 (7 - g)) D_g,
// returned as T / 2^SH in an int64.  Each accumulator goes through one FP32 add of
// 1.5 * 2^23, after which its bit pattern is 0x4B400000 + D_g; the patterns are summed with
// 32 x 32 -> 64-bit multiply-adds and the offsets removed by one constant.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mad_wide(uint32_t a, uint32_t b, unsigned long long c) {
  unsigned long long d;
  asm("mad.wide.u32 %0, %1, %2, %3;\n" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint32_t acc_bits(uint32_t v) {
  return __float_as_uint(__uint_as_float(v) + 12582912.0f);
}
template <int SH>
__device__ __forceinline__ long long recombine8(uint32_t d0, uint32_t d1, uint32_t d2, uint32_t d3, uint32_t d4,
                                                uint32_t d5, uint32_t d6, uint32_t d7) {
  // sum of the offsets 0x4B400000 * (2^21 + 2^14 + 2^7 + 1), for each half
  constexpr unsigned long long OFF = 0x4B400000ULL * ((1ULL << 21) + (1ULL << 14) + (1ULL << 7) + 1ULL);
  unsigned long long h = mad_wide(acc_bits(d0), 1u << 21, 0ULL);
  h = mad_wide(acc_bits(d1), 1u << 14, h);
  h = mad_wide(acc_bits(d2), 1u << 7, h);
  h += acc_bits(d3);
  unsigned long long l = mad_wide(acc_bits(d4), 1u << 21, 0ULL);
  l = mad_wide(acc_bits(d5), 1u << 14, l);
  l = mad_wide(acc_bits(d6), 1u << 7, l);
  l += acc_bits(d7);
  const long long th = (long long)(h - OFF), tl = (long long)(l - OFF);
  return (th << (28 - SH)) + (tl >> SH);
}

// T / 256 from eight region accumulators of 7-bit-digit products over up to 1024 rows,
// T = sum_g 2^(7 (7 - g)) D_g, each D_g an exact FP32 integer with |D_g| <= 2^24,
// |D_1| <= 2^22 and |D_0| <= 2^21 (the leading digits are at most 32 in magnitude).  The
// regions are converted exactly to int32 and combined: regions 0 and 1 in the high word
// (D_0 2^9 + D_1 2^2 < 2^31), the rest in a 64-bit sum; regions 6 and 7 enter as
// floor((128 D_6 + D_7) / 256), an error below one unit of T / 256.
__device__ __forceinline__ long long recombine_g7w(uint32_t d0, uint32_t d1, uint32_t d2, uint32_t d3, uint32_t d4,
                                                   uint32_t d5, uint32_t d6, uint32_t d7) {
  const int D0 = __float2int_rz(__uint_as_float(d0)), D1 = __float2int_rz(__uint_as_float(d1));
  const int D2 = __float2int_rz(__uint_as_float(d2)), D3 = __float2int_rz(__uint_as_float(d3));
  const int D4 = __float2int_rz(__uint_as_float(d4)), D5 = __float2int_rz(__uint_as_float(d5));
  const int D6 = __float2int_rz(__uint_as_float(d6)), D7 = __float2int_rz(__uint_as_float(d7));
  const int hw = D0 * 512 + D1 * 4;
  long long lw = ((long long)D6 * 128 + D7) >> 8;
  lw += (long long)D5 * 64;
  lw += (long long)D4 * (1LL << 13);
  lw += (long long)D3 * (1LL << 20);
  lw += (long long)D2 * (1LL << 27);
  return (long long)((unsigned long long)lw + ((unsigned long long)(unsigned)hw << 32));
}

// (double) t * 2^e for |t| < 2^63 and a result in the normal range (0 for t == 0), through the
// FP64 pipe's int64 conversion: for kernels whose FP64 pipe is otherwise idle and whose issue
// slots are the scarce resource.
__device__ __forceinline__ double int_times_pow2_cvt(long long t, int e) {
  const double y = (double)t;
  const int hi = __double2hiint(y);  // nonzero exactly when t is
  return __hiloint2double(hi + (hi != 0 ? (e << 20) : 0), __double2loint(y));
}

// (double) t * 2^e, rounded to nearest (ties away from zero), for |t| < 2^63 and a result in
// the normal range; 0 for t == 0.  Integer instructions only: the FP64 pipe (about 1/64 of the
// FP32 rate on this part) is left to the callers' additions.
__device__ __forceinline__ double int_times_pow2(long long t, int e) {
  const unsigned long long sgn = (unsigned long long)(t >> 63);
  unsigned long long a = ((unsigned long long)t ^ sgn) - sgn;  // |t|
  const int lz = __clzll((long long)a);                        // 64 when t == 0
  a <<= (lz & 63);                                             // leading one at bit 63
  unsigned long long r = a + 0x400ULL;                         // round at bit 10
  const int carry = r < a;
  r = carry ? (1ULL << 63) : r;
  const unsigned long long ex = (unsigned long long)(1023 + 63 - lz + carry + e);
  const unsigned long long bits = (sgn << 63) | (ex << 52) | ((r >> 11) & 0xFFFFFFFFFFFFFULL);
  return t == 0 ? 0.0 : __longlong_as_double((long long)bits);
}

}  // namespace tc
}  // namespace rq

namespace rq {
namespace tc {

// ---------------------------------------------------------------------------------------
// Balanced byte digits (f16 operands) of the triangular products.  An integer X with
// |X| < 2^54 is written as X = sum_{p=0}^{6} d_p 2^(8p) with d_p in [-128, 127] (the leading
// digit then lies in [-64, 64]): byte p of X + BIAS8, BIAS8 = sum_p 128 * 2^(8p), is d_p + 128.
// f16 holds every digit exactly; a product of two digits is at most 2^14 in magnitude, and
// at most 2^13 when one of them is a leading digit.
// ---------------------------------------------------------------------------------------
constexpr int NDIG8 = 7;
constexpr unsigned long long BIAS8 = 0x80808080808080ULL;

// Digit words of two fixed-point values: w[p] = f16(d_p(xa)) | f16(d_p(xb)) << 16.  One byte
// permute puts byte p of both values in the low bytes of the two halves; f16(1024 + y) is
// 0x6400 | y, and subtracting f16(1152) leaves y - 128 exactly.
__device__ __forceinline__ void digits8_biased(unsigned long long ya, unsigned long long yb, uint32_t (&w)[NDIG8]) {
  const uint32_t la = (uint32_t)ya, ha = (uint32_t)(ya >> 32);
  const uint32_t lb = (uint32_t)yb, hb = (uint32_t)(yb >> 32);
#pragma unroll
  for (int p = 0; p < NDIG8; ++p) {
    const uint32_t q = (uint32_t)(p & 3);
    const uint32_t sel = q | ((q + 4u) << 8);
    const uint32_t v = p < 4 ? __byte_perm(la, lb, sel) : __byte_perm(ha, hb, sel);
    w[p] = hsub2_bits((v & 0x00FF00FFu) | 0x64006400u, 0x64806480u);
  }
}
__device__ __forceinline__ void digits8(long long xa, long long xb, uint32_t (&w)[NDIG8]) {
  digits8_biased((unsigned long long)xa + BIAS8, (unsigned long long)xb + BIAS8, w);
}

// X + BIAS (mod 2^64) for the FP64 value with bit pattern b, X = trunc(|x| 2^(54 - E)) with the
// sign of x, for |x| < 2^E (what digits8 of fix54(x, E) starts from, with BIAS = BIAS8, and
// digits2 with BIAS = DIG_BIAS).  With x = m 2^(ef - 1075)
// (m the 53-bit significand), X = (2m) >> (1022 + E - ef), a shift of at least 0; zeros and
// subnormals (ef = 0) shift everything out.  The sign is applied as (v ^ s) - s with s = 0 or -1.
template <unsigned long long BIAS = BIAS8>
__device__ __forceinline__ unsigned long long fix54_biased(unsigned long long b, int E) {
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const int ef = (int)((hi >> 20) & 0x7ffu);
  // a value at or above 2^E (only possible where a caller guesses E) shifts everything out
  const unsigned amt = min((unsigned)(1022 + E - ef), 63u);
  const unsigned long long m2 = ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 33) | ((unsigned long long)lo << 1);
  const unsigned long long v = m2 >> amt;
  const unsigned long long sgn = (unsigned long long)((long long)b >> 63);
  return (v ^ sgn) + (BIAS - sgn);
}

// T / 2^12 from eight region accumulators of byte-digit products, T = sum_g 2^(8 (7 - g)) D_g,
// each D_g an exact FP32 integer with |D_g| <= 2^22 for g <= 4 and |D_g| < 2^23 for g >= 5, and
// |T| < 2^74.  Regions 0-4 go through the 1.5 * 2^23 offset (bit pattern 0x4B400000 + D_g).
// Region 5 is split into an even part, through the 1.5 * 2^24 offset (0x4BC00000 + D_5 / 2),
// and a remainder in {-1, 0, 1}.  The remainder and regions 6 and 7 are merged by two FP32
// fused multiply-adds (|r| < 2^31) and taken at a resolution of 2^12 through the 1.5 * 2^35
// offset: an error below 2^11 units of region 7, far below the result's last unit.  The bit
// patterns are then summed with integer multiply-adds modulo 2^64 (the offsets cancel
// through one constant per word): regions 0 and 1 land in the high word (32-bit products),
// the rest in a 64-bit chain, so that combining them costs one add.
__device__ __forceinline__ long long recombine_b8(uint32_t d0, uint32_t d1, uint32_t d2, uint32_t d3, uint32_t d4,
                                                  uint32_t d5, uint32_t d6, uint32_t d7) {
  constexpr uint32_t O23 = 0x4B400000u, O24 = 0x4BC00000u, O35 = 0x51400000u;  // 1.5 * 2^23, 2^24, 2^35
  constexpr uint32_t C_HI = (uint32_t)(O23 * 4096ull + O23 * 16ull);
  constexpr unsigned long long C_LO = (unsigned long long)O23 * (1ull << 28) + (unsigned long long)O23 * (1ull << 20) +
                                      (unsigned long long)O23 * (1ull << 12) + (unsigned long long)O24 * 32ull + O35;
  const float M24 = 25165824.0f, M35 = 51539607552.0f;
  const float v5 = __uint_as_float(d5);
  const float c5 = __fadd_rn(v5, M24);
  const float lo = __fsub_rn(v5, __fsub_rn(c5, M24));
  const float r = __fmaf_rn(lo, 65536.0f, __fmaf_rn(__uint_as_float(d6), 256.0f, __uint_as_float(d7)));
  const uint32_t q5 = __float_as_uint(c5), qr = __float_as_uint(__fadd_rn(r, M35));
  const uint32_t hw = acc_bits(d0) * 4096u + acc_bits(d1) * 16u - C_HI;  // modulo 2^32
  unsigned long long lw = mad_wide(qr, 1u, 0ULL - C_LO);
  lw = mad_wide(q5, 32u, lw);
  lw = mad_wide(acc_bits(d4), 1u << 12, lw);
  lw = mad_wide(acc_bits(d3), 1u << 20, lw);
  lw = mad_wide(acc_bits(d2), 1u << 28, lw);
  return (long long)(lw + ((unsigned long long)hw << 32));
}

}  // namespace tc
}  // namespace rq
