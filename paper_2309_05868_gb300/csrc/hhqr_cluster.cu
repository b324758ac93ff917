// hhqr_cluster.cu -- Householder QR of the small sketch Ws (rows x n, row-major), giving R_s
// (Algorithm 3 step 3), on one thread-block cluster of HC_CTAS CTAs that hand the reflectors
// over through distributed shared memory.
//
// CTA b of the cluster keeps the columns k = b + HC_CTAS c in its shared memory (column-major,
// so a warp walks down a column with unit stride).  Step j: the owner of column j has formed
// reflector j (sigma = ||a_(j+1:), j||^2, beta = -sign(a_jj) sqrt(a_jj^2 + sigma),
// tau = (beta - a_jj) / beta, v = a_(j+1:), j / (a_jj - beta), the LAPACK dlarfg form) into its
// publish buffer and raised its flag to j + 1; every CTA waits for that flag (an acquire load
// of the owner's shared memory through the cluster window), copies tau, beta and v into its own
// shared memory, and applies the reflector to its columns k > j, one warp per column.  The owner
// of column j + 1 updates that column first and publishes reflector j + 1 before its other
// columns (look-ahead), so a step costs one column update plus one flag hand-over inside the
// cluster instead of two trips through L2.
//
// A CTA has one publish buffer.  Rewriting it with reflector j + 1 is safe: every other CTA
// published one of the reflectors j + 2 - HC_CTAS .. j (consecutive columns belong to
// consecutive CTAs), which it formed only after reading reflector j + 1 - HC_CTAS, the buffer's
// previous content.  Flags are set before the first cluster barrier, so no CTA reads another's
// shared memory before it is initialised, and a second barrier keeps every CTA alive until no
// other CTA reads its shared memory.  Waits are bounded (RANDQR_ERR_TIMEOUT); a CTA whose wait
// ran out leaves the step loop but still meets the final barrier, and so do the others once
// their own waits run out.
#include "common.cuh"

namespace rq {

namespace {

constexpr int HC_CTAS = 8, HC_THREADS = 256, HC_MAX_WAIT = 1 << 22;

__device__ __forceinline__ uint32_t hc_smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// the address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t hc_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ double hc_ld_remote(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];\n" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ int hc_ld_acquire(uint32_t addr) {
  int v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];\n" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void hc_st_release(uint32_t addr, int v) {
  asm volatile("st.release.cluster.shared::cta.u32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void hc_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ uint32_t hc_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}

// Sum of one value per thread over the CTA, returned to every thread (red: 32 doubles).  Ends
// with a barrier, so shared-memory writes before it are seen by every thread after it.
__device__ __forceinline__ double hc_block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // red is free (an earlier sum's readers are done)
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < HC_THREADS / 32; ++w) t += red[w];
  return t;
}

// Reflector j from local column `col` (one warp): pub = [tau, beta, v_0 .. v_(rows-1)] with v
// stored at its row index (rows j + 1 ..); col keeps beta at row j and v below.
__device__ __forceinline__ void hc_reflect(double *col, int rows, int j, double *pub, int lane) {
  double part = 0.0;
  for (int i = j + 1 + lane; i < rows; i += 32) part = fma(col[i], col[i], part);
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const double x0 = col[j];
  double tau = 0.0, beta = x0, rv0 = 0.0;
  if (part != 0.0) {
    const double alpha = sqrt(x0 * x0 + part);
    beta = (x0 >= 0.0) ? -alpha : alpha;
    rv0 = 1.0 / (x0 - beta);
    tau = (beta - x0) / beta;
  }
  for (int i = j + 1 + lane; i < rows; i += 32) {
    const double v = col[i] * rv0;
    col[i] = v;
    pub[2 + i] = v;
  }
  __syncwarp();  // every lane has read x0
  if (lane == 0) {
    col[j] = beta;
    pub[0] = tau;
    pub[1] = beta;
  }
}

}  // namespace

__global__ void __launch_bounds__(HC_THREADS) k_hhqr_cluster(const double *Ag, int rows, int n, double *Rp,
                                                            DevStatus *st) {
  // every CTA of the cluster runs to the final barrier, also after a failed status
  const bool dead = status_failed(st);
  const int lim = wait_bound(st, HC_MAX_WAIT);
  extern __shared__ double hc_sm[];
  const int b = (int)hc_rank(), tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ncl = (n - b + HC_CTAS - 1) / HC_CTAS;  // local columns: k = b + HC_CTAS c
  const int ncl_max = (n + HC_CTAS - 1) / HC_CTAS;
  double *cols = hc_sm;                                 // ncl_max x rows
  double *vsh = cols + (size_t)ncl_max * rows;          // rows: current reflector's v
  double *pub = vsh + rows;                             // rows + 2: [tau, beta, v]
  double *betas = pub + rows + 2;                       // n: every reflector's beta
  __shared__ int s_flag;                                // reflectors published by this CTA: last j + 1
  __shared__ int s_fail;
  __shared__ double s_tau, s_rv0;
  __shared__ double red[32];
  for (int e = tid; e < ncl * rows; e += HC_THREADS) {
    const int c = e / rows, i = e - c * rows;
    cols[e] = Ag[(size_t)i * n + b + HC_CTAS * c];
  }
  if (tid == 0) {
    s_flag = 0;
    s_fail = dead ? 1 : 0;
  }
  __syncthreads();
  if (!dead && b == 0 && warp == 0) {  // reflector 0 from its owner
    hc_reflect(cols, rows, 0, pub, lane);
    __syncwarp();
    if (lane == 0) hc_st_release(hc_smem_addr(&s_flag), 1);
  }
  hc_cluster_sync();  // flags initialised everywhere before anyone reads them
  const uint32_t flag_local = hc_smem_addr(&s_flag), pub_local = hc_smem_addr(pub);
  for (int j = 0; j < n && !s_fail; ++j) {
    const uint32_t owner = (uint32_t)(j % HC_CTAS);
    if (tid == 0) {
      const uint32_t fa = hc_map(flag_local, owner);
      int ok = 0;
      for (int it = 0; it < lim && !ok; ++it) ok = hc_ld_acquire(fa) >= j + 1;
      if (!ok) {
        s_fail = 1;
        status_fail(st, RANDQR_ERR_TIMEOUT, j + 1, 0);
      }
    }
    __syncthreads();
    if (s_fail) break;
    const uint32_t pa = hc_map(pub_local, owner);
    for (int i = j + 1 + tid; i < rows; i += HC_THREADS) vsh[i] = hc_ld_remote(pa + 8u * (uint32_t)(2 + i));
    if (tid == 0) {
      s_tau = hc_ld_remote(pa);
      betas[j] = hc_ld_remote(pa + 8u);
    }
    __syncthreads();
    const double tau = s_tau;
    // The owner of column j + 1 updates that column and forms reflector j + 1 first (the step's
    // critical path), then its other columns one warp each; the other CTAs go straight to their
    // columns.  Tall sketches (rows >= 256) spread the critical column over all the owner's
    // threads, so its FP64 work runs on every scheduler; shorter ones keep it on one warp.
    const int c_next = (j + 1 < n && (j + 1) % HC_CTAS == b) ? (j + 1) / HC_CTAS : -1;
    const bool coop = rows >= 256;
    if (c_next >= 0 && !coop && warp == 0) {
      double *col = cols + (size_t)c_next * rows;
      if (tau != 0.0) {
        double acc = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) acc = fma(vsh[i], col[i], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double w = tau * (col[j] + acc);
        __syncwarp();
        if (lane == 0) col[j] -= w;
        for (int i = j + 1 + lane; i < rows; i += 32) col[i] = fma(-vsh[i], w, col[i]);
        __syncwarp();
      }
      hc_reflect(col, rows, j + 1, pub, lane);
      __syncwarp();  // the warp's writes of the reflector, then the flag (release, cluster scope)
      if (lane == 0) hc_st_release(flag_local, j + 2);
    }
    if (c_next >= 0 && coop) {
      double *col = cols + (size_t)c_next * rows;
      if (tau != 0.0) {
        double part = 0.0;
        for (int i = j + 1 + tid; i < rows; i += HC_THREADS) part = fma(vsh[i], col[i], part);
        const double w = tau * (col[j] + hc_block_sum(part, red));  // all threads read col[j] ...
        for (int i = j + 1 + tid; i < rows; i += HC_THREADS) col[i] = fma(-vsh[i], w, col[i]);
        __syncthreads();                                            // ... before it changes
        if (tid == 0) col[j] -= w;
      }
      double part = 0.0;
      for (int i = j + 2 + tid; i < rows; i += HC_THREADS) part = fma(col[i], col[i], part);
      const double sigma = hc_block_sum(part, red);  // also orders the update before the reads below
      if (tid == 0) {
        const double x0 = col[j + 1];
        double tau1 = 0.0, beta = x0, rv0 = 0.0;
        if (sigma != 0.0) {
          const double alpha = sqrt(x0 * x0 + sigma);
          beta = (x0 >= 0.0) ? -alpha : alpha;
          rv0 = 1.0 / (x0 - beta);
          tau1 = (beta - x0) / beta;
        }
        s_rv0 = rv0;
        col[j + 1] = beta;
        pub[0] = tau1;
        pub[1] = beta;
      }
      __syncthreads();
      const double rv0 = s_rv0;
      for (int i = j + 2 + tid; i < rows; i += HC_THREADS) {
        const double v = col[i] * rv0;
        col[i] = v;
        pub[2 + i] = v;
      }
      __syncthreads();  // the whole reflector is written, then the flag (release, cluster scope)
      if (tid == 0) hc_st_release(flag_local, j + 2);
    }
    if (tau != 0.0) {
      for (int c = warp; c < ncl; c += HC_THREADS / 32) {
        const int k = b + HC_CTAS * c;
        if (k <= j || c == c_next) continue;
        double *col = cols + (size_t)c * rows;
        double acc = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) acc = fma(vsh[i], col[i], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double w = tau * (col[j] + acc);
        __syncwarp();
        if (lane == 0) col[j] -= w;
        for (int i = j + 1 + lane; i < rows; i += 32) col[i] = fma(-vsh[i], w, col[i]);
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (!s_fail) {
    // R (rows flipped to a positive diagonal), packed column-major upper: this CTA's columns
    for (int c = 0; c < ncl; ++c) {
      const int k = b + HC_CTAS * c;
      for (int i = tid; i <= k; i += HC_THREADS) {
        const double v = i == k ? betas[k] : cols[(size_t)c * rows + i];
        Rp[tri_idx(i, k)] = betas[i] < 0.0 ? -v : v;
      }
    }
    if (b == 0 && tid == 0) {
      double dmin = INFINITY, dmax = 0.0;
      int bad = 0;
      for (int k = 0; k < n; ++k) {
        const double d = fabs(betas[k]);
        if (!(d > 0.0) || !isfinite(d)) bad = bad ? bad : k + 1;
        dmin = fmin(dmin, d);
        dmax = fmax(dmax, d);
      }
      st->dmin = dmin;
      st->dmax = dmax;
      if (bad) status_fail(st, RANDQR_ERR_RANK, bad, 0);
    }
  }
  hc_cluster_sync();  // nobody reads this CTA's shared memory any more
}

size_t hhqr_cluster_smem(int64_t rows, int64_t n) {
  const int64_t ncl_max = (n + HC_CTAS - 1) / HC_CTAS;
  return sizeof(double) * (size_t)(ncl_max * rows + rows + rows + 2 + n);
}

bool hhqr_cluster_ok(int64_t rows, int64_t n) {
  return n >= 2 * HC_CTAS && rows >= n && hhqr_cluster_smem(rows, n) <= 200 * 1024;
}

cudaError_t launch_hhqr_cluster(const double *A, int64_t rows, int64_t n, double *Rpacked, DevStatus *st,
                                cudaStream_t s) {
  const size_t smem = hhqr_cluster_smem(rows, n);
  cudaError_t e = cudaFuncSetAttribute(k_hhqr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(HC_CTAS);
  cfg.blockDim = dim3(HC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = HC_CTAS;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_hhqr_cluster, A, (int)rows, (int)n, Rpacked, st);
}

}  // namespace rq
