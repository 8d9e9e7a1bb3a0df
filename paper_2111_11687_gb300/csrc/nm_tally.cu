// Tally statistics (§2.1 dose and uncertainty maps, Eq. 1-3).
//
// Per batch b of n_b histories the fold moves the int64 batch tally T_b into
// the exact cumulative tally and accumulates, in FP64, S2 = sum_b T_b^2 / n_b
// per voxel and the organ sums O_b = sum over the organ's voxels of the batch
// dose.  With N = sum n_b histories and K batches the per-decay mean of a
// voxel is x = Tsum / N and the batch estimate of its variance is
//   var(x) = (S2 - Tsum^2 / N) / ((K - 1) N),
// the n_b-weighted form of the batch-means estimator.  Every reduction has a
// fixed tree (per-thread columns in shared memory, then fixed warp trees, then
// blocks in index order), so the statistics are the same on every run.
#include "nm_internal.cuh"

namespace nm {
namespace {

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Reduce acc[l][0..kFoldThreads) for every label into out[l] (fixed tree).
__device__ void reduce_label_columns(const double (*acc)[kFoldThreads], double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int nw = kFoldThreads / 32;
  for (int l = wid; l < kLabelSlots; l += nw) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kFoldThreads / 32; ++j) s += acc[l][lane + 32 * j];
    s = warp_sum_d(s);
    if (lane == 0) out[l] = s;
  }
}

__global__ void __launch_bounds__(kFoldThreads) fold_kernel(const FoldParams p) {
  __shared__ double acc[kLabelSlots][kFoldThreads];
  __shared__ ull dep_w[kFoldThreads / 32];
  for (int l = 0; l < kLabelSlots; ++l) acc[l][threadIdx.x] = 0.0;
  const int64_t v0 = (int64_t)blockIdx.x * kFoldTile;
  const int64_t v1 = v0 + kFoldTile < p.V ? v0 + kFoldTile : p.V;
  ull dep = 0;
  const double inv_nb = 1.0 / p.n_b;
  // A thread's voxels v0 + tid + k kFoldThreads, kFold at a time: all their
  // loads are issued before any update (a lone load per voxel left the kernel
  // bound by DRAM latency), and the updates then follow in voxel order, so
  // every sum is formed exactly as one voxel at a time would.
  constexpr int kFold = 8;
  for (int64_t vb = v0 + threadIdx.x; vb < v1; vb += (int64_t)kFold * kFoldThreads) {
    ull t[kFold], ts[kFold];
    double s2v[kFold];
    float rho[kFold];
    int lab[kFold];
#pragma unroll
    for (int j = 0; j < kFold; ++j) {
      const int64_t v = vb + (int64_t)j * kFoldThreads;
      t[j] = v < v1 ? p.tb[v] : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kFold; ++j) {
      const int64_t v = vb + (int64_t)j * kFoldThreads;
      ts[j] = 0; s2v[j] = 0.0; rho[j] = 1.0f; lab[j] = 0;
      if (t[j]) {
        ts[j] = p.tsum[v];
        s2v[j] = p.s2[v];
        if (p.labels) {
          lab[j] = p.labels[v];
          rho[j] = p.density[v];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kFold; ++j) {
      if (!t[j]) continue;
      const int64_t v = vb + (int64_t)j * kFoldThreads;
      p.tb[v] = 0;
      p.tsum[v] = ts[j] + t[j];
      const double x = (double)t[j];
      p.s2[v] = s2v[j] + x * x * inv_nb;
      dep += t[j];
      // Gy per unit in FP32 (GB300's FP64 divide is slow); the sum stays FP64
      if (p.labels) acc[lab[j]][threadIdx.x] += x * (double)__fdiv_rn((float)p.gy_per_unit_vol, rho[j]);
    }
  }
  // deposited-energy counter (integer, so the order of the adds does not matter)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dep += __shfl_xor_sync(0xffffffffu, dep, o);
  if ((threadIdx.x & 31) == 0) dep_w[threadIdx.x >> 5] = dep;
  __syncthreads();
  if (threadIdx.x == 0) {
    ull s = 0;
    for (int w = 0; w < kFoldThreads / 32; ++w) s += dep_w[w];
    if (s) atomicAdd(p.deposited, s);
  }
  if (p.labels) reduce_label_columns(acc, p.organ_partial + (size_t)blockIdx.x * kLabelSlots);
}

// One warp per label: blocks in index order, lane-strided, then a fixed tree.
__global__ void fold_organs_kernel(const FoldParams p, int n_blocks) {
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (l >= kLabelSlots) return;
  double s = 0.0;
  for (int b = lane; b < n_blocks; b += 32) s += p.organ_partial[(size_t)b * kLabelSlots + l];
  s = warp_sum_d(s);
  if (lane == 0) {
    p.org_s1[l] += s;
    p.org_s2[l] += s * s / p.n_b;
  }
}

__global__ void __launch_bounds__(kFoldThreads) finalize_kernel(const FinalizeParams p) {
  extern __shared__ double sm[];
  double(*acc_d)[kFoldThreads] = (double(*)[kFoldThreads])sm;
  double(*acc_e)[kFoldThreads] = (double(*)[kFoldThreads])(sm + kLabelSlots * kFoldThreads);
  for (int l = 0; l < kLabelSlots; ++l) acc_d[l][threadIdx.x] = acc_e[l][threadIdx.x] = 0.0;
  const int64_t v0 = (int64_t)blockIdx.x * kFoldTile;
  const int64_t v1 = v0 + kFoldTile < p.V ? v0 + kFoldTile : p.V;
  // FP64 where cancellation needs it (the variance: S2 - Tsum^2/N) and in the
  // organ sums; the rest in FP32, whose precision the FP32 outputs have anyway
  // (GB300's FP64 rate is a small fraction of its FP32 rate).
  const double inv_n = 1.0 / p.n_total;
  const double inv_k1n = 1.0 / ((p.n_batches - 1.0) * p.n_total);
  const float gy_a = (float)(p.gy_per_unit_vol * p.activity_bq);
  for (int64_t v = v0 + threadIdx.x; v < v1; v += kFoldThreads) {
    const ull ti = p.tsum[v];
    float d = 0.0f, sg = 0.0f;
    if (ti) {
      const double t = (double)ti;
      const double mean = t * inv_n;                       // units per decay
      const double var = fmax(fma(-t, mean, p.s2[v]), 0.0) * inv_k1n;
      const float conv = __fdiv_rn(gy_a, p.density[v]);
      d = (float)mean * conv;                              // Eq. 1, Gy/s
      sg = sqrtf((float)var) * conv;
    }
    if (p.dose) p.dose[v] = d;
    if (p.sigma) p.sigma[v] = sg;
    if (p.labels) {
      const int l = p.labels[v];
      acc_d[l][threadIdx.x] += (double)d;
      const float eps = d > 0.0f ? __fdiv_rn(sg, d) : 1.0f;
      acc_e[l][threadIdx.x] += (double)(eps * eps);
    }
  }
  if (!p.labels) return;
  __syncthreads();
  double* out = p.organ_partial + (size_t)blockIdx.x * 2 * kLabelSlots;
  reduce_label_columns(acc_d, out);
  reduce_label_columns(acc_e, out + kLabelSlots);
}

__global__ void finalize_organs_kernel(const FinalizeParams p, int n_blocks) {
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (l >= kLabelSlots) return;
  double sd = 0.0, se = 0.0;
  for (int b = lane; b < n_blocks; b += 32) {
    sd += p.organ_partial[(size_t)b * 2 * kLabelSlots + l];
    se += p.organ_partial[(size_t)b * 2 * kLabelSlots + kLabelSlots + l];
  }
  sd = warp_sum_d(sd);
  se = warp_sum_d(se);
  if (lane != 0) return;
  const double cnt = (double)p.organ_count[l];
  double mean = 0.0, eps = 0.0, sig = 0.0;
  if (cnt > 0.0) {
    mean = sd / cnt;                                          // Eq. 2
    eps = sqrt(se / cnt);                                     // Eq. 3
    // Batch sigma of the organ mean: m_b = O_b / (n_b cnt) per decay.
    const double N = p.n_total;
    const double mbar = p.org_s1[l] / (N * cnt);
    const double sum_nm2 = p.org_s2[l] / (cnt * cnt);
    const double var = fmax(sum_nm2 - N * mbar * mbar, 0.0) / ((p.n_batches - 1.0) * N);
    sig = sqrt(var) * p.activity_bq;
  }
  p.organ_out[l] = mean;
  p.organ_out[kLabelSlots + l] = eps;
  p.organ_out[2 * kLabelSlots + l] = sig;
  p.organ_out[3 * kLabelSlots + l] = cnt;
}

// Eq. 2 over an arbitrary dose map: per-CTA per-label partial sums (fixed tree).
__global__ void __launch_bounds__(kFoldThreads) map_organ_kernel(const float* __restrict__ dose,
                                                                 const uint8_t* __restrict__ labels, int64_t V,
                                                                 double* __restrict__ part) {
  __shared__ double acc[kLabelSlots][kFoldThreads];
  for (int l = 0; l < kLabelSlots; ++l) acc[l][threadIdx.x] = 0.0;
  const int64_t v0 = (int64_t)blockIdx.x * kFoldTile;
  const int64_t v1 = v0 + kFoldTile < V ? v0 + kFoldTile : V;
  for (int64_t v = v0 + threadIdx.x; v < v1; v += kFoldThreads) {
    const int l = labels[v];
    if (l < kLabelSlots) acc[l][threadIdx.x] += (double)dose[v];
  }
  __syncthreads();
  reduce_label_columns(acc, part + (size_t)blockIdx.x * kLabelSlots);
}

__global__ void map_organ_final_kernel(const double* __restrict__ part, int n_blocks,
                                       const long long* __restrict__ count, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (l >= kLabelSlots) return;
  double s = 0.0;
  for (int b = lane; b < n_blocks; b += 32) s += part[(size_t)b * kLabelSlots + l];
  s = warp_sum_d(s);
  if (lane == 0) out[l] = count[l] > 0 ? s / (double)count[l] : 0.0;
}

__global__ void history_sigma_kernel(const ull* __restrict__ tsum, const ull* __restrict__ lo,
                                     const ull* __restrict__ hi, const float* __restrict__ density, int64_t V,
                                     double n, float gy_a, float* __restrict__ sigma) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const ull t = tsum[v];
    float sg = 0.0f;
    if (t) {
      const double s2 = (double)hi[v] * 18446744073709551616.0 + (double)lo[v];
      const double mean = (double)t / n;                   // units per history
      const double var = fmax(s2 / n - mean * mean, 0.0) / (n - 1.0);   // of the mean
      sg = sqrtf((float)var) * __fdiv_rn(gy_a, density[v]);
    }
    sigma[v] = sg;
  }
}

}  // namespace

cudaError_t launch_history_sigma(const ull* tsum, const ull* s2h_lo, const ull* s2h_hi, const float* density,
                                 int64_t V, double n_total, double gy_a, float* sigma, cudaStream_t s) {
  const int64_t g = (V + 255) / 256;
  history_sigma_kernel<<<(unsigned)(g < 8192 ? g : 8192), 256, 0, s>>>(tsum, s2h_lo, s2h_hi, density, V, n_total,
                                                                       (float)gy_a, sigma);
  return cudaGetLastError();
}

cudaError_t launch_map_organ_means(const float* dose, const uint8_t* labels, int64_t V, double* part,
                                   const long long* count, double* out, cudaStream_t s) {
  const int nb = fold_blocks(V);
  map_organ_kernel<<<nb, kFoldThreads, 0, s>>>(dose, labels, V, part);
  map_organ_final_kernel<<<(kLabelSlots + 3) / 4, 128, 0, s>>>(part, nb, count, out);
  return cudaGetLastError();
}

namespace {

// Statistics of two shards of one run (disjoint history ids): the exact
// tallies and counters add as integers, the 128-bit sums of squared history
// totals add with a carry, and the FP64 batch sums add because the batches of
// both shards are batches of the combined run.
__global__ void merge_stats_kernel(const MergeParams m) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < m.V; v += stride) {
    m.tsum[v] += m.o_tsum[v];
    m.s2[v] += m.o_s2[v];
    if (m.s2h_lo) {
      const ull lo = m.s2h_lo[v] + m.o_lo[v];
      m.s2h_hi[v] += m.o_hi[v] + (lo < m.o_lo[v] ? 1ull : 0ull);
      m.s2h_lo[v] = lo;
    }
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < kLabelSlots; i += blockDim.x) {
      m.org_s1[i] += m.o_org_s1[i];
      m.org_s2[i] += m.o_org_s2[i];
    }
    for (int i = threadIdx.x; i < kCtrCount; i += blockDim.x) m.counters[i] += m.o_counters[i];
  }
}

}  // namespace

cudaError_t launch_merge_stats(const MergeParams& m, int sms, cudaStream_t s) {
  const int64_t want = (m.V + 255) / 256;
  const int grid = (int)(want < 8LL * sms ? (want > 0 ? want : 1) : 8LL * sms);
  merge_stats_kernel<<<grid, 256, 0, s>>>(m);
  return cudaGetLastError();
}

namespace {

// Eq. 1 alone (no uncertainty, no organ sums): the dose rate the finalize
// pass writes, bit for bit (same FP64 mean, same FP32 conversion), streaming
// 16 bytes per voxel.
__global__ void dose_only_kernel(const ull* __restrict__ tsum, const float* __restrict__ density, int64_t V,
                                 double inv_n, float gy_a, float* __restrict__ dose) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
    const ull ti = tsum[v];
    float d = 0.0f;
    if (ti) {
      const double mean = (double)ti * inv_n;
      d = (float)mean * __fdiv_rn(gy_a, density[v]);
    }
    dose[v] = d;
  }
}

}  // namespace

cudaError_t launch_dose_only(const FinalizeParams& p, int sms, cudaStream_t s) {
  const int64_t want = (p.V + 255) / 256;
  const int grid = (int)(want < 8LL * sms ? (want > 0 ? want : 1) : 8LL * sms);
  dose_only_kernel<<<grid, 256, 0, s>>>(p.tsum, p.density, p.V, 1.0 / p.n_total,
                                        (float)(p.gy_per_unit_vol * p.activity_bq), p.dose);
  return cudaGetLastError();
}

int fold_blocks(int64_t V) { return (int)((V + kFoldTile - 1) / kFoldTile); }

cudaError_t launch_fold(const FoldParams& p, cudaStream_t s) {
  const int nb = fold_blocks(p.V);
  fold_kernel<<<nb, kFoldThreads, 0, s>>>(p);
  if (p.labels) fold_organs_kernel<<<(kLabelSlots + 3) / 4, 128, 0, s>>>(p, nb);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t s) {
  const int nb = fold_blocks(p.V);
  const size_t smem = 2 * kLabelSlots * kFoldThreads * sizeof(double);
  // per call: cheap, and correct for every device and calling thread
  cudaError_t e = cudaFuncSetAttribute(finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  finalize_kernel<<<nb, kFoldThreads, smem, s>>>(p);
  if (p.labels) finalize_organs_kernel<<<(kLabelSlots + 3) / 4, 128, 0, s>>>(p, nb);
  return cudaGetLastError();
}

}  // namespace nm

// ---------------------------------------------------------------------------
// Multi-time-point dosimetry: time-integrated activity per voxel.
// ---------------------------------------------------------------------------
namespace nm {
namespace {

constexpr int kMaxTimePoints = 16;

struct TimeIntegralArgs {
  const float* act[kMaxTimePoints];   // activity maps (Bq per voxel)
  double t[kMaxTimePoints];           // their times, seconds
  int n;
};

// Per voxel, in FP64: A_0 t_0 / 2 (linear uptake from zero), the trapezoids
// between time points, and A_n / lambda after the last one (physical decay,
// tail_s = 1 / lambda); the FP64 sum of a CTA's results goes to
// block_sums[block] (fixed tree).  A negative or non-finite activity sets
// NM_DEV_BAD_ACTIVITY.
__global__ void __launch_bounds__(256) time_integral_kernel(const TimeIntegralArgs a, int64_t V, double tail_s,
                                                            float* __restrict__ out, double* __restrict__ block_sums,
                                                            uint32_t* __restrict__ status) {
  __shared__ double red[256];
  double acc = 0.0;
  bool bad = false;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    double prev = (double)a.act[0][v];
    bad |= !(prev >= 0.0) || isinf(prev);
    double s = 0.5 * prev * a.t[0];
    for (int k = 1; k < a.n; ++k) {
      const double cur = (double)a.act[k][v];
      bad |= !(cur >= 0.0) || isinf(cur);
      s += 0.5 * (prev + cur) * (a.t[k] - a.t[k - 1]);
      prev = cur;
    }
    s += prev * tail_s;
    out[v] = (float)s;
    acc += s;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = red[0];
  if (bad) atomicOr(status, (uint32_t)NM_DEV_BAD_ACTIVITY);
}

}  // namespace

cudaError_t launch_time_integral(const float* const* act, const double* t_s, int n, int64_t V, double tail_s,
                                 float* out, double* block_sums, int blocks, cudaStream_t s) {
  if (n < 1 || n > kMaxTimePoints || blocks < 1) return cudaErrorInvalidValue;
  TimeIntegralArgs a;
  for (int k = 0; k < kMaxTimePoints; ++k) {
    a.act[k] = k < n ? act[k] : nullptr;
    a.t[k] = k < n ? t_s[k] : 0.0;
  }
  a.n = n;
  // the status word follows the block sums
  time_integral_kernel<<<blocks, 256, 0, s>>>(a, V, tail_s, out, block_sums,
                                              reinterpret_cast<uint32_t*>(block_sums + blocks));
  return cudaGetLastError();
}

}  // namespace nm
