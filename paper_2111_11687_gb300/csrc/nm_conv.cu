// 3x3x3 convolution (stride 1, zero padding 1) of channels-last BF16 volumes
// on the 5th-generation tensor cores, for the dose denoiser.
//
// Forward and input-gradient passes are one implicit GEMM,
//   Y[p, co] = sum_k A[p, k] W[co, k],  A[p, k] = X[p + offset(tap), ci],  k = tap * Cin + ci,
// with M = voxels (128 per CTA tile), N = Cout, K = 27 Cin padded to 64.  The
// weight gradient is the GEMM dW[co, k] = sum_p A[p, k] dY[p, co] with the
// voxels as reduction dimension, split over CTAs and summed in a fixed order.
//
// Operands are gathered by all threads into shared memory in the tensor
// cores' canonical no-swizzle layout (8x16-byte core matrices), one thread
// issues tcgen05.mma into a tensor-memory accumulator and commits to an
// mbarrier; two stage buffers let the gather of stage s+1 overlap the MMAs of
// stage s.  Every wait is bounded: on time-out the CTA records NM_DEV_TIMEOUT,
// drains what it issued (bounded again), frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdlib>

#include <algorithm>

#include "nm_internal.cuh"
#include "nm_tc.cuh"

namespace nm {
namespace {

constexpr int kBM = 128;        // GEMM rows per CTA
constexpr int kKS = 64;         // K elements per stage (4 MMAs of K = 16)
constexpr int kThreads = 128;
constexpr long long kWaitCycles = 4ll << 30;  // about 2 s at 2 GHz

struct ConvGeom {
  int n, d, h, w;               // output grid (fine)
  int c0, c1, cin, cout, kpad;  // channels; kpad = K padded to a multiple of 64
  int coarse;                   // source 0 is at half resolution (nearest upsampling)
  long long m;                  // voxels = n*d*h*w
};

// Per-voxel part of the im2col gather, computed once per GEMM row: element
// offsets of the voxel in both sources, which of its 27 neighbours lie inside
// the volume, and (half-resolution source) its parities.
struct Row {
  long long off0, off1;
  uint32_t vmask;     // bit t: the neighbour at tap t is inside the volume
  int pz, py, px;     // parities of z, y, x (nearest-upsampled source)
};

__device__ __forceinline__ Row make_row(const ConvGeom& g, long long m) {
  Row r;
  const int x = (int)(m % g.w);
  long long t = m / g.w;
  const int y = (int)(t % g.h);
  t /= g.h;
  const int z = (int)(t % g.d);
  const int b = (int)(t / g.d);
  if (g.coarse) {
    const int dd = g.d >> 1, hh = g.h >> 1, ww = g.w >> 1;
    r.off0 = ((((long long)b * dd + (z >> 1)) * hh + (y >> 1)) * ww + (x >> 1)) * g.c0;
  } else {
    r.off0 = m * g.c0;
  }
  r.off1 = m * g.c1;
  r.pz = z & 1; r.py = y & 1; r.px = x & 1;
  // neighbours inside the volume: axis masks over d in {-1, 0, +1}
  const uint32_t mz = (z > 0 ? 1u : 0u) | 2u | (z < g.d - 1 ? 4u : 0u);
  const uint32_t my = (y > 0 ? 1u : 0u) | 2u | (y < g.h - 1 ? 4u : 0u);
  const uint32_t mx = (x > 0 ? 1u : 0u) | 2u | (x < g.w - 1 ? 4u : 0u);
  uint32_t vm = 1u << 30;  // the row is a voxel of the volume
#pragma unroll
  for (int t2 = 0; t2 < 27; ++t2)
    if (((mz >> (t2 / 9)) & 1u) && ((my >> ((t2 / 3) % 3)) & 1u) && ((mx >> (t2 % 3)) & 1u)) vm |= 1u << t2;
  r.vmask = vm;
  return r;
}

// Column table entry for each 8-wide chunk of K: tap (bits 0-4, 31 = past the
// taps), the tap's axis indices dz+1, dy+1, dx+1 (2 bits each from bit 5) and
// the channel (bits 16-31).
__device__ __forceinline__ uint32_t kchunk_entry(const ConvGeom& g, int k, bool bias_row) {
  const int tap = k / g.cin;
  if (bias_row && k == 27 * g.cin) return 30u;  // (1, 0, ..., 0): the bias-gradient row
  if (tap >= 27) return 31u;
  const int ci = k - tap * g.cin;
  return (uint32_t)tap | ((uint32_t)(tap / 9) << 5) | ((uint32_t)((tap / 3) % 3) << 7) |
         ((uint32_t)(tap % 3) << 9) | ((uint32_t)ci << 16);
}

// Element offset of tap t relative to the voxel, per source (full resolution).
__device__ __forceinline__ int tap_delta(const ConvGeom& g, int t, int c) {
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  return ((dz * g.h + dy) * g.w + dx) * c;
}

// 8 consecutive channels (16 bytes) of the im2col row r at the chunk with
// table entry e, or zeros outside the volume / past 27 taps.
__device__ __forceinline__ uint4 gather8(const ConvGeom& g, const __nv_bfloat16* __restrict__ x0,
                                         const __nv_bfloat16* __restrict__ x1, const Row& r, uint32_t e,
                                         const int* __restrict__ s_d0, const int* __restrict__ s_d1) {
  const int tap = e & 31u;
  if (tap == 30) return make_uint4((r.vmask >> 30) & 1u ? 0x3F80u : 0u, 0, 0, 0);  // BF16 1.0 in a valid row
  if (tap >= 27 || !((r.vmask >> tap) & 1u)) return make_uint4(0, 0, 0, 0);
  const int ci = (int)(e >> 16);
  if (ci < g.c0) {
    if (!g.coarse) return __ldg(reinterpret_cast<const uint4*>(x0 + r.off0 + s_d0[tap] + ci));
    // nearest upsampling: a step of -1 moves to the previous coarse voxel only
    // from an even coordinate, a step of +1 to the next one only from an odd one
    const int az = (int)((e >> 5) & 3u), ay = (int)((e >> 7) & 3u), ax = (int)((e >> 9) & 3u);
    const int cz = az == 0 ? -(r.pz ^ 1) : (az == 2 ? r.pz : 0);
    const int cy = ay == 0 ? -(r.py ^ 1) : (ay == 2 ? r.py : 0);
    const int cx = ax == 0 ? -(r.px ^ 1) : (ax == 2 ? r.px : 0);
    const long long off = r.off0 + ((long long)(cz * (g.h >> 1) + cy) * (g.w >> 1) + cx) * g.c0 + ci;
    return __ldg(reinterpret_cast<const uint4*>(x0 + off));
  }
  return __ldg(reinterpret_cast<const uint4*>(x1 + r.off1 + s_d1[tap] + (ci - g.c0)));
}

// Tables shared by a CTA: chunk entries for all of K, tap deltas per source.
struct GatherTables {
  uint32_t* ktab;  // [kpad / 8]
  int d0[27], d1[27];
};

__device__ __forceinline__ void fill_tables(const ConvGeom& g, uint32_t* ktab, int* d0, int* d1, bool bias_row) {
  for (int i = threadIdx.x; i < g.kpad / 8; i += blockDim.x) ktab[i] = kchunk_entry(g, i * 8, bias_row);
  for (int t = threadIdx.x; t < 27; t += blockDim.x) {
    d0[t] = tap_delta(g, t, g.c0);
    d1[t] = tap_delta(g, t, g.c1);
  }
}

// ---------------------------------------------------------------------------
// Forward / input-gradient: Y = act(A W^T + bias), K-major A and B.
// ---------------------------------------------------------------------------
template <int COUT>
__global__ void __launch_bounds__(kThreads) conv_fwd_kernel(ConvGeom g, const __nv_bfloat16* __restrict__ x0,
                                                            const __nv_bfloat16* __restrict__ x1,
                                                            const __nv_bfloat16* __restrict__ wt,
                                                            const float* __restrict__ bias,
                                                            __nv_bfloat16* __restrict__ y, int relu,
                                                            float* __restrict__ part, int stages_per_split,
                                                            uint32_t* status) {
  constexpr int kNcols = COUT <= 32 ? 32 : COUT <= 64 ? 64 : COUT <= 128 ? 128 : 256;
  constexpr uint32_t kABytes = kBM * kKS * 2;       // 16 KB
  constexpr uint32_t kBBytes = COUT * kKS * 2;
  constexpr uint32_t kSbo = (kKS / 8) * 128;        // 8-row groups are 1 KB apart
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sa = smem;                                // [2][kABytes]
  uint8_t* sb = smem + 2 * kABytes;                  // [2][kBBytes]
  uint32_t* ktab = reinterpret_cast<uint32_t*>(smem + 2 * kABytes + 2 * kBBytes);  // [kpad / 8]
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_d0[27], s_d1[27];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  fill_tables(g, ktab, s_d0, s_d1, false);
  if (warp == 0) tc::tmem_alloc(&s_tmem, kNcols);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  const long long m_row = (long long)blockIdx.x * kBM + tid;  // this thread gathers GEMM row tid
  const bool row_ok = m_row < g.m;
  Row row;
  if (row_ok) row = make_row(g, m_row);
  else row.vmask = 0u;
  // split K: this CTA takes stages [s0, s0 + nstages) of the GEMM depth
  const int s0 = blockIdx.y * stages_per_split;
  int nstages = g.kpad / kKS - s0;
  if (nstages > stages_per_split) nstages = stages_per_split;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, COUT, false, false);
  bool timeout = false;
  int issued = 0;  // stages whose MMAs were issued

  for (int s = 0; s < nstages; ++s) {
    const int buf = s & 1;
    const int sg = s0 + s;
    if (s >= 2 && !tc::mbar_wait_bounded(&bar[buf], ((s >> 1) - 1) & 1, kWaitCycles)) timeout = true;
    if (__syncthreads_or(timeout)) { timeout = true; break; }
    uint8_t* a = sa + buf * kABytes;
    uint8_t* bm = sb + buf * kBBytes;
    // A: this thread's row, 8 chunks of 8 channels.
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
      const uint4 v = gather8(g, x0, x1, row, ktab[sg * (kKS / 8) + kc], s_d0, s_d1);
      *reinterpret_cast<uint4*>(a + (tid >> 3) * kSbo + kc * 128 + (tid & 7) * 16) = v;
    }
    // B: COUT rows x 8 chunks of the weight matrix [Cout][kpad].
#pragma unroll
    for (int i = 0; i < COUT / 16; ++i) {
      const int q = tid + kThreads * i;
      const int r = q >> 3, kc = q & 7;
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(wt + (long long)r * g.kpad + sg * kKS + kc * 8));
      *reinterpret_cast<uint4*>(bm + (r >> 3) * kSbo + kc * 128 + (r & 7) * 16) = v;
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(a), b0 = tc::smem_u32(bm);
#pragma unroll
      for (int kk = 0; kk < kKS / 16; ++kk)
        tc::mma_bf16(tmem, tc::smem_desc(a0 + kk * 256, 128, kSbo), tc::smem_desc(b0 + kk * 256, 128, kSbo),
                     idesc, (s | kk) != 0);
      tc::mma_commit(&bar[buf]);
    }
    issued = s + 1;
  }
  if (!timeout && issued > 0) {
    const int last = issued - 1;
    if (!tc::mbar_wait_bounded(&bar[last & 1], (last >> 1) & 1, kWaitCycles)) timeout = true;
  }
  timeout = __syncthreads_or(timeout);
  if (timeout) {
    if (tid == 0) atomicOr(status, NM_DEV_TIMEOUT);
    // drain: the last issued commit covers every MMA this CTA issued
    if (issued > 0) tc::mbar_wait_bounded(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kWaitCycles);
  } else {
    tc::fence_after_sync();
    const int row = warp * 32 + lane;
    const long long m = (long long)blockIdx.x * kBM + row;
#pragma unroll
    for (int c = 0; c < COUT / 16; ++c) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c * 16, v);
      if (m < g.m && part) {
        float* dst = part + ((long long)blockIdx.y * g.m + m) * COUT + c * 16;
#pragma unroll
        for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      } else if (m < g.m) {
        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float t = v[j] + (bias ? __ldg(bias + c * 16 + j) : 0.0f);
          if (relu) t = fmaxf(t, 0.0f);
          o[j] = __float2bfloat16_rn(t);
        }
        uint4* dst = reinterpret_cast<uint4*>(y + m * COUT + c * 16);
        dst[0] = reinterpret_cast<uint4*>(o)[0];
        dst[1] = reinterpret_cast<uint4*>(o)[1];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kNcols);
}

// ---------------------------------------------------------------------------
// Weight gradient: D[k, co] = sum_p A[p, k] dY[p, co] over this CTA's voxel
// range; rows k are MN-contiguous in the gathered data, so both operands are
// staged MN-major.  Partial results go to part[split][kpad][Cout].
// ---------------------------------------------------------------------------
template <int COUT>
__global__ void __launch_bounds__(kThreads) conv_wgrad_kernel(ConvGeom g, const __nv_bfloat16* __restrict__ x0,
                                                              const __nv_bfloat16* __restrict__ x1,
                                                              const __nv_bfloat16* __restrict__ dy,
                                                              float* __restrict__ part, long long vox_per_split,
                                                              uint32_t* status) {
  constexpr int kNcols = COUT < 32 ? 32 : COUT;
  constexpr uint32_t kABytes = kBM * kKS * 2;
  constexpr uint32_t kBBytes = COUT * kKS * 2;
  constexpr uint32_t kSboA = (kBM / 8) * 128;       // distance of K-adjacent core matrices of A
  constexpr uint32_t kSboB = (COUT / 8) * 128;      // ... and of B
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sa = smem;
  uint8_t* sb = smem + 2 * kABytes;
  uint32_t* ktab = reinterpret_cast<uint32_t*>(smem + 2 * kABytes + 2 * kBBytes);  // [kpad / 8]
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_d0[27], s_d1[27];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  fill_tables(g, ktab, s_d0, s_d1, true);
  if (warp == 0) tc::tmem_alloc(&s_tmem, kNcols);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  const int k0 = blockIdx.x * kBM;                 // GEMM row block (im2col columns)
  const long long p_begin = (long long)blockIdx.y * vox_per_split;
  long long p_end = p_begin + vox_per_split;
  if (p_end > g.m) p_end = g.m;
  const int nstages = p_begin < p_end ? (int)((p_end - p_begin + kKS - 1) / kKS) : 0;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, COUT, true, true);
  bool timeout = false;
  int issued = 0;

  for (int s = 0; s < nstages; ++s) {
    const int buf = s & 1;
    if (s >= 2 && !tc::mbar_wait_bounded(&bar[buf], ((s >> 1) - 1) & 1, kWaitCycles)) timeout = true;
    if (__syncthreads_or(timeout)) { timeout = true; break; }
    uint8_t* a = sa + buf * kABytes;
    uint8_t* bm = sb + buf * kBBytes;
    // A: 64 voxels x 16 chunks (8 GEMM rows each); a thread owns one voxel
    // (tid % 64) and every other chunk.
    {
      const int pl = tid & 63;
      const long long p = p_begin + s * kKS + pl;
      Row row;
      if (p < p_end) row = make_row(g, p);
      else row.vmask = 0u;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int rc = 2 * i + (tid >> 6);
        const uint4 v = gather8(g, x0, x1, row, ktab[(k0 >> 3) + rc], s_d0, s_d1);
        *reinterpret_cast<uint4*>(a + rc * 128 + (pl >> 3) * kSboA + (pl & 7) * 16) = v;
      }
    }
    // B: 64 voxels x COUT/8 chunks of dY.
    for (int q = tid; q < kKS * (COUT / 8); q += kThreads) {
      const int pl = q / (COUT / 8), rc = q % (COUT / 8);
      const long long p = p_begin + s * kKS + pl;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (p < p_end) v = __ldg(reinterpret_cast<const uint4*>(dy + p * COUT + rc * 8));
      *reinterpret_cast<uint4*>(bm + rc * 128 + (pl >> 3) * kSboB + (pl & 7) * 16) = v;
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(a), b0 = tc::smem_u32(bm);
#pragma unroll
      for (int kk = 0; kk < kKS / 16; ++kk)
        // MN-major, no swizzle: the leading byte offset steps along K (8 voxels),
        // the stride byte offset along MN (8 rows).
        tc::mma_bf16(tmem, tc::smem_desc(a0 + kk * 2 * kSboA, kSboA, 128),
                     tc::smem_desc(b0 + kk * 2 * kSboB, kSboB, 128), idesc, (s | kk) != 0);
      tc::mma_commit(&bar[buf]);
    }
    issued = s + 1;
  }
  if (!timeout && issued > 0) {
    const int last = issued - 1;
    if (!tc::mbar_wait_bounded(&bar[last & 1], (last >> 1) & 1, kWaitCycles)) timeout = true;
  }
  timeout = __syncthreads_or(timeout);
  const int row = warp * 32 + lane;
  float* dst = part + ((long long)blockIdx.y * g.kpad + k0 + row) * COUT;
  if (timeout) {
    if (tid == 0) atomicOr(status, NM_DEV_TIMEOUT);
    if (issued > 0) tc::mbar_wait_bounded(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kWaitCycles);
  } else if (issued == 0) {
    for (int c = 0; c < COUT; ++c) dst[c] = 0.0f;
  } else {
    tc::fence_after_sync();
#pragma unroll
    for (int c = 0; c < COUT / 16; ++c) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c * 16, v);
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(dst + c * 16 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kNcols);
}

// dW[co][k] = sum over splits (in order) of part[split][k][co]; row 27*cin
// carries the bias gradient (its A row is all ones), the padding stays zero.
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int splits, int kpad, int kreal,
                                    int cout, float* __restrict__ dw, float* __restrict__ db) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)kpad * cout) return;
  const int k = (int)(i / cout), co = (int)(i % cout);
  float s = 0.0f;
  for (int t = 0; t < splits; ++t) s += part[((long long)t * kpad + k) * cout + co];
  if (k == kreal && db) db[co] = s;
  dw[(long long)co * kpad + k] = k < kreal ? s : 0.0f;
}

// Weights of the input-gradient convolution: the forward weights [Cout][kpad(Cin)]
// with the taps reversed and the channel roles swapped, [Cin][kpad(Cout)].
__global__ void flip_weights_kernel(const __nv_bfloat16* __restrict__ w, int cin, int cout, int kpad_f,
                                    int kpad_b, __nv_bfloat16* __restrict__ wb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)cin * kpad_b) return;
  const int ci = (int)(i / kpad_b), k = (int)(i % kpad_b);
  const int tap = k / cout, co = k % cout;
  __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
  if (tap < 27) v = w[(long long)co * kpad_f + (26 - tap) * cin + ci];
  wb[i] = v;
}

// y = act(sum over splits of part + bias) for split-K forward convolutions.
__global__ void split_finish_kernel(const float* __restrict__ part, int splits, long long m, int cout,
                                    const float* __restrict__ bias, int relu, __nv_bfloat16* __restrict__ y) {
  const long long n = m * cout;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float t = bias ? bias[i % cout] : 0.0f;
    for (int k = 0; k < splits; ++k) t += part[(long long)k * n + i];
    if (relu) t = fmaxf(t, 0.0f);
    y[i] = __float2bfloat16_rn(t);
  }
}

template <int COUT>
size_t fwd_smem_base() { return 2 * (size_t)kBM * kKS * 2 + 2 * (size_t)COUT * kKS * 2; }

// stage buffers plus the K-chunk table
template <int COUT>
size_t fwd_smem(int kpad) { return fwd_smem_base<COUT>() + (size_t)(kpad / 8) * 4; }

template <int COUT>
cudaError_t launch_fwd_t(const ConvGeom& g, const __nv_bfloat16* x0, const __nv_bfloat16* x1,
                         const __nv_bfloat16* w, const float* bias, __nv_bfloat16* y, int relu,
                         uint32_t* status, cudaStream_t s) {
  const size_t smem = fwd_smem<COUT>(g.kpad);
  cudaError_t e = cudaFuncSetAttribute(conv_fwd_kernel<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long grid = (g.m + kBM - 1) / kBM;
  // Few row tiles and a deep K: split K over CTAs so that every SM has work.
  const int nst = g.kpad / kKS;
  int splits = 1;
  if (grid < 2 * 152) {
    splits = (int)((2 * 152 + grid - 1) / grid);
    if (splits > nst / 4) splits = nst / 4 > 1 ? nst / 4 : 1;
  }
  const int per = (nst + splits - 1) / splits;
  splits = (nst + per - 1) / per;
  if (splits == 1) {
    conv_fwd_kernel<COUT><<<(unsigned)grid, kThreads, smem, s>>>(g, x0, x1, w, bias, y, relu, nullptr, per, status);
    return cudaGetLastError();
  }
  float* part = nullptr;
  if ((e = cudaMallocAsync((void**)&part, (size_t)splits * g.m * COUT * sizeof(float), s))) return e;
  conv_fwd_kernel<COUT><<<dim3((unsigned)grid, splits), kThreads, smem, s>>>(g, x0, x1, w, bias, y, relu, part, per,
                                                                           status);
  const long long n = g.m * COUT;
  split_finish_kernel<<<(unsigned)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192), 256, 0, s>>>(
      part, splits, g.m, COUT, bias, relu, y);
  e = cudaGetLastError();
  cudaFreeAsync(part, s);
  return e;
}

// The weight-gradient buffers are over-allocated to 96 KB: every read the
// MMAs can make from the stage buffers stays inside the CTA's allocation.
template <int COUT>
size_t wgrad_smem(int kpad) {
  const size_t need = fwd_smem_base<COUT>() > 96 * 1024 ? fwd_smem_base<COUT>() : 96 * 1024;
  return need + (size_t)(kpad / 8) * 4;
}

template <int COUT>
cudaError_t launch_wgrad_t(const ConvGeom& g, const __nv_bfloat16* x0, const __nv_bfloat16* x1,
                           const __nv_bfloat16* dy, float* part, int splits, uint32_t* status,
                           cudaStream_t s) {
  const size_t smem = wgrad_smem<COUT>(g.kpad);
  cudaError_t e = cudaFuncSetAttribute(conv_wgrad_kernel<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long per = ((g.m + splits - 1) / splits + kKS - 1) / kKS * kKS;
  dim3 grid(g.kpad / kBM, splits);
  conv_wgrad_kernel<COUT><<<grid, kThreads, smem, s>>>(g, x0, x1, dy, part, per, status);
  return cudaGetLastError();
}

}  // namespace

int conv_kpad(int cin) {
  // the weight-gradient GEMM tiles K in rows of 128 and uses row 27*cin (a
  // padding row, so there is always one) for the bias gradient
  const int k = 27 * cin + 1;
  return (k + 127) / 128 * 128;
}

bool conv_geom_ok(const nm_conv3d_desc& d) {
  const int cin = d.c0 + d.c1;
  if (d.n <= 0 || d.d <= 0 || d.h <= 0 || d.w <= 0) return false;
  if (d.c0 <= 0 || d.c0 % 8 || d.c1 < 0 || d.c1 % 8 || cin > 512) return false;
  if (!(d.cout == 16 || d.cout == 32 || d.cout == 48 || d.cout == 64 || d.cout == 96 || d.cout == 128 ||
        d.cout == 192))
    return false;
  if (d.src0_coarse && (d.d % 2 || d.h % 2 || d.w % 2)) return false;
  return true;
}

static ConvGeom make_geom(const nm_conv3d_desc& d) {
  ConvGeom g;
  g.n = d.n; g.d = d.d; g.h = d.h; g.w = d.w;
  g.c0 = d.c0; g.c1 = d.c1; g.cin = d.c0 + d.c1; g.cout = d.cout;
  g.kpad = conv_kpad(g.cin);
  g.coarse = d.src0_coarse;
  g.m = (long long)d.n * d.d * d.h * d.w;
  return g;
}

cudaError_t conv3d_fwd(const nm_conv3d_desc& d, const void* x0, const void* x1, const void* w,
                       const float* bias, void* y, int relu, uint32_t* status, cudaStream_t s) {
  // Single-source convolutions with few output channels take the shifted-window
  // kernel (no im2col gather); NM_CONV_GATHER=1 forces the gather kernel.
  const char* force = getenv("NM_CONV_GATHER");
  if (conv_tile_ok(d) && !(force && force[0] == '1')) return conv3d_fwd_tile(d, x0, w, bias, y, relu, status, s);
  const ConvGeom g = make_geom(d);
  auto X0 = (const __nv_bfloat16*)x0, X1 = (const __nv_bfloat16*)x1, W = (const __nv_bfloat16*)w;
  auto Y = (__nv_bfloat16*)y;
  switch (d.cout) {
    case 16: return launch_fwd_t<16>(g, X0, X1, W, bias, Y, relu, status, s);
    case 32: return launch_fwd_t<32>(g, X0, X1, W, bias, Y, relu, status, s);
    case 48: return launch_fwd_t<48>(g, X0, X1, W, bias, Y, relu, status, s);
    case 64: return launch_fwd_t<64>(g, X0, X1, W, bias, Y, relu, status, s);
    case 96: return launch_fwd_t<96>(g, X0, X1, W, bias, Y, relu, status, s);
    case 128: return launch_fwd_t<128>(g, X0, X1, W, bias, Y, relu, status, s);
    case 192: return launch_fwd_t<192>(g, X0, X1, W, bias, Y, relu, status, s);
    default: return cudaErrorInvalidValue;
  }
}

int conv_wgrad_splits(const nm_conv3d_desc& d) {
  const long long m = (long long)d.n * d.d * d.h * d.w;
  const int mtiles = conv_kpad(d.c0 + d.c1) / kBM;
  // about four CTAs per SM of 152 in total, at least 64 voxels each
  long long splits = (4 * 152 + mtiles - 1) / mtiles;
  if (splits * 64 > m) splits = (m + 63) / 64;
  return (int)(splits < 1 ? 1 : splits);
}

size_t conv_wgrad_workspace(const nm_conv3d_desc& d) {
  const size_t gather = (size_t)conv_wgrad_splits(d) * conv_kpad(d.c0 + d.c1) * d.cout * sizeof(float);
  return conv_wgrad_tile_ok(d) ? std::max(gather, conv_wgrad_tile_workspace(d)) : gather;
}

cudaError_t conv3d_flip_weights(const nm_conv3d_desc& d, const void* w, void* wb, cudaStream_t s) {
  const int cin = d.c0 + d.c1;
  const int kf = conv_kpad(cin), kb = conv_kpad(d.cout);
  const long long n = (long long)cin * kb;
  flip_weights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const __nv_bfloat16*)w, cin, d.cout, kf, kb,
                                                                   (__nv_bfloat16*)wb);
  return cudaGetLastError();
}

cudaError_t conv3d_wgrad(const nm_conv3d_desc& d, const void* x0, const void* x1, const void* dy,
                         float* dw, float* db, void* workspace, uint32_t* status, cudaStream_t s) {
  // Single-source layers with 16 or 32 outputs take the shifted-window kernel;
  // NM_CONV_GATHER=1 forces the gather kernel.
  const char* force = getenv("NM_CONV_GATHER");
  if (conv_wgrad_tile_ok(d) && !(force && force[0] == '1'))
    return conv3d_wgrad_tile(d, x0, dy, dw, db, workspace, status, s);
  const ConvGeom g = make_geom(d);
  const int splits = conv_wgrad_splits(d);
  float* part = (float*)workspace;
  auto X0 = (const __nv_bfloat16*)x0, X1 = (const __nv_bfloat16*)x1, DY = (const __nv_bfloat16*)dy;
  cudaError_t e;
  switch (d.cout) {
    case 16: e = launch_wgrad_t<16>(g, X0, X1, DY, part, splits, status, s); break;
    case 32: e = launch_wgrad_t<32>(g, X0, X1, DY, part, splits, status, s); break;
    case 64: e = launch_wgrad_t<64>(g, X0, X1, DY, part, splits, status, s); break;
    case 128: e = launch_wgrad_t<128>(g, X0, X1, DY, part, splits, status, s); break;
    default: return cudaErrorInvalidValue;  // weight gradients exist for the U-Net's outputs only
  }
  if (e != cudaSuccess) return e;
  const long long n = (long long)g.kpad * g.cout;
  wgrad_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, splits, g.kpad, 27 * g.cin, g.cout, dw, db);
  return cudaGetLastError();
}

}  // namespace nm
