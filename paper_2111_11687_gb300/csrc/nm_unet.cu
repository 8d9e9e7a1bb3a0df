// The dose denoiser: a 3D U-Net on BF16 channels-last volumes whose 3x3x3
// convolutions run on the tensor cores (nm_conv.cu), trained with Adam on FP32
// master weights.  Not part of the paper; it maps a low-count dose map plus
// density and activity to a high-count one.
//
// Architecture (levels L, widths w_i = base * 2^i): per level two 3x3x3
// convolutions with ReLU; 2x2x2 average pooling down; on the way up nearest
// upsampling of the coarser output concatenated with the level's skip
// (read directly by the convolution, never materialised), two convolutions
// with ReLU; a 1x1x1 head whose output is added to input channel 0.
//
// Input channels (8, of which 4 used): 0 = low-count dose / s, 1 = density,
// 2 = activity / a, 3 = activity / (a max(density, 0.1)); the target is the
// high-count dose / s (s, a: body means of the low-count dose and activity).
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "nm_internal.cuh"
#include "nm_trace.h"

using namespace nm;

namespace {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// Elementwise and reduction kernels.
// ---------------------------------------------------------------------------
// Volumes are [n][d][h][w][c] with d, h, w even; the coarse level is half of each.
__global__ void avgpool_kernel(const bf16* __restrict__ x, int n, int d, int h, int w, int c,
                               bf16* __restrict__ y) {
  // one thread per output voxel and 8-channel octet (16-byte loads and
  // store), each channel summed over the 2x2x2 block in the same order;
  // 32-bit indices (callers keep the element count below 2^32)
  const unsigned d2 = d >> 1, h2 = h >> 1, w2 = w >> 1, q = c / 8;
  const unsigned total = (unsigned)n * d2 * h2 * w2 * q;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const unsigned j = i % q, v = i / q;
    const unsigned xx = v % w2, r = v / w2, yy = r % h2, r2 = r / h2, zz = r2 % d2, b = r2 / d2;
    float sum[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) sum[e] = 0.0f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const size_t src = (((size_t)b * d + 2 * zz + dz) * h + 2 * yy + dy) * w + 2 * xx + dx;
          const uint4 u = *reinterpret_cast<const uint4*>(x + src * c + j * 8);
          const __nv_bfloat162* e2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(e2[e]);
            sum[2 * e] += f.x;
            sum[2 * e + 1] += f.y;
          }
        }
    uint4 o;
    __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int e = 0; e < 4; ++e) o2[e] = __floats2bfloat162_rn(sum[2 * e] * 0.125f, sum[2 * e + 1] * 0.125f);
    *reinterpret_cast<uint4*>(y + (size_t)v * c + j * 8) = o;
  }
}

// cat[v] = [coarse[parent(v)] (c0 channels) | skip[v] (c1 channels)], 16 bytes at a time.
__global__ void upsample_concat_kernel(const bf16* __restrict__ coarse, const bf16* __restrict__ skip, int n, int d,
                                       int h, int w, int c0, int c1, bf16* __restrict__ cat) {
  // 32-bit index arithmetic: callers keep n d h w (c0 + c1) / 8 below 2^32
  const unsigned h2 = h >> 1, w2 = w >> 1, c = c0 + c1, q = c / 8;
  const unsigned total = (unsigned)n * d * h * w * q;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const unsigned j = i % q, v = i / q;
    uint4 val;
    if (j * 8 < (unsigned)c0) {
      const unsigned xx = v % w, r = v / w, yy = r % h, r2 = r / h, zz = r2 % d, b = r2 / d;
      const unsigned pv = ((b * (d >> 1) + (zz >> 1)) * h2 + (yy >> 1)) * w2 + (xx >> 1);
      val = *reinterpret_cast<const uint4*>(coarse + (size_t)pv * c0 + j * 8);
    } else {
      val = *reinterpret_cast<const uint4*>(skip + (size_t)v * c1 + (j * 8 - c0));
    }
    *reinterpret_cast<uint4*>(cat + (size_t)v * c + j * 8) = val;
  }
}

// g *= (act > 0), 8 elements (16 bytes) per thread; n is a multiple of 8
__global__ void relu_mask_kernel(bf16* __restrict__ g, const bf16* __restrict__ act, long long n) {
  const unsigned n8 = (unsigned)(n / 8);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += gridDim.x * blockDim.x) {
    uint4 gv = reinterpret_cast<const uint4*>(g)[i];
    const uint4 av = reinterpret_cast<const uint4*>(act)[i];
    bf16* ge = reinterpret_cast<bf16*>(&gv);
    const bf16* ae = reinterpret_cast<const bf16*>(&av);
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (!(__bfloat162float(ae[e]) > 0.0f)) ge[e] = __float2bfloat16_rn(0.0f);
    reinterpret_cast<uint4*>(g)[i] = gv;
  }
}

// Gradient of a decoder input [n][s]^3[c0 + c1] split into the coarse source
// (summed over its 8 children, times the coarse activation's ReLU mask) and
// the skip source (copied); 8 channels (16 bytes) per thread, c0 and c1
// multiples of 8.
__global__ void split_concat_grad_kernel(const bf16* __restrict__ dx, int n, int d, int h, int w, int c0, int c1,
                                         const bf16* __restrict__ coarse_act, bf16* __restrict__ g_coarse,
                                         bf16* __restrict__ g_skip) {
  // 32-bit index arithmetic (training volumes hold far fewer than 2^32 elements)
  const unsigned d2 = d >> 1, h2 = h >> 1, w2 = w >> 1, c = c0 + c1, q0 = c0 / 8, q1 = c1 / 8;
  const unsigned nc = (unsigned)n * d2 * h2 * w2 * q0;
  const unsigned ns = (unsigned)n * d * h * w * q1;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nc + ns; i += gridDim.x * blockDim.x) {
    if (i < nc) {
      const unsigned j = i % q0, v = i / q0;
      const unsigned xx = v % w2, r = v / w2, yy = r % h2, r2 = r / h2, zz = r2 % d2, b = r2 / d2;
      float sum[8] = {};
      for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
          for (int dx2 = 0; dx2 < 2; ++dx2) {
            const uint4 u = *reinterpret_cast<const uint4*>(
                dx + ((((size_t)b * d + 2 * zz + dz) * h + 2 * yy + dy) * w + 2 * xx + dx2) * c + j * 8);
            const bf16* e = reinterpret_cast<const bf16*>(&u);
#pragma unroll
            for (int k = 0; k < 8; ++k) sum[k] += __bfloat162float(e[k]);
          }
      const uint4 av = *reinterpret_cast<const uint4*>(coarse_act + (size_t)i * 8);
      const bf16* ae = reinterpret_cast<const bf16*>(&av);
      uint4 o;
      bf16* oe = reinterpret_cast<bf16*>(&o);
#pragma unroll
      for (int k = 0; k < 8; ++k) oe[k] = __float2bfloat16_rn(__bfloat162float(ae[k]) > 0.0f ? sum[k] : 0.0f);
      *reinterpret_cast<uint4*>(g_coarse + (size_t)i * 8) = o;
    } else {
      const unsigned j = i - nc;
      *reinterpret_cast<uint4*>(g_skip + (size_t)j * 8) =
          *reinterpret_cast<const uint4*>(dx + (size_t)(j / q1) * c + c0 + (j % q1) * 8);
    }
  }
}

// Encoder output gradient: (pool adjoint of the coarser gradient + skip
// gradient) * ReLU mask; 8 channels (16 bytes) per thread.
__global__ void encoder_grad_kernel(const bf16* __restrict__ g_coarse, const bf16* __restrict__ g_skip,
                                    const bf16* __restrict__ act, int n, int d, int h, int w, int c,
                                    bf16* __restrict__ g) {
  // 32-bit index arithmetic (training volumes hold far fewer than 2^32 elements)
  const unsigned h2 = h >> 1, w2 = w >> 1, q = c / 8, uw = w, uh = h, ud = d;
  const unsigned total = (unsigned)n * d * h * w * q;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const unsigned j = i % q, v = i / q;
    const unsigned xx = v % uw, r = v / uw, yy = r % uh, r2 = r / uh, zz = r2 % ud, b = r2 / ud;
    const uint4 sv = *reinterpret_cast<const uint4*>(g_skip + (size_t)i * 8);
    const uint4 cv = *reinterpret_cast<const uint4*>(
        g_coarse + (size_t)((((b * (ud >> 1) + (zz >> 1)) * h2 + (yy >> 1)) * w2 + (xx >> 1)) * q + j) * 8);
    const uint4 av = *reinterpret_cast<const uint4*>(act + (size_t)i * 8);
    const bf16 *se = reinterpret_cast<const bf16*>(&sv), *ce = reinterpret_cast<const bf16*>(&cv),
               *ae = reinterpret_cast<const bf16*>(&av);
    uint4 o;
    bf16* oe = reinterpret_cast<bf16*>(&o);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float t = __bfloat162float(se[k]);
      t += 0.125f * __bfloat162float(ce[k]);
      oe[k] = __float2bfloat16_rn(__bfloat162float(ae[k]) > 0.0f ? t : 0.0f);
    }
    *reinterpret_cast<uint4*>(g + (size_t)i * 8) = o;
  }
}

// Head: y = sum_c top[v][c] hw[c] + hb + x[v][0] (FP32, c in order).  With a
// target, also the weighted squared-error loss partials, dL/dy, d top (BF16)
// and the head's gradient partials.  One thread per voxel (16-byte loads and
// stores of its C channels); per CTA the partials of [loss, dhb, dhw[0..C-1]]
// go through fixed warp shuffle trees and then the four warps in order, and
// are summed over CTAs later in a fixed order.
template <int C>
__global__ void __launch_bounds__(128) head_kernel(const bf16* __restrict__ top, const bf16* __restrict__ x, int cx,
                                                   const float* __restrict__ hw, const float* __restrict__ target,
                                                   const float* __restrict__ weight, long long m, float inv_norm,
                                                   float* __restrict__ y, bf16* __restrict__ dtop,
                                                   float* __restrict__ part) {
  constexpr int S = C + 2;
  __shared__ float red[4][S];
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float mine[S];
#pragma unroll
  for (int j = 0; j < S; ++j) mine[j] = 0.0f;
  if (v < m) {
    float t[C];
    const uint4* tp = reinterpret_cast<const uint4*>(top + v * C);
#pragma unroll
    for (int q = 0; q < C / 8; ++q) {
      const uint4 u = tp[q];
      const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(e[k]);
        t[8 * q + 2 * k] = f.x;
        t[8 * q + 2 * k + 1] = f.y;
      }
    }
    float out = __ldg(hw + C) + __bfloat162float(x[v * cx]);
#pragma unroll
    for (int j = 0; j < C; ++j) out = fmaf(t[j], __ldg(hw + j), out);
    y[v] = out;
    if (target) {
      const float wv = weight ? weight[v] : 1.0f;
      const float diff = out - target[v];
      const float gy = 2.0f * wv * diff * inv_norm;
      mine[0] = wv * diff * diff * inv_norm;
      mine[1] = gy;
      uint4* dp = reinterpret_cast<uint4*>(dtop + v * C);
#pragma unroll
      for (int q = 0; q < C / 8; ++q) {
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int j = 8 * q + 2 * k;
          mine[2 + j] = gy * t[j];
          mine[3 + j] = gy * t[j + 1];
          const __nv_bfloat162 p = __floats2bfloat162_rn(gy * __ldg(hw + j), gy * __ldg(hw + j + 1));
          o[k] = *reinterpret_cast<const uint32_t*>(&p);
        }
        dp[q] = make_uint4(o[0], o[1], o[2], o[3]);
      }
    }
  }
  if (!target) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < S; ++j) {
    float sj = mine[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
    if (lane == 0) red[wid][j] = sj;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < S; j += blockDim.x)
    part[(long long)blockIdx.x * S + j] = ((red[0][j] + red[1][j]) + red[2][j]) + red[3][j];
}

// out[j] = sum over blocks of part[b][j]: one warp per entry, lanes strided
// over the blocks, then a fixed shuffle tree.
__global__ void sum_parts_kernel(const float* __restrict__ part, int blocks, int stride, float* __restrict__ out) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= stride) return;
  float s = 0.0f;
  for (int b = lane; b < blocks; b += 32) s += part[(long long)b * stride + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[j] = s;
}

// Adam on FP32 master weights; writes the BF16 copy the convolutions read.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2, bf16* __restrict__ wb) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float wi = w[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ a, long long n, bf16* __restrict__ b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// Network input channels from whole volumes, for boxes of px x py x pz voxels
// at the given corners: out [np][pz][py][px][8] BF16 = (dose/s, density, act/a,
// act/(a max(density, 0.1)), 0...); target [np][pz][py][px] = dose_high/s (if
// dose_high), weight = (density >= 0.1).  Voxels outside the volume read as 0.
// Linear units keep the squared-error optimum at the conditional mean, so the
// network does not bias organ means.
__global__ void make_patches_kernel(const float* __restrict__ dose, const float* __restrict__ density,
                                    const float* __restrict__ act, const float* __restrict__ dose_high,
                                    int nx, int ny, int nz, float inv_s, float inv_a,
                                    const int* __restrict__ corners, int np, int px, int py, int pz,
                                    bf16* __restrict__ out, float* __restrict__ target,
                                    float* __restrict__ weight) {
  const long long per = (long long)px * py * pz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per * np;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i / per);
    long long r = i % per;
    const int x = (int)(r % px); r /= px;
    const int y = (int)(r % py);
    const int z = (int)(r / py);
    const int gx = corners[3 * p] + x, gy = corners[3 * p + 1] + y, gz = corners[3 * p + 2] + z;
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, c3 = 0.0f, t = 0.0f, wv = 0.0f;
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz) {
      const long long v = ((long long)gz * ny + gy) * nx + gx;
      const float rho = density[v];
      c0 = fmaxf(dose[v], 0.0f) * inv_s;
      c1 = rho;
      c2 = fmaxf(act[v], 0.0f) * inv_a;
      c3 = c2 / fmaxf(rho, 0.1f);  // local (positron) deposit per unit mass
      if (dose_high) t = fmaxf(dose_high[v], 0.0f) * inv_s;
      wv = rho >= 0.1f ? 1.0f : 0.0f;
    }
    __align__(16) bf16 o[8];
    o[0] = __float2bfloat16_rn(c0);
    o[1] = __float2bfloat16_rn(c1);
    o[2] = __float2bfloat16_rn(c2);
    o[3] = __float2bfloat16_rn(c3);
    for (int k = 4; k < 8; ++k) o[k] = __float2bfloat16_rn(0.0f);
    *reinterpret_cast<uint4*>(out + i * 8) = *reinterpret_cast<const uint4*>(o);
    if (target) target[i] = t;
    if (weight) weight[i] = wv;
  }
}

// Writes the core [lo, hi) (box coordinates) of one predicted box of
// px x py x pz voxels at `corner` back into the volume: dose_out = s * y.
__global__ void scatter_box_kernel(const float* __restrict__ y, int cx, int cy, int cz, int px, int py, int pz,
                                   int lox, int loy, int loz, int hix, int hiy, int hiz, int nx, int ny, int nz,
                                   float s, float* __restrict__ dose_out) {
  const long long per = (long long)px * py * pz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per;
       i += (long long)gridDim.x * blockDim.x) {
    long long r = i;
    const int x = (int)(r % px); r /= px;
    const int yy = (int)(r % py);
    const int z = (int)(r / py);
    if (x < lox || x >= hix || yy < loy || yy >= hiy || z < loz || z >= hiz) continue;
    const int gx = cx + x, gy = cy + yy, gz = cz + z;
    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny || gz < 0 || gz >= nz) continue;
    dose_out[((long long)gz * ny + gy) * nx + gx] = s * y[i];
  }
}

// Body statistics in one pass over the volume: per CTA (fixed tree) the sums
// of dose and activity and the voxel count over the body (density >= 0.1),
// and (if box) its bounding box [xmin, ymin, zmin, xmax, ymax, zmax], merged
// with one atomic per CTA and coordinate.
constexpr int kStatBlocks = 1024;
__global__ void __launch_bounds__(256) body_stats_kernel(const float* __restrict__ dose, const float* __restrict__ act,
                                                         const float* __restrict__ density,
                                                         const uint8_t* __restrict__ roi, int nx, int ny, long long n,
                                                         double* __restrict__ part, int* __restrict__ box) {
  __shared__ double sd[256], sa[256], sc[256];
  __shared__ int sb[8][6];
  // per thread FP32 sums of its ~n / 2^18 voxels, then FP64 across threads
  // (fixed tree); 32-bit coordinates (grids hold fewer than 2^31 voxels)
  float vd = 0.0f, va = 0.0f;
  unsigned c = 0;
  int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
  const unsigned unx = (unsigned)nx, uny = (unsigned)ny;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < (unsigned long long)n; i += gridDim.x * blockDim.x) {
    const bool body = density[i] >= 0.1f;
    if (body) {
      vd += dose[i];
      va += act[i];
      ++c;
    }
    if (box && (roi ? roi[i] != 0 : body)) {
      const unsigned r = i / unx, x = i - r * unx, y = r % uny, z = r / uny;
      lo[0] = min(lo[0], (int)x); lo[1] = min(lo[1], (int)y); lo[2] = min(lo[2], (int)z);
      hi[0] = max(hi[0], (int)x); hi[1] = max(hi[1], (int)y); hi[2] = max(hi[2], (int)z);
    }
  }
  sd[threadIdx.x] = vd;
  sa[threadIdx.x] = va;
  sc[threadIdx.x] = (double)c;
  if (box) {
    const int w = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
      lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
      hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
    }
    if ((threadIdx.x & 31) == 0)
      for (int a = 0; a < 3; ++a) {
        sb[w][a] = lo[a];
        sb[w][3 + a] = hi[a];
      }
  }
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sd[threadIdx.x] += sd[threadIdx.x + o];
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = sd[0];
    part[3 * blockIdx.x + 1] = sa[0];
    part[3 * blockIdx.x + 2] = sc[0];
  }
  if (box && threadIdx.x < 6) {
    int v = sb[0][threadIdx.x];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      v = threadIdx.x < 3 ? min(v, sb[w][threadIdx.x]) : max(v, sb[w][threadIdx.x]);
    if (threadIdx.x < 3) atomicMin(box + threadIdx.x, v);
    else atomicMax(box + threadIdx.x, v);
  }
}

// Body means of dose and activity (1 where the body is empty or the sum is
// not positive) and, if box_out, the bounding box of the body, or of the
// non-zero voxels of roi when given (xmax < xmin when empty).  Synchronises
// the stream.
nm_status body_stats(const float* dose, const float* activity, const float* density, const uint8_t* roi, int nx,
                     int ny, long long n, float* dose_scale, float* act_scale, int* box_out, cudaStream_t s);

// Default voxel budget of one inference pass: about 330 bytes of activations
// per voxel over all levels, so about 11 GB.
constexpr long long kInferVoxels = 1ll << 25;

int grid1d(long long n) { return (int)std::min<long long>((n + 255) / 256, 8192); }

struct Layer {
  std::string name;
  int cin, c0, c1, coarse, cout, kpad, level;
  long long w_off, b_off;  // offsets into the flat parameter vector (floats)
};

}  // namespace

struct nm_denoiser {
  nm_denoise_options opt{};
  cudaStream_t s = nullptr;
  int P = 64, B = 1, L = 4, base = 16, cx = 8;
  int PD = 64, PH = 64, PW = 64;   // volume of one batch item (P^3 for training)
  // Inference instance for whole-volume apply: forward buffers of its own
  // size, parameters and status shared with (owned by) this handle.
  nm_denoiser* inf = nullptr;
  bool owns_params = true;
  std::vector<int> widths;
  std::vector<Layer> layers;
  long long n_params = 0;
  long long head_off = 0;
  // parameters
  float* w = nullptr;     // FP32 master, flat
  float* g = nullptr;     // gradients, flat
  float* m1 = nullptr;
  float* m2 = nullptr;
  bf16* wb = nullptr;     // BF16 copy, flat (same offsets)
  bf16* wflip = nullptr;  // flipped weights of the layer being back-propagated
  long long wflip_elems = 0;
  // activations [level tensors]
  std::vector<bf16*> ea, eb, pool, da, db;
  bf16 *gA = nullptr, *gB = nullptr, *gC = nullptr, *gD = nullptr;  // gradient scratch (largest size)
  std::vector<bf16*> gskip;
  std::vector<bf16*> cat;          // materialised decoder inputs (shifted-window path)
  bf16* x_in = nullptr;
  float* y = nullptr;
  float* target = nullptr;
  float* weight = nullptr;
  bf16* dtop = nullptr;
  float* head_part = nullptr;
  float* head_sum = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  uint32_t* status = nullptr;
  long long step = 0;
  int head_blocks = 0;
  bool use_weight = false;         // the train step's loss has a per-voxel weight map
  // Forward, head and backward of a train step, and forward and head of
  // nm_denoise_forward, each as one CUDA graph (captured on a stream of the
  // handle's own, launched on s); re-captured when a setting it bakes in
  // changes (key).
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t train_exec = nullptr, fwd_exec = nullptr;   // train step; forward + head
  int train_key = -1, fwd_key = -1;
  // Test support (nm_denoise_capture): per convolution layer, in forward
  // order, its input (decoder inputs as the concatenation [upsampled coarse |
  // skip]), its output activation and the loss gradient at its output after
  // the ReLU mask, all BF16, refreshed by every train step while on.
  bool capture = false;
  std::vector<bf16*> cap_x, cap_y, cap_g;

  ~nm_denoiser() {
    auto f = [](void* p) { if (p) cudaFree(p); };
    delete inf;
    if (owns_params) {
      f(w); f(g); f(m1); f(m2); f(wb); f(status);
    }
    f(wflip);
    for (auto p : ea) f(p);
    for (auto p : eb) f(p);
    for (auto p : pool) f(p);
    for (auto p : da) f(p);
    for (auto p : db) f(p);
    for (auto p : gskip) f(p);
    for (auto p : cat) f(p);
    f(gA); f(gB); f(gC); f(gD); f(x_in); f(y); f(target); f(weight); f(dtop); f(head_part); f(head_sum);
    f(ws);
    free_capture();
    if (train_exec) cudaGraphExecDestroy(train_exec);
    if (fwd_exec) cudaGraphExecDestroy(fwd_exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }

  void free_capture() {
    for (auto v : {&cap_x, &cap_y, &cap_g})
      for (auto p : *v)
        if (p) cudaFree(p);
    cap_x.clear(); cap_y.clear(); cap_g.clear();
  }

  long long vox(int level) const { return (long long)B * (PD >> level) * (PH >> level) * (PW >> level); }
  nm_conv3d_desc desc(const Layer& l) const {
    nm_conv3d_desc d;
    d.n = B; d.d = PD >> l.level; d.h = PH >> l.level; d.w = PW >> l.level;
    d.c0 = l.c0; d.c1 = l.c1; d.src0_coarse = l.coarse; d.cout = l.cout;
    return d;
  }
};

namespace {

nm_status fail(nm_status st, const char* msg) {
  set_error_message(msg);
  return st;
}
nm_status cfail(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  set_error_message(buf);
  return e == cudaErrorMemoryAllocation ? NM_ERR_OOM : NM_ERR_CUDA;
}
#define CK(call, what)                              \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cfail(e_, what);  \
  } while (0)

template <class T>
cudaError_t dmalloc(T** p, long long n) {
  return cudaMalloc((void**)p, (size_t)std::max<long long>(n, 1) * sizeof(T));
}

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

nm_status check_status(nm_denoiser* h) {
  uint32_t flags = 0;
  CK(cudaMemcpyAsync(&flags, h->status, 4, cudaMemcpyDeviceToHost, h->s), "status");
  CK(cudaStreamSynchronize(h->s), "denoiser");
  if (flags) {
    cudaMemsetAsync(h->status, 0, 4, h->s);
    return fail(NM_ERR_DEVICE, "tensor-core wait timed out");
  }
  return NM_OK;
}

nm_status body_stats(const float* dose, const float* activity, const float* density, const uint8_t* roi, int nx,
                     int ny, long long n, float* dose_scale, float* act_scale, int* box_out, cudaStream_t s) {
  double* part = nullptr;
  int* dbox = nullptr;
  const size_t pbytes = kStatBlocks * 3 * sizeof(double);
  CK(cudaMallocAsync((void**)&part, pbytes + 8 * sizeof(int), s), "body statistics");
  if (box_out) {
    dbox = (int*)((char*)part + pbytes);
    const int init[6] = {INT_MAX, INT_MAX, INT_MAX, -1, -1, -1};
    CK(cudaMemcpyAsync(dbox, init, sizeof init, cudaMemcpyHostToDevice, s), "body statistics");
  }
  std::vector<double> r(kStatBlocks * 3);
  body_stats_kernel<<<kStatBlocks, 256, 0, s>>>(dose, activity, density, roi, nx, ny, n, part, dbox);
  cudaError_t e = cudaMemcpyAsync(r.data(), part, pbytes, cudaMemcpyDeviceToHost, s);
  if (!e && box_out) e = cudaMemcpyAsync(box_out, dbox, 6 * sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(part, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return cfail(e, "body statistics");
  double v[2] = {0, 0}, c = 0;
  for (int b = 0; b < kStatBlocks; ++b) {
    v[0] += r[3 * b];
    v[1] += r[3 * b + 1];
    c += r[3 * b + 2];
  }
  *dose_scale = c > 0 && v[0] > 0 ? (float)(v[0] / c) : 1.0f;
  *act_scale = c > 0 && v[1] > 0 ? (float)(v[1] / c) : 1.0f;
  return NM_OK;
}

// Decoder input convolution as one materialised source (upsampled coarse |
// skip) when the shifted-window kernel can take it.
nm_conv3d_desc single_source(const nm_denoiser* h, const Layer& l) {
  nm_conv3d_desc d = h->desc(l);
  d.c0 = l.c0 + l.c1;
  d.c1 = 0;
  d.src0_coarse = 0;
  return d;
}
bool use_cat(const nm_denoiser* h, const Layer& l) { return l.c1 > 0 && conv_tile_ok(single_source(h, l)); }

// Forward pass.  With fuse_head (inference) the last convolution writes the
// head's output h->y directly when the shifted-window kernel takes it, and
// *fused says so (the caller then skips head()).
nm_status forward(nm_denoiser* h, bool fuse_head = false, bool* fused = nullptr) {
  if (fused) *fused = false;
  cudaStream_t s = h->s;
  const int L = h->L;
  const bf16* in = h->x_in;
  int li = 0;
  // test capture: layer k's input and output activation
  auto keep = [&](int k, const bf16* x, const bf16* y) -> cudaError_t {
    if (!h->capture) return cudaSuccess;
    const Layer& l = h->layers[k];
    const long long v = h->vox(l.level);
    cudaError_t e = x ? cudaMemcpyAsync(h->cap_x[k], x, v * l.cin * sizeof(bf16), cudaMemcpyDeviceToDevice, s)
                      : cudaSuccess;
    if (!e) e = cudaMemcpyAsync(h->cap_y[k], y, v * l.cout * sizeof(bf16), cudaMemcpyDeviceToDevice, s);
    return e;
  };
  for (int i = 0; i < L; ++i) {
    const Layer& la = h->layers[li++];
    const Layer& lb = h->layers[li++];
    CK(conv3d_fwd(h->desc(la), in, nullptr, h->wb + la.w_off, h->w + la.b_off, h->ea[i], 1, h->status, s), "conv");
    CK(conv3d_fwd(h->desc(lb), h->ea[i], nullptr, h->wb + lb.w_off, h->w + lb.b_off, h->eb[i], 1, h->status, s), "conv");
    CK(keep(li - 2, in, h->ea[i]), "capture");
    CK(keep(li - 1, h->ea[i], h->eb[i]), "capture");
    if (i < L - 1) {
      const long long n = h->vox(i + 1) * h->widths[i];
      avgpool_kernel<<<grid1d(n / 8), 256, 0, s>>>(h->eb[i], h->B, h->PD >> i, h->PH >> i, h->PW >> i, h->widths[i],
                                               h->pool[i]);
      in = h->pool[i];
    }
  }
  const bf16* coarse = h->eb[L - 1];
  for (int i = L - 2; i >= 0; --i) {
    const Layer& la = h->layers[li++];
    const Layer& lb = h->layers[li++];
    if (use_cat(h, la)) {
      const long long n = h->vox(i) * (la.cin / 8);
      upsample_concat_kernel<<<grid1d(n), 256, 0, s>>>(coarse, h->eb[i], h->B, h->PD >> i, h->PH >> i, h->PW >> i,
                                                       la.c0, la.c1, h->cat[i]);
      CK(conv3d_fwd(single_source(h, la), h->cat[i], nullptr, h->wb + la.w_off, h->w + la.b_off, h->da[i], 1,
                    h->status, s), "conv");
    } else {
      CK(conv3d_fwd(h->desc(la), coarse, h->eb[i], h->wb + la.w_off, h->w + la.b_off, h->da[i], 1, h->status, s),
         "conv");
    }
    if (h->capture) {
      // the decoder input as one tensor, whichever form the convolution read
      const long long n = h->vox(i) * (la.cin / 8);
      upsample_concat_kernel<<<grid1d(n), 256, 0, s>>>(coarse, h->eb[i], h->B, h->PD >> i, h->PH >> i, h->PW >> i,
                                                       la.c0, la.c1, h->cap_x[li - 2]);
      CK(keep(li - 2, nullptr, h->da[i]), "capture");
    }
    if (i == 0 && fuse_head && lb.cout == 16 && conv_tile_ok(h->desc(lb))) {
      CK(conv3d_fwd_tile_head(h->desc(lb), h->da[0], h->wb + lb.w_off, h->w + lb.b_off, h->w + h->head_off, h->x_in,
                              h->cx, h->y, h->status, s),
         "conv");
      if (fused) *fused = true;
      return NM_OK;
    }
    CK(conv3d_fwd(h->desc(lb), h->da[i], nullptr, h->wb + lb.w_off, h->w + lb.b_off, h->db[i], 1, h->status, s), "conv");
    CK(keep(li - 1, h->da[i], h->db[i]), "capture");
    coarse = h->db[i];
  }
  return NM_OK;
}

nm_status head(nm_denoiser* h, bool train) {
  cudaStream_t s = h->s;
  const long long m = h->vox(0);
  const int c = h->widths[0];
  // loss normalisation: mean over all voxels of the batch (blocks of 128 voxels)
  auto kern = c == 16 ? head_kernel<16> : head_kernel<32>;
  kern<<<h->head_blocks, 128, 0, s>>>(h->db[0], h->x_in, h->cx, h->w + h->head_off, train ? h->target : nullptr,
                                      train && h->use_weight ? h->weight : nullptr, m, 1.0f / (float)m, h->y,
                                      h->dtop, h->head_part);
  CK(cudaGetLastError(), "head");
  if (train) {
    sum_parts_kernel<<<(c + 2 + 3) / 4, 128, 0, s>>>(h->head_part, h->head_blocks, c + 2, h->head_sum);
    CK(cudaGetLastError(), "head");
  }
  return NM_OK;
}

// Forward-only instance of h for one D x H x W volume (multiples of 2^(L-1)),
// sharing h's parameters; kept in h->inf and reused while it is large enough.
nm_status inference_instance(nm_denoiser* h, int D, int H, int W, nm_denoiser** out) {
  const long long need = (long long)D * H * W;
  nm_denoiser* c = h->inf;
  if (!c || (long long)c->PD * c->PH * c->PW < need) {
    delete h->inf;
    h->inf = nullptr;
    c = new nm_denoiser();
    c->owns_params = false;
    c->opt = h->opt; c->s = h->s; c->P = 0; c->B = 1; c->L = h->L; c->base = h->base; c->cx = h->cx;
    c->widths = h->widths; c->layers = h->layers; c->n_params = h->n_params; c->head_off = h->head_off;
    c->w = h->w; c->wb = h->wb; c->status = h->status;
    c->PD = D; c->PH = H; c->PW = W;
    h->inf = c;
    const int L = c->L;
    c->ea.assign(L, nullptr); c->eb.assign(L, nullptr); c->pool.assign(L, nullptr);
    c->da.assign(L, nullptr); c->db.assign(L, nullptr); c->cat.assign(L, nullptr);
    cudaError_t e;
    for (int i = 0; i < L; ++i) {
      const long long n = c->vox(i) * c->widths[i];
      if ((e = dmalloc(&c->ea[i], n)) || (e = dmalloc(&c->eb[i], n))) return cfail(e, "inference activations");
      if (i < L - 1) {
        if ((e = dmalloc(&c->pool[i], c->vox(i + 1) * c->widths[i])) || (e = dmalloc(&c->da[i], n)) ||
            (e = dmalloc(&c->db[i], n)) || (e = dmalloc(&c->cat[i], c->vox(i) * (c->widths[i] + c->widths[i + 1]))))
          return cfail(e, "inference activations");
      }
    }
    if ((e = dmalloc(&c->x_in, c->vox(0) * c->cx)) || (e = dmalloc(&c->y, c->vox(0))))
      return cfail(e, "inference activations");
  }
  // every buffer scales with D H W / 8^level, so a larger allocation serves
  c->PD = D; c->PH = H; c->PW = W;
  c->head_blocks = (int)((c->vox(0) + 127) / 128);
  *out = c;
  return NM_OK;
}

nm_status backward(nm_denoiser* h) {
  cudaStream_t s = h->s;
  const int L = h->L;
  // head gradients: head_sum = [loss, dhb, dhw...] -> g[head_off + j] = dhw[j], g[head_off + c] = dhb
  const int c0w = h->widths[0];
  CK(cudaMemcpyAsync(h->g + h->head_off, h->head_sum + 2, c0w * sizeof(float), cudaMemcpyDeviceToDevice, s), "head grad");
  CK(cudaMemcpyAsync(h->g + h->head_off + c0w, h->head_sum + 1, sizeof(float), cudaMemcpyDeviceToDevice, s), "head grad");
  auto lay = [&](const std::string& n) -> const Layer& {
    for (auto& l : h->layers) if (l.name == n) return l;
    return h->layers[0];
  };
  auto conv_back_input = [&](const Layer& l, const bf16* gout, bf16* gin) -> nm_status {
    nm_conv3d_desc fd = h->desc(l);
    CK(conv3d_flip_weights(fd, h->wb + l.w_off, h->wflip, s), "flip");
    nm_conv3d_desc bd;
    memset(&bd, 0, sizeof bd);
    bd.n = fd.n; bd.d = fd.d; bd.h = fd.h; bd.w = fd.w;
    bd.c0 = l.cout; bd.cout = l.c0 + l.c1;
    CK(conv3d_fwd(bd, gout, nullptr, h->wflip, nullptr, gin, 0, h->status, s), "dgrad");
    return NM_OK;
  };
  // the weight-gradient workspace must hold what the kernel chosen for d writes
  auto wgrad = [&](const nm_conv3d_desc& d, const Layer& l, const bf16* x0, const bf16* x1,
                   const bf16* gout) -> nm_status {
    if (conv_wgrad_workspace(d) > h->ws_bytes) return fail(NM_ERR_STATE, "weight-gradient workspace too small");
    CK(conv3d_wgrad(d, x0, x1, gout, h->g + l.w_off, h->g + l.b_off, h->ws, h->status, s), "wgrad");
    return NM_OK;
  };
  auto conv_back = [&](const Layer& l, const bf16* x0, const bf16* x1, const bf16* gout, bf16* gin) -> nm_status {
    // weight/bias gradients, then (if gin) the input gradient through flipped weights
    nm_status st = wgrad(h->desc(l), l, x0, x1, gout);
    if (st != NM_OK) return st;
    if (gin) {
      nm_conv3d_desc fd = h->desc(l);
      CK(conv3d_flip_weights(fd, h->wb + l.w_off, h->wflip, s), "flip");
      nm_conv3d_desc bd;
      memset(&bd, 0, sizeof bd);
      bd.n = fd.n; bd.d = fd.d; bd.h = fd.h; bd.w = fd.w;
      bd.c0 = l.cout; bd.cout = l.c0 + l.c1;
      CK(conv3d_fwd(bd, gout, nullptr, h->wflip, nullptr, gin, 0, h->status, s), "dgrad");
    }
    return NM_OK;
  };
  // test capture: the gradient at layer l's output, after its ReLU mask
  auto keep_grad = [&](const Layer& l, const bf16* gm) -> cudaError_t {
    if (!h->capture) return cudaSuccess;
    const int k = (int)(&l - h->layers.data());
    return cudaMemcpyAsync(h->cap_g[k], gm, h->vox(l.level) * l.cout * sizeof(bf16), cudaMemcpyDeviceToDevice, s);
  };
  nm_status st;
  // gradient wrt the top decoder output
  bf16* g = h->dtop;
  for (int i = 0; i < L - 1; ++i) {
    const Layer& lb = lay("d" + std::to_string(i) + "b");
    const Layer& la = lay("d" + std::to_string(i) + "a");
    const long long nb = h->vox(i) * h->widths[i];
    relu_mask_kernel<<<grid1d(nb / 8), 256, 0, s>>>(g, h->db[i], nb);
    CK(keep_grad(lb, g), "capture");
    if ((st = conv_back(lb, h->da[i], nullptr, g, h->gA)) != NM_OK) return st;
    relu_mask_kernel<<<grid1d(nb / 8), 256, 0, s>>>(h->gA, h->da[i], nb);
    CK(keep_grad(la, h->gA), "capture");
    const bf16* coarse = i + 1 <= L - 2 ? h->db[i + 1] : h->eb[L - 1];
    if (use_cat(h, la)) {
      // same im2col rows, read from the materialised input
      if ((st = wgrad(single_source(h, la), la, h->cat[i], nullptr, h->gA)) != NM_OK) return st;
      if ((st = conv_back_input(la, h->gA, h->gB)) != NM_OK) return st;
    } else if ((st = conv_back(la, coarse, h->eb[i], h->gA, h->gB)) != NM_OK) {
      return st;
    }
    const long long total = h->vox(i + 1) * h->widths[i + 1] + nb;
    split_concat_grad_kernel<<<grid1d(total / 8), 256, 0, s>>>(h->gB, h->B, h->PD >> i, h->PH >> i, h->PW >> i,
                                                           h->widths[i + 1], h->widths[i],
                                                           coarse, h->gC, h->gskip[i]);
    // gC now holds the (masked) gradient wrt the coarser output; move it to gD
    std::swap(h->gC, h->gD);
    g = h->gD;
  }
  // encoder, deepest first; g = gradient wrt e_{L-1} output (already masked by its ReLU)
  for (int i = L - 1; i >= 0; --i) {
    const Layer& lb = lay("e" + std::to_string(i) + "b");
    const Layer& la = lay("e" + std::to_string(i) + "a");
    const long long nb = h->vox(i) * h->widths[i];
    if (i < L - 1) {
      encoder_grad_kernel<<<grid1d(nb / 8), 256, 0, s>>>(g, h->gskip[i], h->eb[i], h->B, h->PD >> i, h->PH >> i,
                                                     h->PW >> i, h->widths[i], h->gC);
      g = h->gC;
    }
    CK(keep_grad(lb, g), "capture");
    if ((st = conv_back(lb, h->ea[i], nullptr, g, h->gA)) != NM_OK) return st;
    relu_mask_kernel<<<grid1d(nb / 8), 256, 0, s>>>(h->gA, h->ea[i], nb);
    CK(keep_grad(la, h->gA), "capture");
    const bf16* in = i == 0 ? h->x_in : h->pool[i - 1];
    if ((st = conv_back(la, in, nullptr, h->gA, i > 0 ? h->gB : nullptr)) != NM_OK) return st;
    if (i > 0) {
      std::swap(h->gB, h->gD);
      g = h->gD;  // gradient wrt pool[i-1] = pooled e_{i-1} output
    }
  }
  CK(cudaGetLastError(), "backward");
  return NM_OK;
}

}  // namespace

namespace {

// Runs `body` (a fixed sequence of launches on h->s) as a CUDA graph captured
// on a stream of the handle's own and launched on h->s, re-captured when its
// key changes: `key` with the convolution forms the environment selects.
// NM_DENOISE_NO_GRAPH=1, or test capture being on, runs body directly.
template <class F>
nm_status run_steps(nm_denoiser* h, cudaGraphExec_t& exec, int& key_slot, int key, F body) {
  const char* ng = getenv("NM_DENOISE_NO_GRAPH");
  if (h->capture || (ng && ng[0] == '1')) return body();
  const char* envs[] = {"NM_CONV_GATHER", "NM_CONV_TILE_UNPACKED", "NM_WGRAD_TILE_UNPACKED"};
  for (int i = 0; i < 3; ++i) {
    const char* e = getenv(envs[i]);
    if (e && e[0] == '1') key |= 2 << i;
  }
  const cudaStream_t s = h->s;
  if (!exec || key_slot != key) {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "graph stream");
    CK(cudaStreamSynchronize(s), "graph capture");
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    h->s = h->cap_stream;
    const nm_status st = body();
    h->s = s;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
    if (st != NM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ec != cudaSuccess) return cfail(ec, "graph capture");
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      exec = nullptr;
      return cfail(ei, "graph instantiate");
    }
    key_slot = key;
  }
  CK(cudaGraphLaunch(exec, s), "graph launch");
  return NM_OK;
}

}  // namespace

extern "C" {

void nm_denoise_options_default(nm_denoise_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->patch = 64;
  o->batch = 2;
  o->levels = 4;
  o->base_width = 16;
  o->lr = 1e-3f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  o->seed = 1;
  o->infer_voxels = kInferVoxels;
}

nm_status nm_denoise_create(nm_denoiser** out, const nm_denoise_options* opts) {
  if (!out) return fail(NM_ERR_ARG, "out is NULL");
  *out = nullptr;
  nm_denoise_options o;
  if (opts) o = *opts; else nm_denoise_options_default(&o);
  if (o.levels < 2 || o.levels > 4 || o.patch % (1 << (o.levels - 1)) || o.patch < 8 || o.batch < 1 ||
      !(o.base_width == 16 || o.base_width == 32) || (o.base_width << (o.levels - 1)) > 128)
    return fail(NM_ERR_ARG, "denoiser: levels 2..4, patch a multiple of 2^(levels-1), base width 16 or 32, widths <= 128");
  if (o.infer_voxels == 0) o.infer_voxels = kInferVoxels;
  if (o.infer_voxels < 4096) return fail(NM_ERR_ARG, "denoiser: infer_voxels must be >= 4096");
  nm_denoiser* h = new nm_denoiser();
  auto bail = [&](nm_status st) { delete h; return st; };
  h->opt = o;
  h->s = (cudaStream_t)o.stream;
  h->P = o.patch; h->B = o.batch; h->L = o.levels; h->base = o.base_width;
  h->PD = h->PH = h->PW = o.patch;
  for (int i = 0; i < h->L; ++i) h->widths.push_back(h->base << i);
  // layers in forward order
  long long off = 0;
  int c = h->cx;
  auto add = [&](const std::string& n, int c0, int c1, int coarse, int cout, int level) {
    Layer l;
    l.name = n; l.c0 = c0; l.c1 = c1; l.cin = c0 + c1; l.coarse = coarse; l.cout = cout;
    l.kpad = conv_kpad(l.cin); l.level = level;
    l.w_off = off; off += (long long)cout * l.kpad;
    l.b_off = off; off += cout;
    off = (off + 7) / 8 * 8;  // 16-byte aligned BF16 weights
    h->layers.push_back(l);
  };
  for (int i = 0; i < h->L; ++i) {
    add("e" + std::to_string(i) + "a", c, 0, 0, h->widths[i], i);
    add("e" + std::to_string(i) + "b", h->widths[i], 0, 0, h->widths[i], i);
    c = h->widths[i];
  }
  for (int i = h->L - 2; i >= 0; --i) {
    add("d" + std::to_string(i) + "a", c, h->widths[i], 1, h->widths[i], i);
    add("d" + std::to_string(i) + "b", h->widths[i], 0, 0, h->widths[i], i);
    c = h->widths[i];
  }
  h->head_off = off;
  off += h->widths[0] + 1;
  h->n_params = (off + 7) / 8 * 8;

  cudaError_t e;
  if ((e = dmalloc(&h->w, h->n_params)) || (e = dmalloc(&h->g, h->n_params)) || (e = dmalloc(&h->m1, h->n_params)) ||
      (e = dmalloc(&h->m2, h->n_params)) || (e = dmalloc(&h->wb, h->n_params)) || (e = dmalloc(&h->status, 1)))
    return bail(cfail(e, "denoiser parameters"));
  long long flip = 0;
  size_t ws = 0;
  for (auto& l : h->layers) {
    flip = std::max<long long>(flip, (long long)l.cin * conv_kpad(l.cout));
    // a decoder input's weight gradient runs on the two-source description or,
    // when its input is materialised, on the single-source one: the kernels
    // (and workspaces) of the two differ
    ws = std::max(ws, conv_wgrad_workspace(h->desc(l)));
    if (l.c1 > 0) ws = std::max(ws, conv_wgrad_workspace(single_source(h, l)));
  }
  h->wflip_elems = flip;
  h->ws_bytes = ws;
  if ((e = dmalloc(&h->wflip, flip)) || (e = cudaMalloc(&h->ws, ws))) return bail(cfail(e, "denoiser workspace"));
  h->ea.resize(h->L); h->eb.resize(h->L); h->pool.resize(h->L); h->da.resize(h->L); h->db.resize(h->L);
  h->gskip.resize(h->L);
  h->cat.assign(h->L, nullptr);
  for (int i = 0; i + 1 < h->L; ++i)
    if ((e = dmalloc(&h->cat[i], h->vox(i) * (h->widths[i] + h->widths[i + 1])))) return bail(cfail(e, "activations"));
  long long gmax = 0;
  for (int i = 0; i < h->L; ++i) {
    const long long n = h->vox(i) * h->widths[i];
    if ((e = dmalloc(&h->ea[i], n)) || (e = dmalloc(&h->eb[i], n))) return bail(cfail(e, "activations"));
    if (i < h->L - 1) {
      if ((e = dmalloc(&h->pool[i], h->vox(i + 1) * h->widths[i])) || (e = dmalloc(&h->da[i], n)) ||
          (e = dmalloc(&h->db[i], n)) || (e = dmalloc(&h->gskip[i], n)))
        return bail(cfail(e, "activations"));
      gmax = std::max(gmax, h->vox(i) * (long long)(h->widths[i] + h->widths[i + 1]));
    }
    gmax = std::max(gmax, n);
  }
  const long long m = h->vox(0);
  h->head_blocks = (int)((m + 127) / 128);
  if ((e = dmalloc(&h->gA, gmax)) || (e = dmalloc(&h->gB, gmax)) || (e = dmalloc(&h->gC, gmax)) ||
      (e = dmalloc(&h->gD, gmax)) || (e = dmalloc(&h->x_in, m * h->cx)) || (e = dmalloc(&h->y, m)) ||
      (e = dmalloc(&h->target, m)) || (e = dmalloc(&h->weight, m)) || (e = dmalloc(&h->dtop, m * h->widths[0])) ||
      (e = dmalloc(&h->head_part, (long long)h->head_blocks * (h->widths[0] + 2))) ||
      (e = dmalloc(&h->head_sum, h->widths[0] + 2)))
    return bail(cfail(e, "denoiser buffers"));
  // He-normal initialisation on the host (seeded), zero padding columns.
  std::vector<float> w(h->n_params, 0.0f);
  std::mt19937_64 rng(o.seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (auto& l : h->layers) {
    const double std_ = std::sqrt(2.0 / (27.0 * l.cin));
    for (int co = 0; co < l.cout; ++co)
      for (int k = 0; k < 27 * l.cin; ++k) w[l.w_off + (long long)co * l.kpad + k] = (float)(std_ * nd(rng));
  }
  // the head starts at zero: the initial network is the identity on channel 0
  if ((e = cudaMemcpy(h->w, w.data(), h->n_params * sizeof(float), cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(h->g, 0, h->n_params * sizeof(float))) || (e = cudaMemset(h->m1, 0, h->n_params * sizeof(float))) ||
      (e = cudaMemset(h->m2, 0, h->n_params * sizeof(float))) || (e = cudaMemset(h->status, 0, 4)))
    return bail(cfail(e, "denoiser init"));
  to_bf16_kernel<<<grid1d(h->n_params), 256, 0, h->s>>>(h->w, h->n_params, h->wb);
  if ((e = cudaStreamSynchronize(h->s))) return bail(cfail(e, "denoiser init"));
  *out = h;
  return NM_OK;
}

void nm_denoise_destroy(nm_denoiser* h) {
  if (!h) return;
  cudaStreamSynchronize(h->s);
  delete h;
}

int64_t nm_denoise_param_count(const nm_denoiser* h) { return h ? h->n_params : 0; }

nm_status nm_denoise_layer(const nm_denoiser* h, int32_t i, int32_t* cin, int32_t* cout, int32_t* kpad,
                           int64_t* w_offset, int64_t* b_offset) {
  if (!h || i < 0 || i > (int)h->layers.size()) return fail(NM_ERR_ARG, "layer index out of range");
  if (i == (int)h->layers.size()) {  // the head
    if (cin) *cin = h->widths[0];
    if (cout) *cout = 1;
    if (kpad) *kpad = h->widths[0];
    if (w_offset) *w_offset = h->head_off;
    if (b_offset) *b_offset = h->head_off + h->widths[0];
    return NM_OK;
  }
  const Layer& l = h->layers[i];
  if (cin) *cin = l.cin;
  if (cout) *cout = l.cout;
  if (kpad) *kpad = l.kpad;
  if (w_offset) *w_offset = l.w_off;
  if (b_offset) *b_offset = l.b_off;
  return NM_OK;
}

nm_status nm_denoise_params(nm_denoiser* h, float* get, const float* set, float* grads) {
  if (!h) return fail(NM_ERR_ARG, "handle is NULL");
  const size_t bytes = h->n_params * sizeof(float);
  if (set) {
    CK(cudaMemcpyAsync(h->w, set, bytes, cudaMemcpyDefault, h->s), "params");
    to_bf16_kernel<<<grid1d(h->n_params), 256, 0, h->s>>>(h->w, h->n_params, h->wb);
  }
  if (get) CK(cudaMemcpyAsync(get, h->w, bytes, cudaMemcpyDefault, h->s), "params");
  if (grads) CK(cudaMemcpyAsync(grads, h->g, bytes, cudaMemcpyDefault, h->s), "params");
  CK(cudaStreamSynchronize(h->s), "params");
  return NM_OK;
}

nm_status nm_denoise_adam_state(nm_denoiser* h, float* m1, float* m2, int64_t* step) {
  if (!h) return fail(NM_ERR_ARG, "handle is NULL");
  const size_t bytes = h->n_params * sizeof(float);
  if (m1) CK(cudaMemcpyAsync(m1, h->m1, bytes, cudaMemcpyDefault, h->s), "adam state");
  if (m2) CK(cudaMemcpyAsync(m2, h->m2, bytes, cudaMemcpyDefault, h->s), "adam state");
  CK(cudaStreamSynchronize(h->s), "adam state");
  if (step) *step = h->step;
  return NM_OK;
}

nm_status nm_denoise_capture(nm_denoiser* h, int32_t on) {
  if (!h) return fail(NM_ERR_ARG, "handle is NULL");
  CK(cudaStreamSynchronize(h->s), "capture");
  h->free_capture();
  h->capture = false;
  if (!on) return NM_OK;
  const size_t n = h->layers.size();
  h->cap_x.assign(n, nullptr); h->cap_y.assign(n, nullptr); h->cap_g.assign(n, nullptr);
  for (size_t k = 0; k < n; ++k) {
    const Layer& l = h->layers[k];
    const long long v = h->vox(l.level);
    cudaError_t e;
    if ((e = dmalloc(&h->cap_x[k], v * l.cin)) || (e = dmalloc(&h->cap_y[k], v * l.cout)) ||
        (e = dmalloc(&h->cap_g[k], v * l.cout))) {
      h->free_capture();
      return cfail(e, "capture buffers");
    }
  }
  h->capture = true;
  return NM_OK;
}

nm_status nm_denoise_captured(nm_denoiser* h, int32_t layer, int32_t kind, uint16_t* out, int64_t bytes) {
  if (!h || !out) return fail(NM_ERR_ARG, "bad arguments");
  if (!h->capture) return fail(NM_ERR_STATE, "capture is off");
  if (layer < 0 || layer >= (int32_t)h->layers.size() || kind < 0 || kind > 2)
    return fail(NM_ERR_ARG, "layer or kind out of range");
  const Layer& l = h->layers[layer];
  const long long need = h->vox(l.level) * (kind == 0 ? l.cin : l.cout) * (long long)sizeof(bf16);
  if (bytes < need) return fail(NM_ERR_ARG, "output buffer too small");
  const bf16* src = kind == 0 ? h->cap_x[layer] : kind == 1 ? h->cap_y[layer] : h->cap_g[layer];
  CK(cudaMemcpyAsync(out, src, need, cudaMemcpyDefault, h->s), "capture");
  CK(cudaStreamSynchronize(h->s), "capture");
  return NM_OK;
}

nm_status nm_denoise_train_step(nm_denoiser* h, const uint16_t* x, const float* target, const float* weight,
                                float lr, float* loss) {
  NvtxRange range("nm_denoise_train_step");
  if (!h || !x || !target) return fail(NM_ERR_ARG, "bad arguments");
  if (!dev_ptr(x) || !dev_ptr(target) || (weight && !dev_ptr(weight)))
    return fail(NM_ERR_ARG, "x, target and weight must be device pointers");
  cudaStream_t s = h->s;
  const long long m = h->vox(0);
  CK(cudaMemcpyAsync(h->x_in, x, m * h->cx * 2, cudaMemcpyDeviceToDevice, s), "input");
  CK(cudaMemcpyAsync(h->target, target, m * 4, cudaMemcpyDeviceToDevice, s), "input");
  if (weight) CK(cudaMemcpyAsync(h->weight, weight, m * 4, cudaMemcpyDeviceToDevice, s), "input");
  h->use_weight = weight != nullptr;      // no map: every voxel weighs 1
  nm_status st = run_steps(h, h->train_exec, h->train_key, h->use_weight ? 1 : 0, [h]() -> nm_status {
    nm_status r = forward(h);
    if (r == NM_OK) r = head(h, true);
    if (r == NM_OK) r = backward(h);
    return r;
  });
  if (st != NM_OK) return st;
  if (lr > 0.0f) {
    h->step += 1;
    // bias corrections 1 - beta^t in FP64: in FP32 the subtraction cancels
    // (1 - 0.999^2 loses ~3e-5 of its value)
    const float c1 = (float)(1.0 - std::pow((double)h->opt.beta1, (double)h->step));
    const float c2 = (float)(1.0 - std::pow((double)h->opt.beta2, (double)h->step));
    adam_kernel<<<grid1d(h->n_params), 256, 0, s>>>(h->w, h->g, h->m1, h->m2, h->n_params, lr, h->opt.beta1,
                                                   h->opt.beta2, h->opt.eps, c1, c2, h->wb);
    CK(cudaGetLastError(), "adam");
  }
  if (loss) CK(cudaMemcpyAsync(loss, h->head_sum, sizeof(float), cudaMemcpyDeviceToHost, s), "loss");
  return check_status(h);
}

nm_status nm_denoise_forward(nm_denoiser* h, const uint16_t* x, float* y) {
  NvtxRange range("nm_denoise_forward");
  if (!h || !x || !y || !dev_ptr(x) || !dev_ptr(y)) return fail(NM_ERR_ARG, "x and y must be device pointers");
  cudaStream_t s = h->s;
  const long long m = h->vox(0);
  CK(cudaMemcpyAsync(h->x_in, x, m * h->cx * 2, cudaMemcpyDeviceToDevice, s), "input");
  const nm_status st = run_steps(h, h->fwd_exec, h->fwd_key, 0, [h]() -> nm_status {
    nm_status r = forward(h);
    if (r == NM_OK) r = head(h, false);
    return r;
  });
  if (st != NM_OK) return st;
  CK(cudaMemcpyAsync(y, h->y, m * 4, cudaMemcpyDeviceToDevice, s), "output");
  return check_status(h);
}

nm_status nm_denoise_make_patches(const float* dose, const float* density, const float* activity,
                                  const float* dose_high, int32_t nx, int32_t ny, int32_t nz, float dose_scale,
                                  float act_scale, const int32_t* corners, int32_t n_patches, int32_t patch,
                                  uint16_t* x, float* target, float* weight, void* stream) {
  if (!dose || !density || !activity || !corners || !x || nx <= 0 || ny <= 0 || nz <= 0 || n_patches <= 0 ||
      patch <= 0 || !(dose_scale > 0) || !(act_scale > 0))
    return fail(NM_ERR_ARG, "bad arguments");
  if (!dev_ptr(dose) || !dev_ptr(density) || !dev_ptr(activity) || !dev_ptr(corners) || !dev_ptr(x) ||
      (dose_high && !dev_ptr(dose_high)) || (target && !dev_ptr(target)) || (weight && !dev_ptr(weight)))
    return fail(NM_ERR_ARG, "all arrays must be device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = (long long)patch * patch * patch * n_patches;
  make_patches_kernel<<<grid1d(n), 256, 0, s>>>(dose, density, activity, dose_high, nx, ny, nz, 1.0f / dose_scale,
                                                1.0f / act_scale, corners, n_patches, patch, patch, patch, (bf16*)x,
                                                target, weight);
  CK(cudaGetLastError(), "make_patches");
  CK(cudaStreamSynchronize(s), "make_patches");
  return NM_OK;
}

nm_status nm_denoise_scales(const float* dose, const float* activity, const float* density, int64_t n,
                            float* dose_scale, float* act_scale, void* stream) {
  if (!dose || !activity || !density || n <= 0 || !dose_scale || !act_scale) return fail(NM_ERR_ARG, "bad arguments");
  return body_stats(dose, activity, density, nullptr, 1, 1, n, dose_scale, act_scale, nullptr, (cudaStream_t)stream);
}

// Whole-volume inference.  The body's bounding box (density >= 0.1) plus a
// context margin of 8 voxels runs through the network as one volume; above the
// handle's infer_voxels it runs in slabs along z, each with the margin on both
// sides and only its core written back.  Voxels outside the body box keep the
// input.
nm_status nm_denoise_apply(nm_denoiser* h, const float* dose, const float* density, const float* activity,
                           int32_t nx, int32_t ny, int32_t nz, float* dose_out) {
  return nm_denoise_apply_roi(h, dose, density, activity, nullptr, nx, ny, nz, dose_out);
}

nm_status nm_denoise_apply_roi(nm_denoiser* h, const float* dose, const float* density, const float* activity,
                               const uint8_t* roi, int32_t nx, int32_t ny, int32_t nz, float* dose_out) {
  NvtxRange range("nm_denoise_apply_roi");
  if (!h || !dose || !density || !activity || !dose_out || nx <= 0 || ny <= 0 || nz <= 0)
    return fail(NM_ERR_ARG, "bad arguments");
  if (!dev_ptr(dose) || !dev_ptr(density) || !dev_ptr(activity) || !dev_ptr(dose_out) || (roi && !dev_ptr(roi)))
    return fail(NM_ERR_ARG, "volumes must be device pointers");
  cudaStream_t s = h->s;
  const long long V = (long long)nx * ny * nz;
  float ds = 1, as = 1;
  int box[6];
  nm_status st = body_stats(dose, activity, density, roi, nx, ny, V, &ds, &as, box, s);
  if (st != NM_OK) return st;
  if (dose_out != dose) CK(cudaMemcpyAsync(dose_out, dose, V * sizeof(float), cudaMemcpyDeviceToDevice, s), "apply");
  if (box[3] < box[0]) {  // no body (or empty region): nothing to denoise
    CK(cudaStreamSynchronize(s), "apply");
    return NM_OK;
  }
  const int A = 1 << (h->L - 1), mg = 8;
  auto up = [&](int n) { return (n + A - 1) / A * A; };
  const int ex = box[3] + 1 - box[0], ey = box[4] + 1 - box[1], ez = box[5] + 1 - box[2];
  const int W = up(ex + 2 * mg), H = up(ey + 2 * mg);
  // z slabs: core depth tc, network depth D = up(tc + 2 mg) <= the voxel budget
  const long long plane = (long long)W * H;
  int tc = ez;
  const long long budget = h->opt.infer_voxels;
  if (plane * up(ez + 2 * mg) > budget) {
    const int dmax = (int)std::min<long long>(budget / plane, 1 << 30) / A * A;
    if (dmax < 2 * mg + A) return fail(NM_ERR_ARG, "volume cross-section too large for whole-volume inference");
    tc = dmax - 2 * mg;
  }
  const int D = up(tc + 2 * mg);
  nm_denoiser* c = nullptr;
  if ((st = inference_instance(h, D, H, W, &c)) != NM_OK) return st;
  int* dcorn = nullptr;
  CK(cudaMallocAsync((void**)&dcorn, 3 * sizeof(int), s), "apply");
  for (int z0 = box[2]; z0 <= box[5] && st == NM_OK; z0 += tc) {
    const int core = std::min(tc, box[5] + 1 - z0);
    const int corner[3] = {box[0] - mg, box[1] - mg, z0 - mg};
    CK(cudaMemcpyAsync(dcorn, corner, sizeof corner, cudaMemcpyHostToDevice, s), "apply");
    const long long n = (long long)W * H * D;
    make_patches_kernel<<<grid1d(n), 256, 0, s>>>(dose, density, activity, nullptr, nx, ny, nz, 1.0f / ds, 1.0f / as,
                                                  dcorn, 1, W, H, D, c->x_in, nullptr, nullptr);
    bool fused = false;
    if ((st = forward(c, true, &fused)) != NM_OK) break;
    if (!fused && (st = head(c, false)) != NM_OK) break;
    scatter_box_kernel<<<grid1d(n), 256, 0, s>>>(c->y, corner[0], corner[1], corner[2], W, H, D, mg, mg, mg,
                                                 mg + ex, mg + ey, mg + core, nx, ny, nz, ds, dose_out);
    // the corner buffer is reused by the next slab
    CK(cudaStreamSynchronize(s), "apply");
  }
  cudaFreeAsync(dcorn, s);
  if (st != NM_OK) return st;
  CK(cudaGetLastError(), "apply");
  return check_status(h);
}

}  // extern "C"
