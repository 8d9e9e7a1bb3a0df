// 3x3x3 convolution by shifted windows: the tensor cores read the 27 taps
// straight out of one shared-memory halo tile, with no im2col gather.
//
// A CTA computes an output tile of TZ x TY x TX voxels.  Its input tile, with
// a one-voxel halo, is stored as "channel planes": plane j holds channels
// 8j..8j+7 of every padded voxel, 16 bytes per voxel, voxels in x-fastest
// order.  In the no-swizzle K-major operand layout with a stride byte offset of
// 128 (eight 16-byte rows) consecutive voxels are consecutive GEMM rows, so the
// A operand of tap (dz, dy, dx) is the same tile shifted by
// (dz*PY + dy)*PX + dx rows: a different start address in the descriptor.
// GEMM rows run over the padded tile's centre indices; rows whose centre is a
// halo voxel are computed and dropped (20 % for the 16 x 16 x 2 tile).
//
// Channels are consumed 16 at a time (two planes = one MMA K-step): for each
// 16-channel chunk the tile and the chunk's weights are copied with cp.async
// (zero-filled outside the volume) into one of two stage buffers, then one
// thread issues 27 taps x (tile rows / 128) MMAs and commits them to the
// stage's mbarrier.  Waits are bounded as in nm_conv.cu.
#include <cuda_bf16.h>

#include "nm_internal.cuh"
#include "nm_tc.cuh"

namespace nm {
namespace {

constexpr int TX = 16, TY = 16, TZ = 2;
constexpr int PX = TX + 2, PY = TY + 2, PZ = TZ + 2;
constexpr int kRows = PX * PY * PZ;                         // padded tile voxels
constexpr int kCmin = (1 * PY + 1) * PX + 1;                // first centre
constexpr int kCmax = (TZ * PY + TY) * PX + TX;             // last centre
constexpr int kMt = (kCmax - kCmin + 1 + 127) / 128;        // 128-row MMA tiles
constexpr int kDelta = PY * PX + PX + 1;                    // largest tap shift
constexpr int kRowsAlloc = kCmin + kMt * 128 + kDelta;      // rows any MMA may read
constexpr int kThreads = 128;
constexpr long long kWaitCycles = 4ll << 30;

static_assert(kRowsAlloc >= kRows, "tile rows");

template <int COUT>
struct TileLayout {
  static constexpr uint32_t kPlane = kRowsAlloc * 16;       // one 8-channel plane
  static constexpr uint32_t kA = 2 * kPlane;                // 16 channels
  static constexpr uint32_t kSboB = 27 * 16 / 8 * 128;      // 8 weight rows of 27 x 16 channels
  static constexpr uint32_t kB = COUT / 8 * kSboB;
  static constexpr uint32_t kStage = (kA + kB + 1023) / 1024 * 1024;
  static constexpr int kNcols = kMt * COUT <= 32 ? 32 : kMt * COUT <= 64 ? 64 : kMt * COUT <= 128 ? 128
                                : kMt * COUT <= 256 ? 256 : 512;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <int COUT>
__global__ void __launch_bounds__(kThreads) conv_tile_kernel(int n, int d, int h, int w, int cin, int kpad,
                                                             const __nv_bfloat16* __restrict__ x,
                                                             const __nv_bfloat16* __restrict__ wt,
                                                             const float* __restrict__ bias,
                                                             __nv_bfloat16* __restrict__ y, int relu,
                                                             uint32_t* status) {
  typedef TileLayout<COUT> L;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tile origin
  const int tiles_x = (w + TX - 1) / TX, tiles_y = (h + TY - 1) / TY, tiles_z = (d + TZ - 1) / TZ;
  int t = blockIdx.x;
  const int tx = t % tiles_x; t /= tiles_x;
  const int ty = t % tiles_y; t /= tiles_y;
  const int tz = t % tiles_z;
  const int b = t / tiles_z;
  const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;

  if (warp == 0) tc::tmem_alloc(&s_tmem, L::kNcols);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t base = tc::smem_u32(smem);
  const int nchunks = (cin + 15) / 16;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, COUT, false, false);
  bool timeout = false;
  int issued = 0;

  for (int cc = 0; cc < nchunks; ++cc) {
    const int buf = cc & 1;
    if (cc >= 2 && !tc::mbar_wait_bounded(&bar[buf], ((cc >> 1) - 1) & 1, kWaitCycles)) timeout = true;
    if (__syncthreads_or(timeout)) { timeout = true; break; }
    const uint32_t sa = base + buf * L::kStage;
    const uint32_t sb = sa + L::kA;
    // input planes 2cc, 2cc+1 of every padded voxel (zero outside the volume)
    for (int i = tid; i < 2 * kRowsAlloc; i += kThreads) {
      const int p = i / kRowsAlloc, r = i - p * kRowsAlloc;
      const int ch = cc * 16 + p * 8;
      const int pz = r / (PY * PX), py = (r / PX) % PY, px = r % PX;
      const int gz = z0 + pz - 1, gy = y0 + py - 1, gx = x0 + px - 1;
      const bool ok = r < kRows && ch < cin && (unsigned)gz < (unsigned)d && (unsigned)gy < (unsigned)h &&
                      (unsigned)gx < (unsigned)w;
      const __nv_bfloat16* src = ok ? x + ((((long long)b * d + gz) * h + gy) * w + gx) * cin + ch : x;
      cp_async16(sa + p * L::kPlane + r * 16, src, ok);
    }
    // weights of this chunk: row co, K index tap*16 + c
    for (int i = tid; i < COUT * 27 * 2; i += kThreads) {
      const int co = i / 54, rest = i - co * 54;
      const int tap = rest >> 1, j = rest & 1;
      const int ch = cc * 16 + j * 8;
      const bool ok = ch < cin;
      const __nv_bfloat16* src = ok ? wt + (long long)co * kpad + tap * cin + ch : wt;
      const int kchunk = tap * 2 + j;
      cp_async16(sb + (co >> 3) * L::kSboB + kchunk * 128 + (co & 7) * 16, src, ok);
    }
    cp_async_wait_all();
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      for (int tap = 0; tap < 27; ++tap) {
        const int delta = ((tap / 9 - 1) * PY + ((tap / 3) % 3 - 1)) * PX + (tap % 3 - 1);
        const uint64_t bdesc = tc::smem_desc(sb + tap * 256, 128, L::kSboB);
#pragma unroll
        for (int mt = 0; mt < kMt; ++mt) {
          const uint32_t a0 = sa + (uint32_t)(kCmin + mt * 128 + delta) * 16;
          tc::mma_bf16(tmem + mt * COUT, tc::smem_desc(a0, L::kPlane, 128), bdesc, idesc,
                       (cc | tap) != 0);
        }
      }
      tc::mma_commit(&bar[buf]);
    }
    issued = cc + 1;
  }
  if (!timeout && issued > 0) {
    const int last = issued - 1;
    if (!tc::mbar_wait_bounded(&bar[last & 1], (last >> 1) & 1, kWaitCycles)) timeout = true;
  }
  timeout = __syncthreads_or(timeout);
  if (timeout) {
    if (tid == 0) atomicOr(status, NM_DEV_TIMEOUT);
    if (issued > 0) tc::mbar_wait_bounded(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kWaitCycles);
  } else {
    tc::fence_after_sync();
    for (int mt = 0; mt < kMt; ++mt) {
      const int c = kCmin + mt * 128 + warp * 32 + lane;  // this lane's centre
      const int pz = c / (PY * PX), py = (c / PX) % PY, px = c % PX;
      const int gz = z0 + pz - 1, gy = y0 + py - 1, gx = x0 + px - 1;
      const bool ok = c <= kCmax && px >= 1 && px <= TX && py >= 1 && py <= TY && pz >= 1 && pz <= TZ &&
                      gz < d && gy < h && gx < w;
#pragma unroll
      for (int cq = 0; cq < COUT / 16; ++cq) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + mt * COUT + cq * 16, v);
        if (ok) {
          __align__(16) __nv_bfloat16 o[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float tv = v[j] + (bias ? __ldg(bias + cq * 16 + j) : 0.0f);
            if (relu) tv = fmaxf(tv, 0.0f);
            o[j] = __float2bfloat16_rn(tv);
          }
          uint4* dst = reinterpret_cast<uint4*>(y + ((((long long)b * d + gz) * h + gy) * w + gx) * COUT + cq * 16);
          dst[0] = reinterpret_cast<uint4*>(o)[0];
          dst[1] = reinterpret_cast<uint4*>(o)[1];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, L::kNcols);
}

template <int COUT>
cudaError_t launch_tile(const nm_conv3d_desc& g, const void* x, const void* w, const float* bias, void* y,
                        int relu, uint32_t* status, cudaStream_t s) {
  typedef TileLayout<COUT> L;
  const size_t smem = 2 * (size_t)L::kStage;
  cudaError_t e = cudaFuncSetAttribute(conv_tile_kernel<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((g.w + TX - 1) / TX) * ((g.h + TY - 1) / TY) * ((g.d + TZ - 1) / TZ) * g.n;
  const int cin = g.c0;
  conv_tile_kernel<COUT><<<(unsigned)tiles, kThreads, smem, s>>>(g.n, g.d, g.h, g.w, cin, conv_kpad(cin),
                                                                 (const __nv_bfloat16*)x, (const __nv_bfloat16*)w,
                                                                 bias, (__nv_bfloat16*)y, relu, status);
  return cudaGetLastError();
}

}  // namespace

bool conv_tile_ok(const nm_conv3d_desc& d) {
  return d.c1 == 0 && !d.src0_coarse && d.c0 % 8 == 0 && (d.cout == 16 || d.cout == 32);
}

cudaError_t conv3d_fwd_tile(const nm_conv3d_desc& d, const void* x, const void* w, const float* bias, void* y,
                            int relu, uint32_t* status, cudaStream_t s) {
  if (d.cout == 16) return launch_tile<16>(d, x, w, bias, y, relu, status, s);
  return launch_tile<32>(d, x, w, bias, y, relu, status, s);
}

}  // namespace nm
