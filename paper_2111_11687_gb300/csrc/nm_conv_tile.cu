// 3x3x3 convolution by shifted windows: the tensor cores read the 27 taps
// straight out of one shared-memory halo tile, with no im2col gather.
//
// An output tile is TZ x TY x TX voxels.  Its input tile, with a one-voxel
// halo, is stored as "channel planes": plane j holds channels 8j..8j+7 of
// every padded voxel, 16 bytes per voxel, voxels in x-fastest order.  In the
// no-swizzle K-major operand layout with a stride byte offset of 128 (eight
// 16-byte rows) consecutive voxels are consecutive GEMM rows, so the A operand
// of tap (dz, dy, dx) is the same tile shifted by (dz*PY + dy)*PX + dx rows: a
// different start address in the descriptor.  GEMM rows run over the padded
// tile's centre indices; rows whose centre is a halo voxel are computed and
// dropped (20 % for a 16 x 16 x 2 tile, 27 % for 16 x 16 x 4).
//
// The kernel is persistent and warp-specialised (one CTA per SM):
//   warp 0    one thread issues TMA loads: per 16-channel chunk two 5-D tiled
//             tensor loads (the two channel planes of the halo box; the TMA
//             unit zero-fills outside the volume) and one bulk copy of the
//             chunk's weights, pre-arranged in the operand layout;
//   warp 1    one thread issues 27 taps x (tile rows / 128) MMAs per chunk
//             into a TMEM accumulator and commits them to the stage's "empty"
//             barrier, then the tile to the accumulator's "full" barrier;
//   warps 2-13 the epilogue, three warps per TMEM lane quarter (a warp reads
//             only its quarter, warp % 4), warp w taking the 128-row M-tiles
//             mt = (w - 2) / 4 modulo 3: tcgen05.ld, bias, ReLU, BF16, 16-byte
//             stores; then they release the accumulator.  Twelve warps, not
//             four, because the epilogue is bound by the latency of its loads
//             and shuffles (no warp takes more than two of five M-tiles).
// A ring of shared-memory stages and two TMEM accumulators (one when they do
// not fit) let loads, MMAs and the epilogue of consecutive tiles overlap.
//
// Packed variant (16 outputs): an MMA of N = Cout is as slow as one of
// N = 128, bound by reading its 128-row voxel operand from shared memory, so
// the three x-taps of each (dz, dy) share one MMA of N = 3 Cout: its A operand
// is the tile shifted for dx = -1, and its B operand the three taps' weight
// rows, which lie next to each other in the weight image.  Column block j of
// the accumulator then holds tap dx = j - 1 evaluated one row too early per
// unit of dx, and the epilogue adds rows r, r + 1 and r + 2 of the three
// blocks (two warp shuffles per output; the two rows past each warp's last
// lane come from the next warp through shared memory): 9 MMAs per 128 rows and
// chunk instead of 27.
// Every wait is bounded; a time-out sets NM_DEV_TIMEOUT, drains the copies
// and MMAs in flight and frees the tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "nm_internal.cuh"
#include "nm_tc.cuh"

namespace nm {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int TX = 16, TY = 16;
constexpr uint32_t kSboB = 27 * 16 / 8 * 128;               // 8 weight rows of 27 x 16 channels
constexpr int kEpiParts = 3;                               // epilogue warps per TMEM lane quarter
constexpr int kEpiThreads = 128 * kEpiParts;               // warps 2 .. 1 + 4 kEpiParts
constexpr int kThreads = 64 + kEpiThreads;
constexpr long long kWaitCycles = 4ll << 30;

// Tile geometry and resources for COUT outputs and tiles TZ voxels deep.
// Every 128-row M-tile accumulates its 27 taps in order, so the M-tiles are
// the independent MMA chains in flight: 16-output layers, whose small MMAs
// are bound by that chain latency, take deeper tiles (more M-tiles).
template <int COUT, int TZ, bool SWZ, bool PACK = false>
struct TileLayout {
  static constexpr int PX = TX + 2, PY = TY + 2, PZ = TZ + 2;
  static constexpr int kRows = PX * PY * PZ;                // padded tile voxels
  static constexpr int kCmin = (1 * PY + 1) * PX + 1;       // first centre
  static constexpr int kCmax = (TZ * PY + TY) * PX + TX;    // last centre
  // 128-row MMA tiles; packed: two rows of slack, which the epilogue reads
  // past the last centre
  static constexpr int kMt = (kCmax - kCmin + 1 + (PACK ? 2 : 0) + 127) / 128;
  static constexpr int kNcol = PACK ? 3 * COUT : COUT;      // accumulator columns per M-tile
  static constexpr int kDelta = PY * PX + PX + 1;           // largest tap shift
  static constexpr int kRowsAlloc = (kCmin + kMt * 128 + kDelta + 15) / 16 * 16;  // rows any MMA may read
  // SWZ: one 16-channel plane of 32-byte swizzled rows; else two 8-channel
  // planes of 16-byte rows
  static constexpr int kPlanes = SWZ ? 1 : 2;
  static constexpr uint32_t kRowBytes = SWZ ? 32 : 16;
  static constexpr uint32_t kPlane = kRowsAlloc * kRowBytes; // one plane (256-byte multiple)
  static constexpr uint32_t kBoxBytes = kRows * kRowBytes;  // what one plane's TMA load writes
  static constexpr uint32_t kB = COUT / 8 * kSboB;          // one chunk's weights
  static constexpr uint32_t kStage = (kPlanes * kPlane + kB + 1023) / 1024 * 1024;
  static constexpr int kStages = (3 * kStage <= 220 * 1024) ? 3 : 2;
  static constexpr int kAccCols = kMt * kNcol;
  static constexpr int kNacc = 2 * kAccCols <= 512 ? 2 : 1;
  static constexpr int kNcols = kNacc * kAccCols <= 32 ? 32 : kNacc * kAccCols <= 64 ? 64
                                : kNacc * kAccCols <= 128 ? 128 : kNacc * kAccCols <= 256 ? 256 : 512;
  static constexpr size_t kSmem = (size_t)kStages * kStage;
  static_assert(kRowsAlloc >= kRows, "tile rows");
  static_assert(kPlane % 256 == 0, "planes keep 256-byte (swizzle atom) alignment");
  static_assert(kAccCols <= 512, "accumulator fits the tensor memory");
  static_assert(kSmem <= 227 * 1024, "shared memory");
  static_assert(!PACK || SWZ, "the packed variant reads three taps' rows of the swizzled weight image");
  static_assert(!PACK || COUT == 16, "the packed variant serves 16 outputs");
};

// Named barrier 1 joins the epilogue warps of the packed variant;
// epi_all is the same barrier with an AND vote, so that the warps leave their
// loop together when a bounded wait gives up in any of them.
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }
__device__ __forceinline__ bool epi_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"(ok ? 1u : 0u), "n"(kEpiThreads)
      : "memory");
  return r != 0;
}

// Optional fused 1x1x1 head (16-output layers): instead of the activations,
// write yh[v] = hb + x[v][0] + sum_c hw[c] * bf16(act[v][c]) (FP32), the same
// arithmetic, in the same order, as the separate head.
struct TileHead {
  const float* hw;        // [16] weights then the bias; NULL = no head
  const bf16* x;          // network input, cx channels per voxel (channel 0 is added)
  int cx;
  float* yh;
};

struct TileGrid {
  int n, d, h, w, tz, tiles_x, tiles_y, tiles_z;
  long long tiles;
  __device__ void coords(long long t, int& b, int& x0, int& y0, int& z0) const {
    x0 = (int)(t % tiles_x) * TX; t /= tiles_x;
    y0 = (int)(t % tiles_y) * TY; t /= tiles_y;
    z0 = (int)(t % tiles_z) * tz;
    b = (int)(t / tiles_z);
  }
};

template <int COUT, int TZ, bool SWZ, bool PACK>
__global__ void __launch_bounds__(kThreads, 1) conv_tile_kernel(const __grid_constant__ CUtensorMap tmx,
                                                                const TileGrid g, int nchunks,
                                                                const bf16* __restrict__ wt,
                                                                const float* __restrict__ bias,
                                                                bf16* __restrict__ y, int ldy, int relu,
                                                                const TileHead hd, uint32_t* status) {
  typedef TileLayout<COUT, TZ, SWZ, PACK> L;
  constexpr int NC = L::kNcol;
  constexpr int S = L::kStages, NA = L::kNacc;
  constexpr int PX = L::PX, PY = L::PY, kMt = L::kMt, kCmin = L::kCmin, kCmax = L::kCmax;
  constexpr uint32_t kPlane = L::kPlane;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[S], empty[S], tfull[NA], tempty[NA];
  __shared__ uint32_t s_tmem;
  // packed, per M-tile and lane quarter: the accumulator rows of its lanes 0
  // and 1 that the previous quarter adds past its last lane (block 1 of lane
  // 0, block 2 of lanes 0 and 1), and the partial sums of its lanes 30 and 31,
  // which wait for the next quarter's rows
  __shared__ __align__(16) float s_xch[PACK ? kMt * 4 * 48 : 4];
  __shared__ __align__(16) float s_part[PACK ? kMt * 4 * 32 : 4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) tc::tmem_alloc(&s_tmem, L::kNcols);
  if (threadIdx.x == 32) {
    for (int i = 0; i < S; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < NA; ++i) {
      tc::mbar_init(&tfull[i], 1);
      tc::mbar_init(&tempty[i], kEpiThreads);
    }
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t base = tc::smem_u32(smem);
  const long long my_tiles = g.tiles > blockIdx.x ? (g.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  bool timeout = false;

  if (warp == 0) {
    // ---- producer ----------------------------------------------------------------
    if (lane == 0) {
      long long it = 0;
      for (long long k = 0; k < my_tiles && !timeout; ++k) {
        int b, x0, y0, z0;
        g.coords(blockIdx.x + k * gridDim.x, b, x0, y0, z0);
        for (int cc = 0; cc < nchunks; ++cc) {
          const int s = (int)(it % S);
          const long long u = it / S;
          if (it >= S && !tc::mbar_wait_bounded(&empty[s], (uint32_t)((u - 1) & 1), kWaitCycles)) {
            timeout = true;
            break;
          }
          const uint32_t sa = base + s * L::kStage;
          tc::mbar_arrive_expect_tx(&full[s], L::kPlanes * L::kBoxBytes + L::kB);
          tc::tma_load_5d(sa, &tmx, &full[s], cc * 16, x0 - 1, y0 - 1, z0 - 1, b);
          if (!SWZ) tc::tma_load_5d(sa + kPlane, &tmx, &full[s], cc * 16 + 8, x0 - 1, y0 - 1, z0 - 1, b);
          tc::bulk_load(sa + L::kPlanes * kPlane, wt + (size_t)cc * COUT * 432, L::kB, &full[s]);
          ++it;
        }
      }
      // every copy issued has landed before the CTA can finish
      for (long long j = it > S ? it - S : 0; j < it; ++j)
        if (!tc::mbar_wait_bounded(&full[j % S], (uint32_t)((j / S) & 1), kWaitCycles)) timeout = true;
    }
  } else if (warp == 1) {
    // ---- MMA issuer --------------------------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NC, false, false);
      long long it = 0;
      for (long long k = 0; k < my_tiles && !timeout; ++k) {
        const int a = (int)(k % NA);
        if (k >= NA && !tc::mbar_wait_bounded(&tempty[a], (uint32_t)(((k / NA) - 1) & 1), kWaitCycles)) {
          timeout = true;
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = tmem + a * L::kAccCols;
        for (int cc = 0; cc < nchunks; ++cc) {
          const int s = (int)(it % S);
          if (!tc::mbar_wait_bounded(&full[s], (uint32_t)((it / S) & 1), kWaitCycles)) {
            timeout = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = base + s * L::kStage;
          const uint32_t sb = sa + L::kPlanes * kPlane;
          // Descriptors differ only in the start-address field (bits 0-13, in
          // 16-byte units, no carry out for shared-memory addresses): build
          // two once and offset them by compile-time constants, so that the
          // issuing thread spends a few instructions per MMA.
          const uint64_t a_base = SWZ ? tc::smem_desc_sw32(sa, 256) : tc::smem_desc(sa, kPlane, 128);
          const uint64_t b_base = SWZ ? tc::smem_desc_sw32(sb, 256) : tc::smem_desc(sb, 128, kSboB);
          const uint32_t first = cc != 0;
          // packed: the three x-taps of a (dz, dy) pair in one MMA, the voxel
          // operand shifted for the first (dx = -1)
#pragma unroll
          for (int it2 = 0; it2 < (PACK ? 9 : 27); ++it2) {
            const int tap = PACK ? 3 * it2 : it2;
            const int delta = ((tap / 9 - 1) * PY + ((tap / 3) % 3 - 1)) * PX + (tap % 3 - 1);
            const uint64_t bdesc = b_base + (uint64_t)((SWZ ? tap * COUT * 32 : tap * 256) >> 4);
#pragma unroll
            for (int mt = 0; mt < kMt; ++mt) {
              const uint64_t adesc = a_base + (uint64_t)(((kCmin + mt * 128 + delta) * (int)L::kRowBytes) >> 4);
              tc::mma_bf16(acc + mt * NC, adesc, bdesc, idesc, it2 == 0 ? first : 1u);
            }
          }
          tc::mma_commit(&empty[s]);
          ++it;
        }
        if (timeout) break;
        tc::mma_commit(&tfull[a]);
      }
      // the MMAs issued last have completed before the tensor memory is freed
      if (it > 0 && !tc::mbar_wait_bounded(&empty[(it - 1) % S], (uint32_t)(((it - 1) / S) & 1), kWaitCycles))
        timeout = true;
    }
  } else {
    // ---- epilogue ----------------------------------------------------------------
    const int q = warp & 3;                  // TMEM lane quarter of this warp
    const int part = (warp - 2) >> 2;        // this warp's M-tiles: mt = part modulo kEpiParts
    const uint32_t lanes = tmem + ((uint32_t)(q * 32) << 16);
    // padded-tile coordinates of centre c packed as pz << 16 | py << 8 | px,
    // or -1 when c is not a centre of the tile
    auto centre_code = [](int c) {
      const int pz = c / (PY * PX), py = (c / PX) % PY, px = c % PX;
      return c >= kCmin && c <= kCmax && px >= 1 && px <= TX && py >= 1 && py <= TY && pz >= 1 && pz <= TZ
                 ? (pz << 16) | (py << 8) | px
                 : -1;
    };
    if constexpr (PACK) {
      // Output row r = block 0 of row r + block 1 of row r + 1 + block 2 of
      // row r + 2.  One pass over this warp's M-tiles: lanes 0-29 finish with
      // two shuffles; lanes 0 and 1 export the rows the previous quarter
      // needs and lanes 30 and 31 park their partial sums; the accumulator is
      // released; after one barrier every parked row is finished by one
      // thread.  The next tile's opening barrier orders the reuse of the
      // exchange rows.
      constexpr int kSlots = (kMt + kEpiParts - 1) / kEpiParts;   // M-tiles per warp (at most)
      static_assert(kMt * 8 <= kEpiThreads, "one parked row per thread");
      float bs[16], hw[17];                  // biases and the head's weights, per kernel
#pragma unroll
      for (int j = 0; j < 16; ++j) bs[j] = bias ? __ldg(bias + j) : 0.0f;
#pragma unroll
      for (int j = 0; j < 17; ++j) hw[j] = hd.hw ? __ldg(hd.hw + j) : 0.0f;
      int pc[kSlots];                        // this lane's centre in each of its M-tiles
#pragma unroll
      for (int i = 0; i < kSlots; ++i) pc[i] = centre_code(kCmin + (kEpiParts * i + part) * 128 + q * 32 + lane);
      const int item = threadIdx.x - 64;     // the parked row this thread finishes
      const int imq = item >> 1, il2 = item & 1;
      const int icode = item < kMt * 8 ? centre_code(kCmin + (imq >> 2) * 128 + (imq & 3) * 32 + 30 + il2) : -1;
      for (long long k = 0; k < my_tiles; ++k) {
        const int a = (int)(k % NA);
        bool got = tc::mbar_wait_bounded(&tfull[a], (uint32_t)((k / NA) & 1), kWaitCycles);
        got = epi_all(got);                  // the warps meet at barriers below: decide together
        if (!got) {
          timeout = true;
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = lanes + a * L::kAccCols;
        int b, x0, y0, z0;
        g.coords(blockIdx.x + k * gridDim.x, b, x0, y0, z0);
        auto voxel = [&](int code, long long& vox) {
          const int gz = z0 + (code >> 16) - 1, gy = y0 + ((code >> 8) & 255) - 1, gx = x0 + (code & 255) - 1;
          vox = (((long long)b * g.d + gz) * g.h + gy) * g.w + gx;
          return code >= 0 && gz < g.d && gy < g.h && gx < g.w;
        };
        // bias, ReLU, BF16 and the 32-byte store (or the fused head's dot
        // product, in the order of the separate head)
        auto emit16 = [&](const float (&v)[16], long long vox) {
          if (hd.hw) {
            float out = hw[16] + __bfloat162float(hd.x[vox * hd.cx]);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float tv = v[j] + bs[j];
              if (relu) tv = fmaxf(tv, 0.0f);
              out = fmaf(__bfloat162float(__float2bfloat16_rn(tv)), hw[j], out);
            }
            hd.yh[vox] = out;
            return;
          }
          uint32_t o[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float t0 = v[2 * j] + bs[2 * j], t1 = v[2 * j + 1] + bs[2 * j + 1];
            if (relu) {
              t0 = fmaxf(t0, 0.0f);
              t1 = fmaxf(t1, 0.0f);
            }
            const __nv_bfloat162 p = __floats2bfloat162_rn(t0, t1);   // t0 in the low half
            o[j] = *reinterpret_cast<const uint32_t*>(&p);
          }
          uint4* dst = reinterpret_cast<uint4*>(y + vox * ldy);
          dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
          dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
        };
#pragma unroll
        for (int i = 0; i < kSlots; ++i) {
          const int mt = kEpiParts * i + part;
          if (mt >= kMt) break;              // warp-uniform
          float v[16], v2[16], v3[16];
          __syncwarp();
          tc::tmem_ld16x3(acc + mt * NC, acc + mt * NC + 16, acc + mt * NC + 32, v, v2, v3);
          float4* xb = reinterpret_cast<float4*>(s_xch + (mt * 4 + q) * 48);
          if (lane == 0) {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              xb[m] = make_float4(v2[4 * m], v2[4 * m + 1], v2[4 * m + 2], v2[4 * m + 3]);
              xb[4 + m] = make_float4(v3[4 * m], v3[4 * m + 1], v3[4 * m + 2], v3[4 * m + 3]);
            }
          } else if (lane == 1) {
#pragma unroll
            for (int m = 0; m < 4; ++m) xb[8 + m] = make_float4(v3[4 * m], v3[4 * m + 1], v3[4 * m + 2], v3[4 * m + 3]);
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float n2 = __shfl_down_sync(0xffffffffu, v2[j], 1);
            const float n3 = __shfl_down_sync(0xffffffffu, v3[j], 2);
            v[j] += lane < 31 ? n2 : 0.0f;
            v[j] += lane < 30 ? n3 : 0.0f;
          }
          long long vox;
          if (lane >= 30) {
            float4* pp = reinterpret_cast<float4*>(s_part + ((mt * 4 + q) * 2 + lane - 30) * 16);
#pragma unroll
            for (int m = 0; m < 4; ++m) pp[m] = make_float4(v[4 * m], v[4 * m + 1], v[4 * m + 2], v[4 * m + 3]);
          } else if (voxel(pc[i], vox)) {
            emit16(v, vox);
          }
        }
        tc::fence_before_sync();
        tc::mbar_arrive(&tempty[a]);         // the accumulator has been read
        epi_sync();
        long long vox;
        if (voxel(icode, vox)) {             // the last quarter's parked rows are never centres
          const float4* xb = reinterpret_cast<const float4*>(s_xch + (imq + 1) * 48);
          const float4* pp = reinterpret_cast<const float4*>(s_part + item * 16);
          float v[16];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const float4 p = pp[m];
            if (il2) {                       // lane 31: rows r + 1 and r + 2 are the next quarter's lanes 0, 1
              const float4 n2 = xb[m], n3 = xb[8 + m];
              v[4 * m] = (p.x + n2.x) + n3.x;
              v[4 * m + 1] = (p.y + n2.y) + n3.y;
              v[4 * m + 2] = (p.z + n2.z) + n3.z;
              v[4 * m + 3] = (p.w + n2.w) + n3.w;
            } else {                         // lane 30: row r + 2 is the next quarter's lane 0
              const float4 n3 = xb[4 + m];
              v[4 * m] = p.x + n3.x;
              v[4 * m + 1] = p.y + n3.y;
              v[4 * m + 2] = p.z + n3.z;
              v[4 * m + 3] = p.w + n3.w;
            }
          }
          emit16(v, vox);
        }
      }
    } else {
      for (long long k = 0; k < my_tiles; ++k) {
        const int a = (int)(k % NA);
        // the warp leaves together (tcgen05.ld below is warp-collective)
        if (!__all_sync(0xffffffffu, tc::mbar_wait_bounded(&tfull[a], (uint32_t)((k / NA) & 1), kWaitCycles))) {
          timeout = true;
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = lanes + a * L::kAccCols;
        int b, x0, y0, z0;
        g.coords(blockIdx.x + k * gridDim.x, b, x0, y0, z0);
        for (int mt = part; mt < kMt; mt += kEpiParts) {
          const int code = centre_code(kCmin + mt * 128 + q * 32 + lane);   // this lane's centre
          const int gz = z0 + (code >> 16) - 1, gy = y0 + ((code >> 8) & 255) - 1, gx = x0 + (code & 255) - 1;
          const long long vox = (((long long)b * g.d + gz) * g.h + gy) * g.w + gx;
          const bool ok = code >= 0 && gz < g.d && gy < g.h && gx < g.w;
#pragma unroll
          for (int cq = 0; cq < COUT / 16; ++cq) {
            float v[16];
            __syncwarp();
            tc::tmem_ld16(acc + mt * NC + cq * 16, v);
            if (ok && COUT == 16 && hd.hw) {  // fused head: the order of the separate head
              float out = __ldg(hd.hw + 16) + __bfloat162float(hd.x[vox * hd.cx]);
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                float tv = v[j] + (bias ? __ldg(bias + j) : 0.0f);
                if (relu) tv = fmaxf(tv, 0.0f);
                out = fmaf(__bfloat162float(__float2bfloat16_rn(tv)), __ldg(hd.hw + j), out);
              }
              hd.yh[vox] = out;
            } else if (ok) {
              __align__(16) bf16 o[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                float tv = v[j] + (bias ? __ldg(bias + cq * 16 + j) : 0.0f);
                if (relu) tv = fmaxf(tv, 0.0f);
                o[j] = __float2bfloat16_rn(tv);
              }
              uint4* dst = reinterpret_cast<uint4*>(y + vox * ldy + cq * 16);
              dst[0] = reinterpret_cast<uint4*>(o)[0];
              dst[1] = reinterpret_cast<uint4*>(o)[1];
            }
          }
        }
        tc::fence_before_sync();
        tc::mbar_arrive(&tempty[a]);
      }
    }
  }
  if (timeout) atomicOr(status, NM_DEV_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, L::kNcols);
}

// Weights [cout][kpad] (K index tap * cin + c) -> per 16-channel chunk the
// shared-memory image of the B operand, zero for channels >= cin:
//   swz:  [chunk][27 taps][cout rows][2 halves of 8 channels], the halves of
//         row co exchanged when bit 2 of co is set (32-byte swizzle);
//   else: [chunk][cout / 8][27 taps x 2 halves][8 rows][8 channels].
__global__ void tile_weights_kernel(const bf16* __restrict__ w, int cin, int kpad, int cout, int nchunks, int swz,
                                    bf16* __restrict__ out) {
  const long long total = (long long)nchunks * cout * 432;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i % 8);
    long long t = i / 8;
    int co, tap, half, cc;
    if (swz) {
      const int pos = (int)(t % 2); t /= 2;
      co = (int)(t % cout); t /= cout;
      tap = (int)(t % 27);
      cc = (int)(t / 27);
      half = pos ^ ((co >> 2) & 1);
    } else {
      const int r = (int)(t % 8); t /= 8;
      const int kc = (int)(t % 54); t /= 54;
      const int grp = (int)(t % (cout / 8));
      cc = (int)(t / (cout / 8));
      co = grp * 8 + r;
      tap = kc >> 1;
      half = kc & 1;
    }
    const int ch = cc * 16 + half * 8 + e;
    out[i] = ch < cin ? w[(long long)co * kpad + tap * cin + ch] : __float2bfloat16_rn(0.0f);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  return n;
}

// y: output voxel v's channels at y + v ldy (ldy = COUT, or the full width
// when a wider convolution is computed COUT outputs at a time).
template <int COUT, int TZ, bool SWZ, bool PACK = false>
cudaError_t launch_tile(const nm_conv3d_desc& d, const void* x, const void* w, const float* bias, void* y,
                        int relu, const TileHead& hd, uint32_t* status, cudaStream_t s, int ldy = COUT) {
  typedef TileLayout<COUT, TZ, SWZ, PACK> L;
  const int cin = d.c0;
  const int nchunks = (cin + 15) / 16;
  // the input as a 5-D tensor (c, x, y, z, n); boxes of 8 channels x the padded tile
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[5] = {(cuuint64_t)cin, (cuuint64_t)d.w, (cuuint64_t)d.h, (cuuint64_t)d.d, (cuuint64_t)d.n};
  const cuuint64_t strides[4] = {(cuuint64_t)cin * 2, (cuuint64_t)d.w * cin * 2, (cuuint64_t)d.h * d.w * cin * 2,
                                 (cuuint64_t)d.d * d.h * d.w * cin * 2};
  const cuuint32_t box[5] = {SWZ ? 16u : 8u, (cuuint32_t)L::PX, (cuuint32_t)L::PY, (cuuint32_t)L::PZ, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, SWZ ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  bf16* wt = nullptr;
  const size_t welems = (size_t)nchunks * COUT * 432;
  cudaError_t e = cudaMallocAsync((void**)&wt, welems * sizeof(bf16), s);
  if (e != cudaSuccess) return e;
  tile_weights_kernel<<<(unsigned)std::min<size_t>((welems + 255) / 256, 4096), 256, 0, s>>>(
      (const bf16*)w, cin, conv_kpad(cin), COUT, nchunks, SWZ ? 1 : 0, wt);
  TileGrid g;
  g.n = d.n; g.d = d.d; g.h = d.h; g.w = d.w;
  g.tiles_x = (d.w + TX - 1) / TX;
  g.tiles_y = (d.h + TY - 1) / TY;
  g.tz = TZ;
  g.tiles_z = (d.d + TZ - 1) / TZ;
  g.tiles = (long long)g.tiles_x * g.tiles_y * g.tiles_z * g.n;
  e = cudaFuncSetAttribute(conv_tile_kernel<COUT, TZ, SWZ, PACK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)L::kSmem);
  if (e == cudaSuccess) {
    const long long grid = std::min<long long>(g.tiles, sm_count());
    conv_tile_kernel<COUT, TZ, SWZ, PACK><<<(unsigned)grid, kThreads, L::kSmem, s>>>(map, g, nchunks, wt, bias,
                                                                                      (bf16*)y, ldy, relu, hd,
                                                                                      status);
    e = cudaGetLastError();
  }
  cudaFreeAsync(wt, s);
  return e;
}

}  // namespace

namespace {

// An mbarrier that nothing ever arrives on, waited for with the bounded wait
// of the tensor-core kernels: the wait must give up after max_cycles and
// record NM_DEV_TIMEOUT, leaving the context usable.
__global__ void check_wait_kernel(long long max_cycles, uint32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait_bounded(&bar, 0, max_cycles)) atomicOr(status, NM_DEV_TIMEOUT);
}

}  // namespace

cudaError_t launch_check_wait(long long max_cycles, uint32_t* status, cudaStream_t s) {
  check_wait_kernel<<<1, 32, 0, s>>>(max_cycles, status);
  return cudaGetLastError();
}

bool conv_tile_ok(const nm_conv3d_desc& d) {
  return d.c1 == 0 && !d.src0_coarse && d.c0 % 8 == 0 &&
         (d.cout == 16 || d.cout == 32 || d.cout == 48 || d.cout == 64 || d.cout == 96 || d.cout == 192);
}

// The packed variant serves 16 outputs; NM_CONV_TILE_UNPACKED=1 selects the
// one-tap-per-MMA form instead (both are tested).  With 32 outputs the packed
// form measured no faster: its accumulators (N = 96 per M-tile) leave room for
// one in the tensor memory, so the MMAs of a tile wait for the previous
// tile's epilogue.
static bool packed_tiles() {
  const char* e = getenv("NM_CONV_TILE_UNPACKED");
  return !(e && e[0] == '1');
}

cudaError_t conv3d_fwd_tile(const nm_conv3d_desc& d, const void* x, const void* w, const float* bias, void* y,
                            int relu, uint32_t* status, cudaStream_t s) {
  constexpr bool kSwz = true;
  const TileHead none{nullptr, nullptr, 0, nullptr};
  if (d.cout == 16 && packed_tiles()) return launch_tile<16, 2, kSwz, true>(d, x, w, bias, y, relu, none, status, s);
  if (d.cout == 16) return launch_tile<16, 4, kSwz>(d, x, w, bias, y, relu, none, status, s);
  if (d.cout == 32) return launch_tile<32, 2, kSwz>(d, x, w, bias, y, relu, none, status, s);
  if (d.cout == 48) return launch_tile<48, 2, kSwz>(d, x, w, bias, y, relu, none, status, s);
  if (d.cout == 64) return launch_tile<64, 2, kSwz>(d, x, w, bias, y, relu, none, status, s);
  // 96 and 192 outputs (input gradients of the decoders' two-source layers):
  // 48 or 64 output channels per launch, written at the full channel stride
  const int P = d.cout == 96 ? 48 : 64;
  nm_conv3d_desc dp = d;
  dp.cout = P;
  for (int p = 0; p < d.cout / P; ++p) {
    const void* wp = (const bf16*)w + (size_t)p * P * conv_kpad(d.c0);
    const float* bp = bias ? bias + p * P : nullptr;
    void* yp = (bf16*)y + p * P;
    const cudaError_t e = P == 48 ? launch_tile<48, 2, kSwz>(dp, x, wp, bp, yp, relu, none, status, s, d.cout)
                                  : launch_tile<64, 2, kSwz>(dp, x, wp, bp, yp, relu, none, status, s, d.cout);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t conv3d_fwd_tile_head(const nm_conv3d_desc& d, const void* x, const void* w, const float* bias,
                                 const float* head_w, const void* xin, int cx, float* yh, uint32_t* status,
                                 cudaStream_t s) {
  if (d.cout != 16 || !conv_tile_ok(d)) return cudaErrorInvalidValue;
  const TileHead hd{head_w, (const bf16*)xin, cx, yh};
  if (packed_tiles()) return launch_tile<16, 2, true, true>(d, x, w, bias, nullptr, 1, hd, status, s);
  return launch_tile<16, 4, true>(d, x, w, bias, nullptr, 1, hd, status, s);
}

}  // namespace nm
