// Weight gradient of a 3x3x3 convolution by shifted windows:
//   dW[co][tap][ci] = sum over voxels v of dY[v][co] * X[v + off_tap][ci].
//
// A GEMM over voxels (K) with M = output channels and N = 16-channel chunks
// of input channels.  Both operands come from halo tiles in shared memory in
// the 32-byte-swizzled MN-major layout (a voxel row of 16 channels, 32 bytes),
// loaded by TMA: dY over the tile's z-planes, X with its one-voxel halo.  dY
// is zeroed at the halo positions (they belong to other tiles), so K may run
// over padded rows.  Substituting v' = v + off moves the tap's shift from X to
// dY: sum over v' of dY[v' - off][co] X[v'][ci].  The three taps dx = +1, 0,
// -1 of one (dy, dz) pair then read dY at three consecutive rows, which one
// MMA covers: its M = 64 operand is four 16-row atoms (16 output channels
// each) at a leading-byte offset of one row (32 bytes), so atom q reads dY
// shifted by q rows (taps dx = 1 - q; the fourth atom's rows of D are never
// read).  Per tile 9 (dy, dz) groups x 39 K-steps of 16 voxel rows; X moves
// by the group's (dz PY + dy) PX rows.  N = 16, 32 or 48 input channels per
// MMA; the groups' accumulators stay in TMEM across all of a CTA's tiles.
// With one input chunk (N = 16) the three (dy) groups of one dz read X at
// shifts PX rows apart, so one MMA of N = 48 covers them: its B operand is
// three 16-channel atoms of the same chunk at a leading-byte offset of PX
// rows (dy = -1, 0, +1), and a tile takes 3 x 39 MMAs instead of 9 x 39.
//
// Persistent, warp-specialised (one CTA per SM), passes over groups of input
// chunks (and of (dy, dz) groups where TMEM needs it):
//   warp 0    TMA producer (dY atoms + the pass's X chunks per tile) into a stage ring;
//   warp 1    MMA issuer: per tile the pass's groups x 39 K-steps, commits to "empty";
//   warps 2-5 zero dY's halo rows of each landed stage (then "ready"), and at
//             the end of a pass the warps whose TMEM lane quarters hold the
//             taps dx = +1, 0, -1 (warps 4, 5, 2) write the CTA's partial dW.
// Partials are summed over CTAs in a fixed order by the caller (deterministic);
// the bias gradient is a separate fixed-order reduction.  Every wait is
// bounded; a time-out sets NM_DEV_TIMEOUT and drains what is in flight.
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

constexpr int TX = 16, TY = 16, TZ = 2;
constexpr int PX = TX + 2, PY = TY + 2, PZ = TZ + 2;
constexpr int kRows = PX * PY * PZ;                          // X box rows
constexpr int kCmin = (1 * PY + 1) * PX + 1;                 // first centre
constexpr int kCmax = (TZ * PY + TY) * PX + TX;              // last centre
constexpr int kKRows = ((kCmax - kCmin + 1 + 127) / 128) * 128;  // K rows per tile (640)
constexpr int kDelta = PY * PX + PX + 1;                     // largest tap shift
constexpr int kXRows = (kCmin + kKRows + kDelta + 15) / 16 * 16;  // rows any MMA may read from X
constexpr int kYOff = PY * PX;                               // dY box starts one z-plane in
constexpr int kYBox = PX * PY * TZ;                          // dY box rows
constexpr int kYRows = (kCmin - kYOff + kKRows + 15) / 16 * 16;   // rows read from dY (>= kYBox)
// the three x-taps of a group: X rows from kCmin - 1 + group shift, 612 of them
constexpr int kKSteps3 = (kCmax - kCmin + 1 + 2 + 15) / 16;  // 39
constexpr int kARow0 = kCmin - 1 - 1 - kYOff;               // dY row of atom 0 (dx = +1) at K row 0
static_assert(kARow0 >= 0 && kARow0 + kKSteps3 * 16 + 3 <= kYBox, "dY rows of the shifted atoms");
static_assert(kCmin - 1 - (PY + 1) * PX >= 0 && kCmin - 1 + (PY + 1) * PX + kKSteps3 * 16 <= kXRows,
              "X rows of the groups");
constexpr uint32_t kXBytes = kXRows * 32;
constexpr uint32_t kYBytes = kYRows * 32;
constexpr int kThreads = 192;
constexpr long long kWaitCycles = 4ll << 30;
constexpr int kBiasBlocks = 256;

static_assert(kXRows >= kRows && kYRows >= kYBox, "tile rows");

// G = input-channel atoms (16 channels each) per MMA: N = 16 G.  With more
// atoms one MMA covers more of the input channels, so fewer instructions are
// issued (their rate, not the tensor math, bounds these small GEMMs); the
// (dy, dz) groups of a pass are limited by TMEM (groups x output halves x
// 16 G columns <= 512).
// DY: one chunk, the three dy groups of a dz in one MMA (groups are then the
// three dz, N = 48).
template <int COUT, int G, bool DY = false>
struct WLayout {
  static_assert(!DY || G == 1, "dy packing takes one input chunk per MMA");
  static constexpr int kYAtoms = COUT / 16;
  static constexpr int kN = DY ? 48 : 16 * G;             // accumulator columns per group and output atom
  static constexpr int kGroups = DY ? 3 : 512 / (16 * G * kYAtoms) < 9 ? 512 / (16 * G * kYAtoms) : 9;
  static constexpr int kAllGroups = DY ? 3 : 9;
  static_assert(kGroups * kYAtoms * kN <= 512, "accumulators fit the tensor memory");
  static constexpr uint32_t kUsed = kYAtoms * kYBytes + G * kXBytes;
  static constexpr uint32_t kSpan = kUsed;
  static constexpr uint32_t kStage = (kSpan + 1023) / 1024 * 1024;
  static constexpr int kStages = 3 * kStage <= 220 * 1024 ? 3 : 2 * kStage <= 220 * 1024 ? 2 : 1;
  static constexpr size_t kSmem = (size_t)kStages * kStage;
  static_assert(kSmem <= 227 * 1024, "shared memory");
};

struct WGrid {
  int n, d, h, w, tiles_x, tiles_y, tiles_z, cin, kpad;
  long long tiles;
  __device__ void coords(long long t, int& b, int& x0, int& y0, int& z0) const {
    x0 = (int)(t % tiles_x) * TX; t /= tiles_x;
    y0 = (int)(t % tiles_y) * TY; t /= tiles_y;
    z0 = (int)(t % tiles_z) * TZ;
    b = (int)(t / tiles_z);
  }
};

__device__ __forceinline__ uint64_t desc_mn_sw32(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  // MN-major, 32-byte swizzle: LBO = stride between 16-element atoms along
  // M/N, SBO = stride between groups of 8 K rows (checked on the device)
  return tc::smem_desc(saddr, lbo, sbo) | ((uint64_t)6 << 61);
}

template <int COUT, int G, bool DY>
__global__ void __launch_bounds__(kThreads, 1) wgrad_tile_kernel(const __grid_constant__ CUtensorMap tmx,
                                                                 const __grid_constant__ CUtensorMap tmy,
                                                                 const WGrid g, float* __restrict__ part,
                                                                 uint32_t* status) {
  typedef WLayout<COUT, G, DY> L;
  constexpr int S = L::kStages, GP = L::kGroups, NG = L::kAllGroups, NN = L::kN;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[S], ready[S], empty[S], acc_full, acc_empty;
  __shared__ uint32_t s_tmem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (g.cin + 15) / 16;
  const long long my_tiles = g.tiles > blockIdx.x ? (g.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  // passes: groups of G input chunks x runs of GP (dy, dz) groups
  const int n_tg = (NG + GP - 1) / GP;
  const int passes = (nchunks + G - 1) / G * n_tg;

  if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
  // rows past the TMA boxes are read by the last K-steps but never loaded:
  // zero them once per stage (dY there must be 0; X must at least be finite)
  for (int i = threadIdx.x; i < S * L::kYAtoms * (kYRows - kYBox) * 2; i += blockDim.x) {
    const int half = i & 1, r = kYBox + (i >> 1) % (kYRows - kYBox);
    const int rest = (i >> 1) / (kYRows - kYBox);
    const int atom = rest % L::kYAtoms, s = rest / L::kYAtoms;
    *reinterpret_cast<uint4*>(smem + s * L::kStage + atom * kYBytes + r * 32 + half * 16) = make_uint4(0, 0, 0, 0);
  }
  for (int i = threadIdx.x; i < S * G * (kXRows - kRows) * 2; i += blockDim.x) {
    const int half = i & 1, r = kRows + (i >> 1) % (kXRows - kRows);
    const int rest = (i >> 1) / (kXRows - kRows), a = rest % G, s = rest / G;
    *reinterpret_cast<uint4*>(smem + s * L::kStage + L::kYAtoms * kYBytes + a * kXBytes + r * 32 + half * 16) =
        make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < S; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&ready[i], 128);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(&acc_full, 1);
    tc::mbar_init(&acc_empty, 96);
    tc::mbar_fence_init();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t base = tc::smem_u32(smem);
  bool timeout = false;

  if (warp == 0) {
    // ---- producer: for every pass (input chunk), every tile ------------------
    if (lane == 0) {
      long long it = 0;
      for (int ps = 0; ps < passes && !timeout; ++ps) {
        const int c0 = ps / n_tg * G, na = min(G, nchunks - c0);
        for (long long k = 0; k < my_tiles; ++k, ++it) {
          const int s = (int)(it % S);
          if (it >= S && !tc::mbar_wait_bounded(&empty[s], (uint32_t)(((it / S) - 1) & 1), kWaitCycles)) {
            timeout = true;
            break;
          }
          int b, x0, y0, z0;
          g.coords(blockIdx.x + k * gridDim.x, b, x0, y0, z0);
          const uint32_t sa = base + s * L::kStage;
          tc::mbar_arrive_expect_tx(&full[s], (L::kYAtoms * kYBox + na * kRows) * 32);
          for (int q = 0; q < L::kYAtoms; ++q)
            tc::tma_load_5d(sa + q * kYBytes, &tmy, &full[s], q * 16, x0 - 1, y0 - 1, z0, b);
          for (int a = 0; a < na; ++a)
            tc::tma_load_5d(sa + L::kYAtoms * kYBytes + a * kXBytes, &tmx, &full[s], (c0 + a) * 16, x0 - 1,
                            y0 - 1, z0 - 1, b);
        }
      }
      for (long long j = it > S ? it - S : 0; j < it; ++j)
        if (!tc::mbar_wait_bounded(&full[j % S], (uint32_t)((j / S) & 1), kWaitCycles)) timeout = true;
    }
  } else if (warp == 1) {
    // ---- MMA issuer -------------------------------------------------------------------
    if (lane == 0) {
      long long it = 0;
      for (int ps = 0; ps < passes && !timeout; ++ps) {
        const int c0 = ps / n_tg * G, na = min(G, nchunks - c0);
        const int g0 = ps % n_tg * GP, g1 = min(NG, g0 + GP);
        const uint32_t idesc = tc::idesc_bf16_f32(64, DY ? 48 : 16 * na, true, true);
        // the previous pass's accumulators have been read out
        if (ps > 0 && !tc::mbar_wait_bounded(&acc_empty, (uint32_t)((ps - 1) & 1), kWaitCycles)) {
          timeout = true;
          break;
        }
        tc::fence_after_sync();
        for (long long k = 0; k < my_tiles; ++k, ++it) {
          const int s = (int)(it % S);
          if (!tc::mbar_wait_bounded(&ready[s], (uint32_t)((it / S) & 1), kWaitCycles)) {
            timeout = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sy = base + s * L::kStage;
          const uint32_t sx = sy + L::kYAtoms * kYBytes;
          const uint32_t first = k == 0 ? 0u : 1u;
          for (int ks = 0; ks < kKSteps3; ++ks) {
            for (int g = g0; g < g1; ++g) {
              // group g = (dz + 1) 3 + (dy + 1), X rows from kCmin - 1 + shift;
              // DY: group g = dz + 1, atoms dy = -1, 0, +1 from the dy = -1 shift
              const int shift = DY ? ((g - 1) * PY - 1) * PX : ((g / 3 - 1) * PY + (g % 3 - 1)) * PX;
              const uint64_t bdesc =
                  desc_mn_sw32(sx + (kCmin - 1 + shift + ks * 16) * 32, DY ? PX * 32 : kXBytes, 256);
#pragma unroll
              for (int h = 0; h < L::kYAtoms; ++h) {
                const uint64_t adesc = desc_mn_sw32(sy + h * kYBytes + (kARow0 + ks * 16) * 32, 32, 256);
                tc::mma_bf16(tmem + ((g - g0) * L::kYAtoms + h) * NN, adesc, bdesc, idesc, ks == 0 ? first : 1u);
              }
            }
          }
          tc::mma_commit(&empty[s]);
        }
        if (timeout) break;
        tc::mma_commit(&acc_full);
      }
      if (it > 0 && !tc::mbar_wait_bounded(&empty[(it - 1) % S], (uint32_t)(((it - 1) / S) & 1), kWaitCycles))
        timeout = true;
    }
  } else {
    // ---- halo zeroing, and the partial dW at the end of each pass -----------------
    const int t = threadIdx.x - 64;                  // 0..127
    long long it = 0;
    for (int ps = 0; ps < passes && !timeout; ++ps) {
      const int c0 = ps / n_tg * G, na = min(G, nchunks - c0);
      const int g0 = ps % n_tg * GP, g1 = min(NG, g0 + GP);
      for (long long k = 0; k < my_tiles; ++k, ++it) {
        const int s = (int)(it % S);
        const bool got = tc::mbar_wait_bounded(&full[s], (uint32_t)((it / S) & 1), kWaitCycles);
        if (!__all_sync(0xffffffffu, got)) {
          timeout = true;
          break;
        }
        // dY rows of x or y halo positions (2 z-planes x 68): zero both 16-byte halves
        uint8_t* sy = smem + s * L::kStage;
        for (int i = t; i < L::kYAtoms * TZ * 68 * 2; i += 128) {
          const int half = i & 1, j = (i >> 1) % (TZ * 68), atom = (i >> 1) / (TZ * 68);
          const int zp = j / 68, h = j % 68;
          int xp, yp;
          if (h < 18) { yp = 0; xp = h; }
          else if (h < 36) { yp = PY - 1; xp = h - 18; }
          else { yp = 1 + (h - 36) / 2; xp = (h & 1) ? PX - 1 : 0; }
          const int r = (zp * PY + yp) * PX + xp;
          *reinterpret_cast<uint4*>(sy + atom * kYBytes + r * 32 + half * 16) = make_uint4(0, 0, 0, 0);
        }
        tc::fence_async_smem();
        tc::mbar_arrive(&ready[s]);
      }
      if (timeout) break;
      // end of the pass: with M = 64, D row i sits in TMEM lane (i % 16) +
      // 32 (i / 16), so atom q (tap dx = 1 - q) is lanes 0-15 of quarter q,
      // read by the warp of that quarter (warp 4: q 0, 5: 1, 2: 2; quarter 3
      // holds the unused fourth atom)
      const int q = warp & 3;
      if (q != 3) {
        const bool got = tc::mbar_wait_bounded(&acc_full, (uint32_t)(ps & 1), kWaitCycles);
        if (!__all_sync(0xffffffffu, got)) {
          timeout = true;
          break;
        }
        tc::fence_after_sync();
        float* dst = part + (size_t)blockIdx.x * g.kpad * COUT;
        for (int gg = g0; gg < g1; ++gg) {
          for (int h = 0; h < L::kYAtoms; ++h)
            for (int a = 0; a < (DY ? 3 : na); ++a) {
              // the column atom a is input chunk c0 + a, or with DY tap dy = a - 1
              const int grp = DY ? gg * 3 + a : gg;          // (dz + 1) 3 + (dy + 1)
              const int tap = grp * 3 + (2 - q);             // (dz + 1) 9 + (dy + 1) 3 + (dx + 1)
              const int cc = DY ? c0 : c0 + a;
              float v[16];
              tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + ((gg - g0) * L::kYAtoms + h) * NN + a * 16, v);
              if (lane < 16)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  const int ci = cc * 16 + j;
                  if (ci < g.cin) dst[(size_t)(tap * g.cin + ci) * COUT + h * 16 + lane] = v[j];
                }
            }
        }
        tc::fence_before_sync();
        tc::mbar_arrive(&acc_empty);
      }
    }
  }
  if (timeout) atomicOr(status, NM_DEV_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Bias gradient db[co] = sum over voxels of dY[v][co].  Each thread sums one
// 8-channel octet of a fixed, strided set of voxels (16-byte loads); a
// block's threads of one octet are added in thread order, the blocks by
// bias_grad_final in a fixed order.
template <int COUT>
__global__ void __launch_bounds__(256) bias_grad_partial(const bf16* __restrict__ dy, long long m,
                                                         float* __restrict__ part) {
  constexpr int L = COUT / 8;       // octets per voxel
  constexpr int VPB = 256 / L;      // voxels per block and step
  __shared__ float red[256][9];
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
  const int oct = threadIdx.x % L;
  for (long long v = (long long)blockIdx.x * VPB + threadIdx.x / L; v < m; v += (long long)gridDim.x * VPB) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(dy + v * COUT) + oct);
    const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 f = __bfloat1622float2(e[j]);
      acc[2 * j] += f.x;
      acc[2 * j + 1] += f.y;
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) red[threadIdx.x][j] = acc[j];
  __syncthreads();
  if (threadIdx.x < COUT) {
    const int o = threadIdx.x / 8, j = threadIdx.x % 8;
    float s = 0.0f;
    for (int t = o; t < 256; t += L) s += red[t][j];
    part[(size_t)blockIdx.x * COUT + threadIdx.x] = s;
  }
}

// One warp per channel: lanes strided over the blocks, then a fixed tree.
__global__ void bias_grad_final(const float* __restrict__ part, int blocks, int cout, float* __restrict__ db) {
  const int c = blockIdx.x, lane = threadIdx.x;
  float s = 0.0f;
  for (int b = lane; b < blocks; b += 32) s += part[(size_t)b * cout + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) db[c] = s;
}

// dW = the CTAs' partials part[cta][k][co] summed in a fixed order: per
// element, eight warps each add a contiguous run of CTAs, then the runs are
// added in order.  A warp reads 32 consecutive floats of the (k, co) layout.
__global__ void __launch_bounds__(256) wgrad_tile_reduce(const float* __restrict__ part, int splits, int kpad,
                                                         int kreal, int cout, float* __restrict__ dw) {
  __shared__ float red[8][33];
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const long long n = (long long)kpad * cout;
  const long long e = (long long)blockIdx.x * 32 + lane;
  const int per = (splits + 7) / 8;
  const int t1 = min(splits, (seg + 1) * per);
  float s = 0.0f;
  if (e < n)
    for (int t = seg * per; t < t1; ++t) s += part[(long long)t * n + e];
  red[seg][lane] = s;
  __syncthreads();
  if (seg == 0 && e < n) {
    float r = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) r += red[q][lane];
    const int k = (int)(e / cout), co = (int)(e % cout);
    dw[(long long)co * kpad + k] = k < kreal ? r : 0.0f;
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

bool encode(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map, const void* t, int c, const nm_conv3d_desc& d,
            int box_z) {
  const cuuint64_t dims[5] = {(cuuint64_t)c, (cuuint64_t)d.w, (cuuint64_t)d.h, (cuuint64_t)d.d, (cuuint64_t)d.n};
  const cuuint64_t strides[4] = {(cuuint64_t)c * 2, (cuuint64_t)d.w * c * 2, (cuuint64_t)d.h * d.w * c * 2,
                                 (cuuint64_t)d.d * d.h * d.w * c * 2};
  const cuuint32_t box[5] = {16, PX, PY, (cuuint32_t)box_z, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(t), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int COUT, int G, bool DY = false>
cudaError_t launch_wgrad_tile(const nm_conv3d_desc& d, const void* x, const void* dy, float* dw, float* db,
                              void* workspace, uint32_t* status, cudaStream_t s) {
  typedef WLayout<COUT, G, DY> L;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap mx, my;
  if (!encode(enc, &mx, x, d.c0, d, PZ) || !encode(enc, &my, dy, COUT, d, TZ)) return cudaErrorInvalidValue;
  WGrid g;
  g.n = d.n; g.d = d.d; g.h = d.h; g.w = d.w;
  g.tiles_x = (d.w + TX - 1) / TX;
  g.tiles_y = (d.h + TY - 1) / TY;
  g.tiles_z = (d.d + TZ - 1) / TZ;
  g.tiles = (long long)g.tiles_x * g.tiles_y * g.tiles_z * g.n;
  g.cin = d.c0;
  g.kpad = conv_kpad(d.c0);
  // every CTA gets at least one tile (its pass-end read-out waits for MMAs)
  const int grid = (int)std::min<long long>(g.tiles, sm_count());
  float* part = (float*)workspace;
  float* bpart = part + (size_t)grid * g.kpad * COUT;
  cudaError_t e = cudaFuncSetAttribute(wgrad_tile_kernel<COUT, G, DY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L::kSmem);
  if (e != cudaSuccess) return e;
  wgrad_tile_kernel<COUT, G, DY><<<grid, kThreads, L::kSmem, s>>>(mx, my, g, part, status);
  const long long n = (long long)g.kpad * COUT;
  wgrad_tile_reduce<<<(unsigned)((n + 31) / 32), 256, 0, s>>>(part, grid, g.kpad, 27 * d.c0, COUT, dw);
  if (db) {
    const long long m = (long long)d.n * d.d * d.h * d.w;
    bias_grad_partial<COUT><<<kBiasBlocks, 256, 0, s>>>((const bf16*)dy, m, bpart);
    bias_grad_final<<<COUT, 32, 0, s>>>(bpart, kBiasBlocks, COUT, db);
  }
  return cudaGetLastError();
}

}  // namespace

bool conv_wgrad_tile_ok(const nm_conv3d_desc& d) {
  return d.c1 == 0 && !d.src0_coarse && d.c0 % 8 == 0 && (d.cout == 16 || d.cout == 32);
}

size_t conv_wgrad_tile_workspace(const nm_conv3d_desc& d) {
  return ((size_t)sm_count() * conv_kpad(d.c0) * d.cout + (size_t)kBiasBlocks * d.cout) * sizeof(float);
}

cudaError_t conv3d_wgrad_tile(const nm_conv3d_desc& d, const void* x, const void* dy, float* dw, float* db,
                              void* workspace, uint32_t* status, cudaStream_t s) {
  // input-channel atoms per MMA: as many as the input has, up to three
  const int nchunks = (d.c0 + 15) / 16;
  // one chunk: the three dy groups of a dz share an MMA, unless
  // NM_WGRAD_TILE_UNPACKED=1 (both forms are tested)
  const char* env = getenv("NM_WGRAD_TILE_UNPACKED");
  const bool dyp = !(env && env[0] == '1');
  if (d.cout == 16) {
    if (nchunks == 1 && dyp) return launch_wgrad_tile<16, 1, true>(d, x, dy, dw, db, workspace, status, s);
    if (nchunks == 1) return launch_wgrad_tile<16, 1>(d, x, dy, dw, db, workspace, status, s);
    if (nchunks == 2) return launch_wgrad_tile<16, 2>(d, x, dy, dw, db, workspace, status, s);
    return launch_wgrad_tile<16, 3>(d, x, dy, dw, db, workspace, status, s);
  }
  if (nchunks == 1 && dyp) return launch_wgrad_tile<32, 1, true>(d, x, dy, dw, db, workspace, status, s);
  if (nchunks == 1) return launch_wgrad_tile<32, 1>(d, x, dy, dw, db, workspace, status, s);
  if (nchunks == 2) return launch_wgrad_tile<32, 2>(d, x, dy, dw, db, workspace, status, s);
  return launch_wgrad_tile<32, 3>(d, x, dy, dw, db, workspace, status, s);
}

}  // namespace nm
