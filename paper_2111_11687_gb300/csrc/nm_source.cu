// Phantom and source set-up (§2.1): CT numbers to density/material, voxel
// packing, and the decay sampler's alias table built in FP64 on the device.
//
// Alias table (Walker's method) without a serial stack: with weights
// normalised to mean 1, "light" columns (w < 1) have a deficit 1 - w and
// "heavy" ones a surplus w - 1.  Sweeping lights and heavies in index order,
// the current heavy absorbs the lights' deficits and, once its own weight
// drops below 1, becomes a column itself that borrows from the next heavy.
// In prefix-sum form (D_k: deficits of lights 1..k, S_m: surpluses of heavies
// 1..m) the sweep has a closed form that every column evaluates on its own:
//   light k:  prob = w, alias = heavy m with m = min{m : S_m >= D_(k-1)};
//   heavy m:  with k = min{k : D_k > S_m}: prob = 1 - (D_k - S_m),
//             alias = heavy m+1 (prob 1 if no such k, or for the last heavy).
// Each item's probability mass then sums to its weight exactly.  The scans
// use a fixed reduction tree, so the table is the same on every run.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "nm_internal.cuh"

namespace nm {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// ---- CT -> phantom ----------------------------------------------------------
__constant__ int c_node_hu[5] = {-1000, -750, -100, 40, 1000};
__constant__ float c_node_rho[5] = {0.0012f, 0.26f, 0.95f, 1.03f, 1.85f};

__global__ void ct_to_phantom_kernel(const int16_t* __restrict__ hu, int64_t n,
                                     float* __restrict__ density, uint8_t* __restrict__ material) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int h = hu[i];
    float rho;
    if (h <= c_node_hu[0]) {
      rho = c_node_rho[0];
    } else if (h >= c_node_hu[4]) {
      rho = c_node_rho[4];
    } else {
      int s = 0;
      while (h > c_node_hu[s + 1]) ++s;
      const float f = (float)(h - c_node_hu[s]) / (float)(c_node_hu[s + 1] - c_node_hu[s]);
      rho = fmaf(f, c_node_rho[s + 1] - c_node_rho[s], c_node_rho[s]);
    }
    // Nearest node in HU, ties to the lower node: 2h <= a + b picks a over b.
    int m = 0;
    while (m < 4 && 2 * h > c_node_hu[m] + c_node_hu[m + 1]) ++m;
    density[i] = rho;
    material[i] = (uint8_t)m;
  }
}

// ---- voxel packing ------------------------------------------------------------
__global__ void pack_voxels_kernel(const float* __restrict__ density,
                                   const uint8_t* __restrict__ material, int64_t V, int n_mat,
                                   uint32_t* __restrict__ vox, uint32_t* __restrict__ rho_max_bits,
                                   uint32_t* status) {
  __shared__ uint32_t s_max[NM_MAX_MATERIALS];
  if (threadIdx.x < NM_MAX_MATERIALS) s_max[threadIdx.x] = 0;
  __syncthreads();
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float rho = density[i];
    const uint32_t m = material[i];
    if (!(rho > 0.0f) || !(rho < 1e30f) || m >= (uint32_t)n_mat) {
      bad = true;
      vox[i] = 0x3f800000u;  // 1 g/cm^3 of material 0; the create call fails anyway
      continue;
    }
    // Density with its 3 lowest mantissa bits replaced by the material id:
    // relative change below 2^-20, one 32-bit load per flight step.
    const uint32_t w = (__float_as_uint(rho) & ~7u) | m;
    vox[i] = w;
    atomicMax(&s_max[m], w & ~7u);  // positive floats order like their bit patterns
  }
  if (bad) atomicOr(status, NM_DEV_BAD_VOXEL);
  __syncthreads();
  if (threadIdx.x < NM_MAX_MATERIALS && s_max[threadIdx.x])
    atomicMax(rho_max_bits + threadIdx.x, s_max[threadIdx.x]);
}

// ---- deterministic block scans -------------------------------------------------
template <class T>
__device__ T block_inclusive_scan(T v, T* warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  if (wid > 0) v += warp_tot[wid - 1];
  __syncthreads();
  return v;
}

// Tile sums: each thread sums kScanItems consecutive items in order.
template <class T, class Load>
__global__ void tile_sum_kernel(Load load, int64_t n, T* tile_sum) {
  __shared__ T wt[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j)
    if (base + j < n) s += load(base + j);
  s = block_inclusive_scan<T>(s, wt);
  if (threadIdx.x == blockDim.x - 1) tile_sum[blockIdx.x] = s;
}

// Exclusive scan of the tile sums in one block: thread t owns a contiguous run.
template <class T>
__global__ void tile_prefix_kernel(T* tile_sum, int64_t n_tiles, T* total) {
  __shared__ T wt[32];
  const int64_t per = (n_tiles + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = (int64_t)threadIdx.x * per;
  T s = T(0);
  for (int64_t i = b0; i < b0 + per && i < n_tiles; ++i) s += tile_sum[i];
  const T incl = block_inclusive_scan<T>(s, wt);
  T run = incl - s;
  for (int64_t i = b0; i < b0 + per && i < n_tiles; ++i) {
    const T v = tile_sum[i];
    tile_sum[i] = run;
    run += v;
  }
  if (threadIdx.x == blockDim.x - 1) *total = incl;
}

template <class T, class Load>
__global__ void tile_scan_kernel(Load load, int64_t n, const T* tile_prefix, T* out) {
  __shared__ T wt[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < n ? load(base + j) : T(0);
    s += v[j];
  }
  const T incl = block_inclusive_scan<T>(s, wt);
  T run = incl - s + tile_prefix[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    run += v[j];
    if (base + j < n) out[base + j] = run;
  }
}

// Inclusive scan out[i] = load(0) + ... + load(i); *total (device) = sum.
template <class T, class Load>
cudaError_t inclusive_scan(Load load, int64_t n, T* out, T* tiles, T* total, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(total, 0, sizeof(T), s);
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  tile_sum_kernel<T, Load><<<(unsigned)nt, kScanThreads, 0, s>>>(load, n, tiles);
  tile_prefix_kernel<T><<<1, 1024, 0, s>>>(tiles, nt, total);
  tile_scan_kernel<T, Load><<<(unsigned)nt, kScanThreads, 0, s>>>(load, n, tiles, out);
  return cudaGetLastError();
}

struct ActiveFlag {
  const float* a;
  __device__ int operator()(int64_t i) const { return a[i] > 0.0f ? 1 : 0; }
};
struct LightFlag {
  const double* w;
  __device__ int operator()(int64_t i) const { return w[i] < 1.0 ? 1 : 0; }
};
struct DoubleLoad {
  const double* x;
  __device__ double operator()(int64_t i) const { return x[i]; }
};
struct ActiveWeight {
  const float* a;
  const int32_t* vox;
  __device__ double operator()(int64_t i) const { return (double)a[vox[i]]; }
};

__global__ void check_activity_kernel(const float* a, int64_t V, uint32_t* status) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = a[i];
    if (!(x >= 0.0f) || !(x < 3.0e38f)) bad = true;
  }
  if (bad) atomicOr(status, NM_DEV_BAD_ACTIVITY);
}

__global__ void compact_active_kernel(const float* a, const int32_t* incl, int64_t V,
                                      int32_t* active_vox) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] > 0.0f) active_vox[incl[i] - 1] = (int32_t)i;
}

// w_i = A_i * n / W; split into lights and heavies in index order.
__global__ void classify_kernel(const float* a, const int32_t* active_vox, int64_t n,
                                const double* total, double* w) {
  const double scale = (double)n / *total;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (double)a[active_vox[i]] * scale;
}

__global__ void split_kernel(const double* w, const int32_t* light_incl, int64_t n,
                             int32_t* light_idx, double* light_def, int32_t* heavy_idx,
                             double* heavy_sur) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t li = light_incl[i];
    if (w[i] < 1.0) {
      light_idx[li - 1] = (int32_t)i;
      light_def[li - 1] = 1.0 - w[i];
    } else {
      const int64_t hi = i - li;
      heavy_idx[hi] = (int32_t)i;
      heavy_sur[hi] = w[i] - 1.0;
    }
  }
}

// first index j in [0, n) with x[j] >= t (n if none)
__device__ int64_t lower_bound(const double* x, int64_t n, double t) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (x[mid] < t) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// first index j in [0, n) with x[j] > t (n if none)
__device__ int64_t upper_bound(const double* x, int64_t n, double t) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (x[mid] <= t) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void light_columns_kernel(const double* w, const int32_t* light_idx, const double* D,
                                     int64_t a, const int32_t* heavy_idx, const double* S,
                                     int64_t b, const int32_t* active_vox, uint4* table) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = light_idx[k];
    if (b == 0) {
      // Rounding left every weight just below 1: the table is uniform.
      table[i] = make_uint4(__float_as_uint(1.0f), (uint32_t)active_vox[i], (uint32_t)active_vox[i], 0u);
      continue;
    }
    const double before = k > 0 ? D[k - 1] : 0.0;
    int64_t m = lower_bound(S, b, before);
    if (m >= b) m = b - 1;
    const float prob = (float)w[i];
    table[i] = make_uint4(__float_as_uint(prob), (uint32_t)active_vox[i],
                          (uint32_t)active_vox[heavy_idx[m]], 0u);
  }
}

__global__ void heavy_columns_kernel(const double* D, int64_t a, const int32_t* heavy_idx,
                                     const double* S, int64_t b, const int32_t* active_vox,
                                     uint4* table) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < b;
       m += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = heavy_idx[m];
    float prob = 1.0f;
    int32_t alias = i;
    if (m + 1 < b) {
      const int64_t k = upper_bound(D, a, S[m]);
      if (k < a) {
        const double p = 1.0 - (D[k] - S[m]);
        prob = (float)fmin(fmax(p, 0.0), 1.0);
        alias = heavy_idx[m + 1];
      }
    }
    table[i] = make_uint4(__float_as_uint(prob), (uint32_t)active_vox[i],
                          (uint32_t)active_vox[alias], 0u);
  }
}

__global__ void region_box_kernel(const uint32_t* __restrict__ vox, int nx, int ny, int nz, float thresh,
                                  int* box) {
  // box: [xmin, ymin, zmin, xmax, ymax, zmax]
  int lo[3] = {nx, ny, nz}, hi[3] = {-1, -1, -1};
  const long long V = (long long)nx * ny * nz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    if (__uint_as_float(vox[i] & ~7u) > thresh) {
      const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
      lo[0] = min(lo[0], x); lo[1] = min(lo[1], y); lo[2] = min(lo[2], z);
      hi[0] = max(hi[0], x); hi[1] = max(hi[1], y); hi[2] = max(hi[2], z);
    }
  }
  for (int a = 0; a < 3; ++a) {
    lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
    hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
  }
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; ++a) {
      atomicMin(box + a, lo[a]);
      atomicMax(box + 3 + a, hi[a]);
    }
}

__global__ void region_rho_out_kernel(const uint32_t* __restrict__ vox, int nx, int ny, int nz, int x0, int y0,
                                      int z0, int x1, int y1, int z1, uint32_t* rho_max_bits) {
  __shared__ uint32_t s_max[NM_MAX_MATERIALS];
  if (threadIdx.x < NM_MAX_MATERIALS) s_max[threadIdx.x] = 0;
  __syncthreads();
  const long long V = (long long)nx * ny * nz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
    if (x >= x0 && x <= x1 && y >= y0 && y <= y1 && z >= z0 && z <= z1) continue;
    const uint32_t w = vox[i];
    atomicMax(&s_max[w & 7u], w & ~7u);
  }
  __syncthreads();
  if (threadIdx.x < NM_MAX_MATERIALS && s_max[threadIdx.x]) atomicMax(rho_max_bits + threadIdx.x, s_max[threadIdx.x]);
}

// Voxels per label, and the lowest voxel index whose label exceeds n_labels
// (first_bad keeps its initial value when there is none).
__global__ void label_count_kernel(const uint8_t* labels, int64_t V, int n_labels, long long* count,
                                   ull* first_bad) {
  __shared__ long long s[kLabelSlots];
  if (threadIdx.x < kLabelSlots) s[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int l = labels[i];
    if (l > n_labels) atomicMin(first_bad, (ull)i);
    // neighbouring voxels mostly share a label: one shared-memory atomic per
    // distinct label of the warp instead of one per voxel
    const int slot = l < kLabelSlots ? l : 0;
    const unsigned peers = __match_any_sync(__activemask(), slot);
    if ((int)(threadIdx.x & 31u) == __ffs(peers) - 1) atomicAdd((ull*)&s[slot], (ull)__popc(peers));
  }
  __syncthreads();
  if (threadIdx.x < kLabelSlots && s[threadIdx.x])
    atomicAdd((ull*)(count + threadIdx.x), (ull)s[threadIdx.x]);
}

int grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

// Scratch layout for the alias build.
struct AliasBufs {
  int32_t *incl, *active_vox, *light_incl, *light_idx, *heavy_idx;
  double *w, *light_def, *heavy_sur, *D, *S, *wsum, *dtiles;
  int32_t *itiles, *itotal;
  double* dtotal;
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

AliasBufs carve(void* base, int64_t V) {
  const int64_t nt = (V + kScanTile - 1) / kScanTile + 1;
  char* p = (char*)base;
  AliasBufs b;
  auto take = [&](size_t bytes) { char* r = p; p += align_up(bytes); return (void*)r; };
  b.incl = (int32_t*)take(4 * V);
  b.active_vox = (int32_t*)take(4 * V);
  b.light_incl = (int32_t*)take(4 * V);
  b.light_idx = (int32_t*)take(4 * V);
  b.heavy_idx = (int32_t*)take(4 * V);
  b.w = (double*)take(8 * V);
  b.light_def = (double*)take(8 * V);
  b.heavy_sur = (double*)take(8 * V);
  b.D = (double*)take(8 * V);
  b.S = (double*)take(8 * V);
  b.wsum = (double*)take(8 * V);
  b.dtiles = (double*)take(8 * nt);
  b.itiles = (int32_t*)take(4 * nt);
  b.itotal = (int32_t*)take(4);
  b.dtotal = (double*)take(8 * 4);
  return b;
}

}  // namespace

size_t AliasScratch::bytes(int64_t V) {
  const int64_t nt = (V + kScanTile - 1) / kScanTile + 1;
  return align_up(4 * V) * 5 + align_up(8 * V) * 6 + align_up(8 * nt) + align_up(4 * nt) +
         align_up(4) + align_up(32);
}

cudaError_t launch_ct_to_phantom(const int16_t* hu, int64_t n, float* density, uint8_t* material,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ct_to_phantom_kernel<<<grid_for(n), 256, 0, s>>>(hu, n, density, material);
  return cudaGetLastError();
}

cudaError_t launch_pack_voxels(const float* density, const uint8_t* material, int64_t V, int n_mat,
                               uint32_t* vox, uint32_t* rho_max_bits, uint32_t* status,
                               cudaStream_t s) {
  pack_voxels_kernel<<<grid_for(V), 256, 0, s>>>(density, material, V, n_mat, vox, rho_max_bits,
                                                 status);
  return cudaGetLastError();
}

cudaError_t woodcock_regions(const uint32_t* vox, int nx, int ny, int nz, int* box_dev, uint32_t* rho_dev,
                             float blo[3], float bhi[3], float rho_out[NM_MAX_MATERIALS], cudaStream_t s) {
  const long long V = (long long)nx * ny * nz;
  const int init[6] = {nx, ny, nz, -1, -1, -1};
  int b[6];
  uint32_t bits[NM_MAX_MATERIALS];
  cudaError_t e = cudaMemcpyAsync(box_dev, init, sizeof init, cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemsetAsync(rho_dev, 0, sizeof bits, s);
  if (e) return e;
  region_box_kernel<<<grid_for(V), 256, 0, s>>>(vox, nx, ny, nz, kRegionDensity, box_dev);
  if ((e = cudaGetLastError()) || (e = cudaMemcpyAsync(b, box_dev, sizeof b, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return e;
  const int n[3] = {nx, ny, nz};
  const bool empty = b[3] < b[0];
  for (int a = 0; a < 3; ++a) {
    blo[a] = empty ? 0.0f : (float)std::max(b[a] - 1, 0);
    bhi[a] = empty ? 0.0f : (float)std::min(b[3 + a] + 2, n[a]);
  }
  region_rho_out_kernel<<<grid_for(V), 256, 0, s>>>(vox, nx, ny, nz, b[0], b[1], b[2], b[3], b[4], b[5], rho_dev);
  if ((e = cudaGetLastError()) || (e = cudaMemcpyAsync(bits, rho_dev, sizeof bits, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return e;
  for (int m = 0; m < NM_MAX_MATERIALS; ++m) memcpy(&rho_out[m], &bits[m], 4);
  return cudaSuccess;
}

void majorant_table(const MaterialCoef* mat, int n_mat, const float* rho, const float* kn, double e_lo, double dln,
                    float* minv) {
  for (int i = 0; i < kKnTable; ++i) {
    const double ei = std::exp(std::log(e_lo) + i * dln);
    double maj = 0.0;
    for (int m = 0; m < n_mat; ++m) {
      const double mu = (double)mat[m].za * (double)kn[i] + (double)mat[m].zp / (ei * ei * ei) +
                        (double)mat[m].zr / (ei * ei);
      maj = std::max(maj, (double)rho[m] * mu);
    }
    maj = std::max(maj * (1.0 + 1e-4), 1e-12);
    minv[i] = std::nextafter((float)(1.0 / maj), 0.0f);
  }
}

cudaError_t launch_label_count(const uint8_t* labels, int64_t V, int n_labels, long long* count,
                               unsigned long long* first_bad, cudaStream_t s) {
  label_count_kernel<<<grid_for(V), 256, 0, s>>>(labels, V, n_labels, count, first_bad);
  return cudaGetLastError();
}

cudaError_t build_alias_table(const float* activity, int64_t V, AliasScratch scratch, uint4* table,
                              int64_t* n_active_host, uint32_t* status, cudaStream_t s) {
  AliasBufs b = carve(scratch.base, V);
  cudaError_t e;
  check_activity_kernel<<<grid_for(V), 256, 0, s>>>(activity, V, status);
  // Active voxels (A > 0) in index order.
  if ((e = inclusive_scan<int32_t>(ActiveFlag{activity}, V, b.incl, b.itiles, b.itotal, s))) return e;
  int32_t n32 = 0;
  if ((e = cudaMemcpyAsync(&n32, b.itotal, 4, cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  const int64_t n = n32;
  *n_active_host = n;
  if (n == 0) return cudaSuccess;
  compact_active_kernel<<<grid_for(V), 256, 0, s>>>(activity, b.incl, V, b.active_vox);
  // Total weight W with the fixed-tree scan, then w_i = A_i n / W.
  if ((e = inclusive_scan<double>(ActiveWeight{activity, b.active_vox}, n, b.wsum, b.dtiles,
                                  b.dtotal, s)))
    return e;
  classify_kernel<<<grid_for(n), 256, 0, s>>>(activity, b.active_vox, n, b.dtotal, b.w);
  if ((e = inclusive_scan<int32_t>(LightFlag{b.w}, n, b.light_incl, b.itiles, b.itotal, s))) return e;
  int32_t a32 = 0;
  if ((e = cudaMemcpyAsync(&a32, b.itotal, 4, cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  const int64_t a = a32, hb = n - a32;
  split_kernel<<<grid_for(n), 256, 0, s>>>(b.w, b.light_incl, n, b.light_idx, b.light_def,
                                           b.heavy_idx, b.heavy_sur);
  if ((e = inclusive_scan<double>(DoubleLoad{b.light_def}, a, b.D, b.dtiles, b.dtotal + 1, s))) return e;
  if ((e = inclusive_scan<double>(DoubleLoad{b.heavy_sur}, hb, b.S, b.dtiles, b.dtotal + 2, s))) return e;
  if (a > 0)
    light_columns_kernel<<<grid_for(a), 256, 0, s>>>(b.w, b.light_idx, b.D, a, b.heavy_idx, b.S, hb,
                                                      b.active_vox, table);
  heavy_columns_kernel<<<grid_for(hb), 256, 0, s>>>(b.D, a, b.heavy_idx, b.S, hb, b.active_vox,
                                                    table);
  return cudaGetLastError();
}

}  // namespace nm
