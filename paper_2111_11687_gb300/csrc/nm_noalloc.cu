// nm_dose_tally_noalloc: the whole tally computation (voxel packing, alias
// table, transport) for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or arena (where a stray cudaMalloc fragments or
// escapes the pool's accounting), real-time or safety-constrained services
// that forbid allocation after start-up, and hosts that hand the library only
// pre-allocated buffers.  For them this entry point takes device inputs and a
// device output and keeps all of its working memory in one file-scope device
// array of fixed size, so it allocates nothing.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "nm_internal.cuh"

using namespace nm;

namespace {

// Grids up to 64^3 voxels.  The array is about 24 MiB and every GPU that loads
// the library keeps it until the process exits.
constexpr int64_t kMaxVoxels = int64_t(1) << 18;
constexpr size_t kScratchBytes = size_t(24) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
CUcontext g_scratch_ctx[kMaxDevices] = {nullptr};

nm_status fail(nm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_error_message(buf);
  return st;
}

nm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(NM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// True for device memory of the current device, or managed memory.  Memory
// of another GPU is refused: this call has no handle that names a device, so
// every pointer must belong to the one that is current.
bool on_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

double kn_sigma(double e_mev) {
  const double k = e_mev / kElectronMassMeV;
  const double a = 1.0 + 2.0 * k;
  const double l = std::log1p(2.0 * k);
  return 2.0 * M_PI * kClassicalRadiusCm * kClassicalRadiusCm *
         ((1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k) + l / (2.0 * k) -
          (1.0 + 3.0 * k) / (a * a));
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// The address of the scratch array on the current device.  Host code cannot
// use the array's name as a device address, so the address is looked up once
// per device, with that device current, and kept.  The entry is keyed by the
// device's current context as well: after cudaDeviceReset the runtime makes a
// new primary context and loads the module again, possibly at another
// address, and the lookup is then repeated instead of trusting the old one.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

static CUcontext current_context() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return (CtxGetCurrentFn)f;
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

static nm_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(NM_ERR_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  const CUcontext ctx = current_context();
  if (!g_scratch_ptr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = current_context();   // the lookup made the context current if it was not
  }
  *out = (unsigned char*)g_scratch_ptr[dev];
  return NM_OK;
}

extern "C" nm_status nm_dose_tally_noalloc(const nm_grid* g, const nm_materials* mt,
                                           const float* activity, const nm_options* opts,
                                           uint64_t n_decays, uint64_t seed, int64_t* tally,
                                           nm_counters* counters) {
  if (!g || !mt || !tally) return fail(NM_ERR_ARG, "grid, materials and tally are required");
  nm_options o;
  if (opts) o = *opts; else nm_options_default(&o);
  // The same checks as nm_dose_create (sizes, spacing, constants, energies),
  // before anything below derives fixed-point units or table sizes from them.
  const nm_status cp = check_problem(g, mt, o, activity);
  if (cp != NM_OK) return cp;
  const int64_t V = (int64_t)g->nx * g->ny * g->nz;
  if (V > kMaxVoxels)
    return fail(NM_ERR_ARG, "grid of %lld voxels exceeds the no-allocation limit of %lld voxels",
                (long long)V, (long long)kMaxVoxels);
  const bool decay = o.source_mode == NM_SOURCE_DECAY;
  int cur = 0;
  cudaError_t ce = cudaGetDevice(&cur);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
  if (!on_device(g->density, cur) || !on_device(g->material, cur) || !on_device(tally, cur) ||
      (decay && !on_device(activity, cur)))
    return fail(NM_ERR_ARG,
                "density, material, tally (and activity in decay mode) must be memory of the current device");
  if (o.beta_max_mev != 0.0 || o.n_beta != 0 || o.n_gamma != 0 || o.no_annihilation != 0)
    return fail(NM_ERR_ARG, "beta spectra, gamma lines and other radionuclides need a handle (nm_dose_create)");
  const int32_t q_e0 = q_units((float)o.photon_mev);
  const int32_t q_pos = decay ? q_units((float)o.positron_mev) : 0;
  const uint64_t per = decay ? 2ull * q_e0 + q_pos : (uint64_t)q_e0;
  if (n_decays > (uint64_t)INT64_MAX / per) return fail(NM_ERR_OVERFLOW, "too many histories for the int64 tally");

  unsigned char* base = nullptr;
  nm_status st = scratch_for_current_device(&base);
  if (st != NM_OK) return st;
  // Carve the scratch array.
  size_t off = 0;
  auto take = [&](size_t bytes) { unsigned char* p = base + off; off += up256(bytes); return p; };
  uint32_t* vox = (uint32_t*)take(4 * V);
  uint4* alias = (uint4*)take(16 * V);
  float* kn_d = (float*)take(4 * kKnTable);
  float* minv_d = (float*)take(8 * kKnTable);     // whole grid, then outside the tracking box
  int* box_d = (int*)take(64);
  ull* ctr_d = (ull*)take(sizeof(ull) * kCtrCount);
  unsigned* work = (unsigned*)take(sizeof(unsigned));
  uint32_t* status = (uint32_t*)take(sizeof(uint32_t));
  uint32_t* rho_bits_d = (uint32_t*)take(4 * NM_MAX_MATERIALS);
  float* kn_inv_d = (float*)take(sizeof(float) * kKnInvE * (kKnInvU + 1));
  void* alias_scratch = take(AliasScratch::bytes(V));
  if (off > kScratchBytes) return fail(NM_ERR_ARG, "grid too large for the no-allocation scratch");

  cudaStream_t s = (cudaStream_t)o.stream;
  cudaError_t e;
  // Everything read below must start at zero: the array keeps the previous call's contents.
  if ((e = cudaMemsetAsync(ctr_d, 0, sizeof(ull) * kCtrCount, s)) ||
      (e = cudaMemsetAsync(status, 0, 4, s)) ||
      (e = cudaMemsetAsync(rho_bits_d, 0, 4 * NM_MAX_MATERIALS, s)) ||
      (e = launch_pack_voxels(g->density, g->material, V, mt->n, vox, rho_bits_d, status, s)))
    return cuda_fail(e, "voxel packing");
  uint32_t rho_bits[NM_MAX_MATERIALS] = {0};
  uint32_t flags = 0;
  if ((e = cudaMemcpyAsync(rho_bits, rho_bits_d, sizeof rho_bits, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(&flags, status, 4, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "voxel packing");
  if (flags & NM_DEV_BAD_VOXEL) return fail(NM_ERR_ARG, "density must be finite and > 0 and material < %d", mt->n);

  // Physics tables on the stack: Klein-Nishina per electron times N_A on the
  // log-energy grid, and the per-bin inverse majorant.
  TransportParams p;
  memset(&p, 0, sizeof p);
  const double e_lo = 0.5 * mt->photon_cut_mev, e_hi = 1.05 * o.photon_mev;
  const double dln = (std::log(e_hi) - std::log(e_lo)) / (kKnTable - 1);
  float kn[kKnTable], minv[2 * kKnTable];
  for (int i = 0; i < kKnTable; ++i) kn[i] = (float)(kAvogadro * kn_sigma(std::exp(std::log(e_lo) + i * dln)));
  for (int m = 0; m < mt->n; ++m) {
    p.mat[m].za = (float)mt->z_over_a[m];
    p.mat[m].zp = (float)(mt->pe_coeff * std::pow(mt->zeff[m], mt->pe_exp));
    p.mat[m].zr = mt->rayleigh ? (float)(mt->rayleigh_coeff * mt->zeff[m] * mt->zeff[m]) : 0.0f;
    memcpy(&p.mat[m].rho_max, &rho_bits[m], 4);
  }
  float rho_max[NM_MAX_MATERIALS], rho_out[NM_MAX_MATERIALS];
  for (int m = 0; m < NM_MAX_MATERIALS; ++m) rho_max[m] = p.mat[m].rho_max;
  if ((e = woodcock_regions(vox, g->nx, g->ny, g->nz, box_d, (uint32_t*)(box_d + 8), p.g.blo, p.g.bhi, rho_out, s)))
    return cuda_fail(e, "tracking regions");
  majorant_table(p.mat, mt->n, rho_max, kn, e_lo, dln, minv);
  majorant_table(p.mat, mt->n, rho_out, kn, e_lo, dln, minv + kKnTable);
  if ((e = cudaMemcpyAsync(kn_d, kn, sizeof kn, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(minv_d, minv, sizeof minv, cudaMemcpyHostToDevice, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "physics tables");
  if (o.kn_sampler == 0) {
    const std::vector<float>& kt = kn_inverse_cdf(mt->photon_cut_mev, o.photon_mev);
    if ((e = cudaMemcpyAsync(kn_inv_d, kt.data(), kt.size() * sizeof(float), cudaMemcpyHostToDevice, s)) ||
        (e = cudaStreamSynchronize(s)))
      return cuda_fail(e, "Klein-Nishina table");
    p.kn_inv = kn_inv_d;
    p.kn_inv_lo = (float)std::log(mt->photon_cut_mev);
    p.kn_inv_idln = (float)((kKnInvE - 1) / (std::log(o.photon_mev) - std::log(mt->photon_cut_mev)));
  }

  int64_t n_active = 0;
  if (decay) {
    if ((e = build_alias_table(activity, V, AliasScratch{alias_scratch}, alias, &n_active, status, s)) ||
        (e = cudaMemcpyAsync(&flags, status, 4, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
      return cuda_fail(e, "alias table");
    if (flags & NM_DEV_BAD_ACTIVITY) return fail(NM_ERR_ARG, "activity must be finite and >= 0");
    if (n_active == 0) return fail(NM_ERR_ARG, "activity map sums to zero");
  }

  p.g.vox = vox;
  p.g.alias = alias;
  p.g.tally = (ull*)tally;
  p.g.counters = ctr_d;
  p.g.work = work;
  p.g.n_active = (uint64_t)n_active;
  p.g.nx = g->nx; p.g.ny = g->ny; p.g.nz = g->nz;
  p.g.fnx = (float)g->nx; p.g.fny = (float)g->ny; p.g.fnz = (float)g->nz;
  p.g.inv_dx = 1.0f / g->dx; p.g.inv_dy = 1.0f / g->dy; p.g.inv_dz = 1.0f / g->dz;
  p.g.source_mode = o.source_mode;
  p.g.px = o.point[0] / g->dx; p.g.py = o.point[1] / g->dy; p.g.pz = o.point[2] / g->dz;
  p.g.q_positron = q_pos;
  p.annihilate = 1;
  p.status = status;
  p.kn = kn_d;
  p.minv = minv_d;
  p.minv_out = minv_d + kKnTable;
  p.key = philox_key((uint32_t)seed, (uint32_t)(seed >> 32));
  p.e0 = (float)o.photon_mev;
  p.q_e0 = q_e0;
  p.cut = (float)mt->photon_cut_mev;
  p.n_mat = mt->n;
  p.ln_e_lo = (float)std::log(e_lo);
  p.inv_dln_e = (float)(1.0 / dln);
  p.chunk = 256;
  p.max_steps = o.max_steps;
  p.regroup_compton = p.regroup_refill = 12;
  const bool warp_agg = !decay, rayleigh = mt->rayleigh != 0, regroup = true;
  const int block = 256;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    return cuda_fail(e, "device query");
  const int per_sm = transport_max_blocks_per_sm(block, warp_agg, rayleigh, regroup);
  if (per_sm <= 0) return fail(NM_ERR_CUDA, "transport kernel cannot be launched");

  if ((e = cudaMemsetAsync(tally, 0, 8 * V, s))) return cuda_fail(e, "tally clear");
  for (uint64_t done = 0; done < n_decays;) {
    const uint64_t part = std::min<uint64_t>(n_decays - done, 1ull << 31);
    p.g.hist_begin = done;
    p.g.n_hist = part;
    if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned), s)) ||
        (e = launch_transport(p, per_sm * sms, block, warp_agg, rayleigh, regroup, s)))
      return cuda_fail(e, "transport");
    done += part;
  }
  ull c[kCtrCount];
  if ((e = cudaMemcpyAsync(c, ctr_d, sizeof c, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(&flags, status, 4, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "transport");
  if (counters) {
    memset(counters, 0, sizeof *counters);
    counters->histories = n_decays;
    counters->emitted = (int64_t)(n_decays * per);
    counters->escaped = (int64_t)c[kCtrEscapedUnits];
    counters->killed = (int64_t)c[kCtrKilledUnits];
    counters->steps = c[kCtrSteps];
    counters->compton = c[kCtrCompton];
    counters->photo = c[kCtrPhoto];
    counters->rayleigh = c[kCtrRayleigh];
    counters->cutoff = c[kCtrCutoff];
    counters->escapes = c[kCtrEscapes];
    counters->deposited = counters->emitted - counters->escaped - counters->killed;
    counters->device_status = flags;
    counters->block_threads = block;
    counters->chunk = p.chunk;
    counters->warp_aggregate = warp_agg;
    counters->regroup = regroup;
    counters->regroup_lanes = p.regroup_compton;
    counters->grid_blocks = per_sm * sms;
  }
  if (flags) return fail(NM_ERR_DEVICE, "device check fired (flags 0x%x)", flags);
  return NM_OK;
}
