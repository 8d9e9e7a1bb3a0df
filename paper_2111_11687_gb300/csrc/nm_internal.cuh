// Internal declarations shared by the CUDA translation units of libnmdose.
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

#include "nm_dose.h"

namespace nm {

typedef unsigned long long ull;

constexpr float kInvElectronMassMeV = 1.0f / 0.51099895f;  // 1 / m_e c^2
constexpr double kElectronMassMeV = 0.51099895;
constexpr double kClassicalRadiusCm = 2.8179403262e-13;
constexpr double kAvogadro = 6.02214076e23;
constexpr double kJoulePerEv = 1.602176634e-19;
constexpr float kTwoPi = 6.283185307179586f;
constexpr int kKnTable = 1024;      // log-energy nodes of the Klein-Nishina table
constexpr int kFoldThreads = 128;   // fold / finalize CTA size
constexpr int kFoldTile = 8192;     // voxels per fold CTA
constexpr int kLabelSlots = NM_MAX_LABELS + 1;

// Fixed-point energy: round-to-nearest-even of the FP32 product E * 6.4e7.
// Deposits are differences of these values, so energy bookkeeping is exact
// whatever the rounding.
__host__ __device__ inline int32_t q_units(float e_mev) {
#ifdef __CUDA_ARCH__
  return __float2int_rn(__fmul_rn(e_mev, 64.0e6f));
#else
  const float p = e_mev * 64.0e6f;
  return (int32_t)__builtin_rintf(p);
#endif
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// -> 64-bit multiplies with the key bumped by the Weyl constants between rounds.
// The bumped keys depend on the seed alone, so they are formed once per launch
// (PhiloxKey, in the kernel's parameters): each round then XORs a parameter
// word instead of first adding a Weyl constant to a register.
// ---------------------------------------------------------------------------
struct PhiloxKey {
  uint32_t rk[20];            // round r: (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85) at 2r, 2r + 1
};

__host__ __device__ inline PhiloxKey philox_key(uint32_t k0, uint32_t k1) {
  PhiloxKey k;
  for (int r = 0; r < 10; ++r) {
    k.rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
    k.rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
  return k;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKey& k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.rk[2 * r], lo1, hi0 ^ c.w ^ k.rk[2 * r + 1], lo0);
  }
  return c;
}

// Uniform float in the open interval (0, 1) from 23 random bits.
__device__ __forceinline__ float u01(uint32_t r) { return ((float)(r >> 9) + 0.5f) * 0x1p-23f; }

// Random-stream ids inside one history: gamma line j flies on stream
// kStreamGamma0 + j after the emission draws of kStreamGammaSelect.
enum : uint32_t {
  kStreamSource = 0, kStreamPhotonA = 1, kStreamPhotonB = 2, kStreamPositron = 3, kStreamGammaSelect = 4,
  kStreamGamma0 = 8
};
constexpr int kMaxGammaLines = 8;
constexpr int kMaxBetaBranches = 8;
constexpr int kBetaTable = 1024;   // inverse-CDF nodes of the beta+ spectrum (+1)
// Klein-Nishina inverse CDF of x = 1 - cos(theta): kKnInvE energies (log
// spaced from the photon cutoff to the source energy) x kKnInvU + 1
// cumulative-probability nodes.
constexpr int kKnInvE = 64, kKnInvU = 256;

struct MaterialCoef {
  float za;       // (Z/A) * N_A * sigma-table scale: mu_c/rho = za * kn(E)
  float zp;       // pe_coeff * Zeff^pe_exp:            mu_pe/rho = zp / E^3
  float zr;       // rayleigh_coeff * Zeff^2:           mu_R/rho = zr / E^2
  float rho_max;  // largest density of this material in the grid (host side)
};

// Per-patient (per-grid) part of a transport launch.
struct PatientGeom {
  const uint32_t* vox;        // packed voxel: density bits with the low 3 bits = material
  const uint4* alias;         // {prob bits, voxel, alias voxel, 0}
  ull* tally;                 // batch tally, units
  ull* counters;              // device counters (see CounterSlot)
  unsigned* work;             // histories handed out in this launch (< 2^32 per launch)
  uint64_t n_active;
  uint64_t hist_begin;        // first global history id of this launch
  uint64_t n_hist;            // histories in this launch
  int nx, ny, nz;
  float fnx, fny, fnz;        // grid size as float (voxel units)
  float inv_dx, inv_dy, inv_dz;
  int source_mode;
  float px, py, pz;           // point source, voxel units
  int32_t q_positron;         // q_units(positron energy), 0 in point mode and with beta_tab
  // Beta+ spectrum (decay mode, optional): positron kinetic energy (MeV) at
  // cumulative probability i / kBetaTable, i = 0..kBetaTable; NULL = the
  // constant local deposit q_positron.
  const float* beta_tab;
  // Two-region Woodcock tracking: the box [blo, bhi) (voxel units) holds every
  // voxel denser than kRegionDensity plus a one-voxel margin; outside it the
  // majorant is TransportParams::minv_out.
  float blo[3], bhi[3];
};

struct TransportParams {
  PatientGeom g;              // the patient of a single-patient launch
  const PatientGeom* patients;  // multi-patient launch: n_patients entries (device memory)
  int n_patients;
  uint32_t* status;           // NM_DEV_* flags
  const float* kn;            // kKnTable nodes of N_A * sigma_KN(E)
  const float* minv;          // kKnTable bins: 1 / majorant (cm) on [E_i, E_i+1)
  const float* minv_out;      // the same outside the tracking box (much larger)
  const float* kn_inv;        // Klein-Nishina inverse CDF [kKnInvE][kKnInvU + 1]; NULL = Kahn's sampler
  float kn_inv_lo, kn_inv_idln; // ln of its first energy, 1 / its ln-energy step
  PhiloxKey key;              // round keys of the Philox key = seed
  float e0;                   // photon energy, MeV
  int32_t q_e0;               // q_units(e0)
  float cut;                  // photon cutoff, MeV
  int n_mat;
  MaterialCoef mat[NM_MAX_MATERIALS];
  float ln_e_lo, inv_dln_e;   // table grid: ln E = ln_e_lo + i / inv_dln_e
  int chunk;                  // histories per warp work grab
  int max_steps;
  int regroup_compton;        // regrouped variant: lanes that must wait before a Compton pass
  int regroup_refill;         // regrouped variant: lanes that must wait before a refill pass
  // History-by-history statistics (single-patient launches): per voxel the
  // 128-bit sum over histories of each history's squared total deposit.
  ull* s2h_lo;
  ull* s2h_hi;
  // Decay of another radionuclide (single-patient launches, the nuclide
  // variant): whether the annihilation pair is emitted, and the gamma lines
  // (energy, fixed-point energy, emission probability per decay).
  int annihilate;
  int n_gamma;
  float gamma_e[kMaxGammaLines];
  int32_t gamma_q[kMaxGammaLines];
  float gamma_y[kMaxGammaLines];
};

constexpr int kHistVoxels = 16;     // voxels a lane keeps per history (history statistics)

constexpr int kMaxBatchPatients = 64;

enum CounterSlot {
  kCtrSteps = 0, kCtrCompton, kCtrPhoto, kCtrRayleigh, kCtrCutoff, kCtrEscapes,
  kCtrEscapedUnits, kCtrKilledUnits, kCtrDepositedUnits, kCtrHistSplits, kCtrPositronUnits, kCtrGammaUnits,
  kCtrCount
};

// Sets the message that nm_last_error() returns on the calling thread.
void set_error_message(const char* msg);

// Argument checks shared by nm_dose_create and nm_dose_tally_noalloc (grid,
// materials, energies, options; nothing about where the pointers live).
// NM_OK, or NM_ERR_ARG with the message set.
nm_status check_problem(const nm_grid* g, const nm_materials* mt, const nm_options& o, const float* activity);

// ---- launchers (host side), one translation unit each ---------------------
// history: history-by-history statistics (needs !warp_agg and !multi); a
// single-patient launch whose p.g.beta_tab is set runs the beta+ variant
// (needs !warp_agg).
cudaError_t launch_transport(const TransportParams& p, int grid, int block, bool warp_agg,
                             bool rayleigh, bool regroup, cudaStream_t s, bool multi = false,
                             bool history = false);
// True for a single-patient launch that needs the nuclide variant (a beta
// spectrum, gamma lines or no annihilation pair).
bool nuclide_launch(const TransportParams& p);
// Per-voxel time-integrated activity (trapezoid between time points, linear
// uptake before the first, physical decay after the last), FP64 per voxel.
cudaError_t launch_time_integral(const float* const* act, const double* t_s, int n, int64_t V, double tail_s,
                                 float* out, double* block_sums, int blocks, cudaStream_t s);
int transport_max_blocks_per_sm(int block, bool warp_agg, bool rayleigh, bool regroup,
                                bool multi = false, bool history = false, bool beta = false);
cudaError_t launch_check_philox(const uint4* ctr, const uint2* key, int64_t n, uint4* out,
                                cudaStream_t s);
// Klein-Nishina inverse-CDF table [kKnInvE][kKnInvU + 1] of x = 1 - cos(theta)
// for photons between e_lo and e_hi (MeV), built in FP64 on the host once per
// pair and kept (thread-safe; the reference stays valid).
const std::vector<float>& kn_inverse_cdf(double e_lo, double e_hi);

cudaError_t launch_check_wait(long long max_cycles, uint32_t* status, cudaStream_t s);
cudaError_t launch_check_kn_table(const TransportParams& p, float e, int64_t n, float* out, cudaStream_t s);
cudaError_t launch_check_beta(const float* tab, int64_t n, uint32_t k0, uint32_t k1, float* out, cudaStream_t s);
cudaError_t launch_check_kahn(float e, int64_t n, uint32_t k0, uint32_t k1, float* out,
                              uint32_t* status, cudaStream_t s);
cudaError_t launch_check_source(const TransportParams& p, uint64_t first, int64_t n, int32_t* voxel,
                                float* pos, float* dir, cudaStream_t s);

// HU -> density/material (§2.1).
cudaError_t launch_ct_to_phantom(const int16_t* hu, int64_t n, float* density, uint8_t* material,
                                 cudaStream_t s);

// Woodcock regions of a packed grid: the tracking box [blo, bhi) in voxel
// units (the voxels denser than kRegionDensity, one voxel of margin, clamped to
// the grid; empty when there are none) and the per-material largest density
// outside the unpadded box.  box_dev (6 ints) and rho_dev (NM_MAX_MATERIALS
// words) are device scratch; synchronises the stream.
constexpr float kRegionDensity = 0.05f;   // g/cm^3: denser than any air, lighter than lung
cudaError_t woodcock_regions(const uint32_t* vox, int nx, int ny, int nz, int* box_dev, uint32_t* rho_dev,
                             float blo[3], float bhi[3], float rho_out[NM_MAX_MATERIALS], cudaStream_t s);
// Per-bin inverse majorant (cm) for the materials at densities rho[m]: every
// mu/rho decreases with E, so the value at a bin's lower edge bounds the bin.
// FP64 from the FP32 coefficients the kernel uses, 1e-4 margin for the
// kernel's FP32 rounding, reciprocal rounded down; an empty region gets a
// finite 1e12 cm.
void majorant_table(const MaterialCoef* mat, int n_mat, const float* rho, const float* kn, double e_lo, double dln,
                    float* minv);

// Voxel packing and validation; per-material maximum density (as float bits).
cudaError_t launch_pack_voxels(const float* density, const uint8_t* material, int64_t V, int n_mat,
                               uint32_t* vox, uint32_t* rho_max_bits, uint32_t* status,
                               cudaStream_t s);

// Alias table over the positive entries of activity[V] in FP64 on the device.
// Scratch is owned by the caller (AliasScratch::bytes(V)).
struct AliasScratch {
  static size_t bytes(int64_t V);
  void* base;
};
cudaError_t build_alias_table(const float* activity, int64_t V, AliasScratch scratch, uint4* table,
                              int64_t* n_active_host, uint32_t* status, cudaStream_t s);

// Batch fold (per batch) and finalize.
struct FoldParams {
  ull* tb;                  // batch tally, zeroed by the fold
  ull* tsum;                // cumulative tally
  double* s2;               // sum over batches of T_b^2 / n_b
  const float* density;
  const uint8_t* labels;    // may be NULL
  int64_t V;
  double n_b;               // histories in this batch
  double gy_per_unit_vol;   // J per unit / (1e-3 kg/g * voxel volume cm^3)
  double* organ_partial;    // [blocks][kLabelSlots]
  double* org_s1;           // [kLabelSlots] sum_b O_b
  double* org_s2;           // [kLabelSlots] sum_b O_b^2 / n_b
  ull* deposited;           // counter
};
int fold_blocks(int64_t V);
cudaError_t launch_fold(const FoldParams& p, cudaStream_t s);

// Adds another shard's statistics (o_*) into a handle's (all device arrays;
// s2h_lo/hi and o_lo/hi NULL without history statistics).
struct MergeParams {
  ull* tsum; double* s2; ull* s2h_lo; ull* s2h_hi; double* org_s1; double* org_s2; ull* counters;
  const ull* o_tsum; const double* o_s2; const ull* o_lo; const ull* o_hi;
  const double* o_org_s1; const double* o_org_s2; const ull* o_counters;
  int64_t V;
};
cudaError_t launch_merge_stats(const MergeParams& m, int sms, cudaStream_t s);

struct FinalizeParams {
  const ull* tsum;
  const double* s2;
  const float* density;
  const uint8_t* labels;
  int64_t V;
  double n_total;           // histories
  double n_batches;         // K
  double gy_per_unit_vol;
  double activity_bq;
  float* dose;              // may be NULL
  float* sigma;             // may be NULL
  double* organ_partial;    // [blocks][2][kLabelSlots]
  const double* org_s1;
  const double* org_s2;
  const long long* organ_count;  // [kLabelSlots]
  double* organ_out;        // [4][kLabelSlots]: mean, eps_rms, sigma_mean, count
};
// Eq. 1 dose rate only into p.dose (bit-identical to launch_finalize's).
cudaError_t launch_dose_only(const FinalizeParams& p, int sms, cudaStream_t s);
cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t s);
// Voxels per label into count[kLabelSlots] (labels >= kLabelSlots count as 0),
// and atomicMin of first_bad with every voxel index whose label exceeds n_labels.
cudaError_t launch_label_count(const uint8_t* labels, int64_t V, int n_labels, long long* count,
                               unsigned long long* first_bad, cudaStream_t s);
// History-by-history sigma of the mean dose rate: sigma[v] = sqrt((S2/N -
// (T/N)^2) / (N - 1)) * gy_a / density[v], S2 = hi * 2^64 + lo.
cudaError_t launch_history_sigma(const ull* tsum, const ull* s2h_lo, const ull* s2h_hi, const float* density,
                                 int64_t V, double n_total, double gy_a, float* sigma, cudaStream_t s);
cudaError_t launch_map_organ_means(const float* dose, const uint8_t* labels, int64_t V, double* part,
                                   const long long* count, double* out, cudaStream_t s);

// ---- 3x3x3 convolution on the tensor cores (nm_conv.cu) -------------------
int conv_kpad(int cin);
bool conv_geom_ok(const nm_conv3d_desc& d);
int conv_wgrad_splits(const nm_conv3d_desc& d);
size_t conv_wgrad_workspace(const nm_conv3d_desc& d);
cudaError_t conv3d_fwd(const nm_conv3d_desc& d, const void* x0, const void* x1, const void* w,
                       const float* bias, void* y, int relu, uint32_t* status, cudaStream_t s);
bool conv_tile_ok(const nm_conv3d_desc& d);
cudaError_t conv3d_fwd_tile(const nm_conv3d_desc& d, const void* x, const void* w, const float* bias, void* y,
                            int relu, uint32_t* status, cudaStream_t s);
// The same with the denoiser's 1x1x1 head fused into the epilogue (16
// outputs, ReLU): yh[v] = head_w[16] + xin[v][0] + sum_c head_w[c] act[v][c].
cudaError_t conv3d_fwd_tile_head(const nm_conv3d_desc& d, const void* x, const void* w, const float* bias,
                                 const float* head_w, const void* xin, int cx, float* yh, uint32_t* status,
                                 cudaStream_t s);
cudaError_t conv3d_flip_weights(const nm_conv3d_desc& d, const void* w, void* wb, cudaStream_t s);
// Shifted-window weight gradient (nm_wgrad_tile.cu): single source, 16 or 32 outputs.
bool conv_wgrad_tile_ok(const nm_conv3d_desc& d);
size_t conv_wgrad_tile_workspace(const nm_conv3d_desc& d);
cudaError_t conv3d_wgrad_tile(const nm_conv3d_desc& d, const void* x, const void* dy, float* dw, float* db,
                              void* workspace, uint32_t* status, cudaStream_t s);
cudaError_t conv3d_wgrad(const nm_conv3d_desc& d, const void* x0, const void* x1, const void* dy,
                         float* dw, float* db, void* workspace, uint32_t* status, cudaStream_t s);

}  // namespace nm
